// Toeplitz mode products by FFT (Sec. 3.1: on a regular grid each SE factor
// K_k is a symmetric Toeplitz matrix, K_k[a][b] = kappa_k(|a - b|), and FFTs
// give O(m log m) products with K_UU).
//
// K_k embeds as the leading m x m block of an L x L circulant C (L the
// smallest power of two >= 2m - 1) whose first column is
//   c = [kappa(0), .., kappa(m-1), 0, .., 0, kappa(m-1), .., kappa(1)];
// C = F^-1 diag(F c) F, so K_k x is the first m entries of
// IFFT(F c .* FFT(x zero-padded to L)).  F c is real (c is real and even).
//
// One CTA transforms two rows of the operand at once as one complex vector
// z = x_r + i x_{r+1}: the spectrum multiplier is real, so the inverse
// transform returns K x_r in the real part and K x_{r+1} in the imaginary
// part exactly (linearity), and no real-to-complex unpacking is needed.
// The forward transform is a decimation-in-frequency radix-2 pass (natural
// order in, bit-reversed out), the multiplier is stored bit-reversed, and the
// inverse is a decimation-in-time pass (bit-reversed in, natural out), so no
// permutation pass is needed.  Everything is FP64 in shared memory; the
// twiddles exp(-2 pi i j / L) come from sincospi once per factor.
//
// The output is written in the layout of the other mode products: contracted
// mode first (one step of the cyclic mode rotation), Y[j][r] = scale (K X)[r][j].
#include <cuda_runtime.h>

#include <algorithm>

#include "dski_internal.cuh"

namespace dski {
namespace {

constexpr int FFT_THREADS = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {   // a * conj(b)
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}

// forward DIF over z[0..L): natural order in, bit-reversed order out
__device__ void fft_dif(double2* z, int L, const double2* __restrict__ tw) {
  for (int h = L >> 1, ts = 1; h >= 1; h >>= 1, ts <<= 1) {
    for (int b = threadIdx.x; b < (L >> 1); b += blockDim.x) {
      const int j = b & (h - 1);
      const int i0 = ((b - j) << 1) + j;
      const double2 u = z[i0], v = z[i0 + h];
      z[i0] = make_double2(u.x + v.x, u.y + v.y);
      z[i0 + h] = cmul(make_double2(u.x - v.x, u.y - v.y), tw[j * ts]);
    }
    __syncthreads();
  }
}

// inverse DIT over z[0..L): bit-reversed order in, natural order out,
// unnormalised (the 1/L is folded into the multiplier)
__device__ void ifft_dit(double2* z, int L, const double2* __restrict__ tw) {
  for (int h = 1, ts = L >> 1; h < L; h <<= 1, ts >>= 1) {
    for (int b = threadIdx.x; b < (L >> 1); b += blockDim.x) {
      const int j = b & (h - 1);
      const int i0 = ((b - j) << 1) + j;
      const double2 u = z[i0], v = cmulc(z[i0 + h], tw[j * ts]);
      z[i0] = make_double2(u.x + v.x, u.y + v.y);
      z[i0 + h] = make_double2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
  }
}

// tw[j] = exp(-2 pi i j / L), j < L/2
__global__ void k_fft_twiddles(int L, double2* __restrict__ tw) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= (L >> 1)) return;
  double s, c;
  sincospi(-2.0 * (double)j / (double)L, &s, &c);
  tw[j] = make_double2(c, s);
}

// lam = (F c) / L in bit-reversed order, c the circulant column built from
// kappa = the first row of K_k (one CTA)
__global__ void k_fft_multiplier(const double* __restrict__ K, int m, int L,
                                 const double2* __restrict__ tw, double* __restrict__ lam) {
  extern __shared__ double2 zs[];
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    double v = 0.0;
    if (i < m) v = K[i];
    else if (i > L - m) v = K[L - i];
    zs[i] = make_double2(v, 0.0);
  }
  __syncthreads();
  fft_dif(zs, L, tw);
  const double inv = 1.0 / (double)L;
  for (int i = threadIdx.x; i < L; i += blockDim.x) lam[i] = zs[i].x * inv;
}

// Y_q[j][r] = scale sum_i K[j][i] X_q[r][i] for the row pair (r0, r0 + 1) of
// CTA blockIdx.x and column q = blockIdx.y; X_q is R x m (contracted mode
// contiguous), Y_q is m x R.
__global__ void __launch_bounds__(FFT_THREADS) k_mode_fft(const double* __restrict__ X,
                                                         const double2* __restrict__ tw,
                                                         const double* __restrict__ lam,
                                                         double* __restrict__ Y, int m, int L,
                                                         long long R, double scale) {
  extern __shared__ double2 zs[];
  const long long r0 = 2LL * blockIdx.x;
  const bool two = r0 + 1 < R;
  const long long qoff = (long long)blockIdx.y * R * m;
  const double* x0 = X + qoff + r0 * m;
  const double* x1 = two ? x0 + m : x0;
  for (int i = threadIdx.x; i < L; i += blockDim.x)
    zs[i] = i < m ? make_double2(x0[i], two ? x1[i] : 0.0) : make_double2(0.0, 0.0);
  __syncthreads();
  fft_dif(zs, L, tw);
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    const double l = lam[i];
    zs[i] = make_double2(zs[i].x * l, zs[i].y * l);
  }
  __syncthreads();
  ifft_dit(zs, L, tw);
  double* Yq = Y + qoff;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double2 v = zs[j];
    Yq[(long long)j * R + r0] = scale * v.x;
    if (two) Yq[(long long)j * R + r0 + 1] = scale * v.y;
  }
}

}  // namespace

int fft_circulant_size(int m) {
  int L = 1;
  while (L < 2 * m - 1) L <<= 1;
  return L;
}

size_t fft_smem_bytes(int L) { return (size_t)L * sizeof(double2); }

int fft_prepare(dski_handle h) {
  for (int k = 0; k < h->d; ++k) {
    const int m = h->m[k];
    const int L = fft_circulant_size(m);
    if (h->fft_tw[k].ensure((size_t)std::max(L / 2, 1) * sizeof(double2)) ||
        h->fft_lam[k].ensure((size_t)L * sizeof(double)))
      return set_error(DSKI_ERR_ALLOC, "device allocation failed for the FFT multipliers");
    const size_t smem = fft_smem_bytes(L);
    if (smem > 48 * 1024) {
      DSKI_CUDA(cudaFuncSetAttribute(k_fft_multiplier, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
      DSKI_CUDA(cudaFuncSetAttribute(k_mode_fft, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    }
    double2* tw = h->fft_tw[k].as<double2>();
    if (L >= 2)
      k_fft_twiddles<<<(L / 2 + 255) / 256, 256, 0, h->stream>>>(L, tw);
    k_fft_multiplier<<<1, FFT_THREADS, smem, h->stream>>>(h->K64[k].as<double>(), m, L, tw,
                                                          h->fft_lam[k].as<double>());
    count_launches(L >= 2 ? 2 : 1);
    DSKI_LAUNCHED();
  }
  return DSKI_OK;
}

int mode_fft(dski_handle h, int k, const double* X, double* Y, long long R, int s,
             double scale) {
  const int m = h->m[k];
  const int L = fft_circulant_size(m);
  const dim3 grd((unsigned)((R + 1) / 2), (unsigned)s);
  StageScope sc(h, ST_KRON, h->stream);
  k_mode_fft<<<grd, FFT_THREADS, fft_smem_bytes(L), h->stream>>>(
      X, h->fft_tw[k].as<double2>(), h->fft_lam[k].as<double>(), Y, m, L, R, scale);
  DSKI_LAUNCHED();
  return DSKI_OK;
}

}  // namespace dski
