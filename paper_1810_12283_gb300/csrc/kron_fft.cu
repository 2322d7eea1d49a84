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
// The forward transform decimates in frequency (natural order in, bit-
// reversed out), the multiplier is stored bit-reversed, and the inverse
// decimates in time (bit-reversed in, natural out), so no permutation pass is
// needed.  Both run radix-4 stages (one radix-2 stage when log2 L is odd).
// The first forward stage skips the zero-padded upper half, the multiplier
// is folded into the first inverse stage, and the last inverse stage forms
// only the m outputs and writes them straight to global memory.  Everything
// is FP64 in shared memory, the twiddles exp(-2 pi i j / L) included (from
// sincospi once per factor).
//
// The output is written in the layout of the other mode products: contracted
// mode first (one step of the cyclic mode rotation), Y[j][r] = scale (K X)[r][j].
#include <cuda_runtime.h>

#include <algorithm>

#include "dski_internal.cuh"

namespace dski {
namespace {

constexpr int FFT_THREADS = 256;

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {   // a * conj(b)
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ double2 mul_mi(double2 a) { return make_double2(a.y, -a.x); }   // -i a
__device__ __forceinline__ double2 mul_pi(double2 a) { return make_double2(-a.y, a.x); }   //  i a

// exp(-2 pi i k / L) for 0 <= k < L from the table of its first half
__device__ __forceinline__ double2 twv(const double2* T, int k, int half) {
  if (k < half) return T[k];
  const double2 t = T[k - half];
  return make_double2(-t.x, -t.y);
}

// The radix-4 stages below are each two radix-2 stages fused (half sizes 2q
// and q), so every transform keeps the radix-2 orderings: decimation in
// frequency takes natural order to bit-reversed order, decimation in time
// takes it back.  With W = exp(-2 pi i / 4q), j < q, and a0..a3 the entries
// j, j + q, j + 2q, j + 3q of a group of 4q:
//   DIF:  t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = -i (a1 - a3);
//         out = t0 + t2, (t0 - t2) W^2j, (t1 + t3) W^j, (t1 - t3) W^3j
//   DIT (V = conj W):  c1 = a1 V^2j, c2 = a2 V^j, c3 = a3 V^3j;
//         out = (a0 + c1) + (c2 + c3), (a0 - c1) + i (c2 - c3),
//               (a0 + c1) - (c2 + c3), (a0 - c1) - i (c2 - c3)

// radix-2 DIF stage with half size L/2 over the whole vector
__device__ void dif2_top(double2* z, int L, const double2* T) {
  const int half = L >> 1;
  for (int b = threadIdx.x; b < half; b += blockDim.x) {
    const double2 u = z[b], v = z[b + half];
    z[b] = cadd(u, v);
    z[b + half] = cmul(csub(u, v), T[b]);
  }
  __syncthreads();
}

__device__ void dif4(double2* z, int L, int q, const double2* T) {
  const int half = L >> 1, ts = L / (4 * q);
  for (int b = threadIdx.x; b < (L >> 2); b += blockDim.x) {
    const int j = b & (q - 1);
    const int i0 = ((b - j) << 2) + j;
    const double2 a0 = z[i0], a1 = z[i0 + q], a2 = z[i0 + 2 * q], a3 = z[i0 + 3 * q];
    const double2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3),
                  t3 = mul_mi(csub(a1, a3));
    z[i0] = cadd(t0, t2);
    z[i0 + q] = cmul(csub(t0, t2), twv(T, 2 * j * ts, half));
    z[i0 + 2 * q] = cmul(cadd(t1, t3), twv(T, j * ts, half));
    z[i0 + 3 * q] = cmul(csub(t1, t3), twv(T, 3 * j * ts, half));
  }
  __syncthreads();
}

// radix-4 DIT stage; lam (optional) multiplies the inputs first (the
// circulant spectrum, bit-reversed order like the inputs)
__device__ void dit4(double2* z, int L, int q, const double2* T, const double* __restrict__ lam) {
  const int half = L >> 1, ts = L / (4 * q);
  for (int b = threadIdx.x; b < (L >> 2); b += blockDim.x) {
    const int j = b & (q - 1);
    const int i0 = ((b - j) << 2) + j;
    double2 a0 = z[i0], a1 = z[i0 + q], a2 = z[i0 + 2 * q], a3 = z[i0 + 3 * q];
    if (lam) {
      const double l0 = lam[i0], l1 = lam[i0 + q], l2 = lam[i0 + 2 * q], l3 = lam[i0 + 3 * q];
      a0 = make_double2(a0.x * l0, a0.y * l0);
      a1 = make_double2(a1.x * l1, a1.y * l1);
      a2 = make_double2(a2.x * l2, a2.y * l2);
      a3 = make_double2(a3.x * l3, a3.y * l3);
    }
    const double2 c1 = cmulc(a1, twv(T, 2 * j * ts, half));
    const double2 c2 = cmulc(a2, twv(T, j * ts, half));
    const double2 c3 = cmulc(a3, twv(T, 3 * j * ts, half));
    const double2 e0 = cadd(a0, c1), e1 = csub(a0, c1), f0 = cadd(c2, c3),
                  f1 = mul_pi(csub(c2, c3));
    z[i0] = cadd(e0, f0);
    z[i0 + q] = cadd(e1, f1);
    z[i0 + 2 * q] = csub(e0, f0);
    z[i0 + 3 * q] = csub(e1, f1);
  }
  __syncthreads();
}

// forward transform of a full vector in shared memory (natural order in,
// bit-reversed order out), L = 2^p >= 8
__device__ void fft_forward(double2* z, int L, int p, const double2* T) {
  int q;
  if (p & 1) {
    dif2_top(z, L, T);
    q = L >> 3;
  } else {
    q = L >> 2;
  }
  for (; q >= 1; q >>= 2) dif4(z, L, q, T);
}

// tw[j] = exp(-2 pi i j / L), j < L/2
__global__ void k_fft_twiddles(int L, double2* __restrict__ tw) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= (L >> 1)) return;
  double s, c;
  sincospi(-2.0 * (double)j / (double)L, &s, &c);
  tw[j] = make_double2(c, s);
}

__device__ __forceinline__ int log2_pow2(int L) { return 31 - __clz(L); }

// lam = (F c) / L in bit-reversed order, c the circulant column built from
// kappa = the first row of K_k (one CTA)
__global__ void k_fft_multiplier(const double* __restrict__ K, int m, int L,
                                 const double2* __restrict__ tw, double* __restrict__ lam) {
  extern __shared__ double2 smem[];
  double2* T = smem;
  double2* zs = smem + (L >> 1);
  for (int i = threadIdx.x; i < (L >> 1); i += blockDim.x) T[i] = tw[i];
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    double v = 0.0;
    if (i < m) v = K[i];
    else if (i > L - m) v = K[L - i];
    zs[i] = make_double2(v, 0.0);
  }
  __syncthreads();
  fft_forward(zs, L, log2_pow2(L), T);
  const double inv = 1.0 / (double)L;
  for (int i = threadIdx.x; i < L; i += blockDim.x) lam[i] = zs[i].x * inv;
}

// Y_q[j][r] = scale sum_i K[j][i] X_q[r][i] for the row pair (r0, r0 + 1) of
// CTA blockIdx.x and column q = blockIdx.y; X_q is R x m (contracted mode
// contiguous), Y_q is m x R.  L = 2^p >= 8 and m <= L/2, so the upper half
// of the padded input is zero: the first forward stage reads only the lower
// half (from global memory), and the last inverse stage forms only the
// outputs below L/2 and writes those below m.
__global__ void __launch_bounds__(FFT_THREADS) k_mode_fft(const double* __restrict__ X,
                                                         const double2* __restrict__ tw,
                                                         const double* __restrict__ lam,
                                                         double* __restrict__ Y, int m, int L,
                                                         long long R, double scale) {
  extern __shared__ double2 smem[];
  const int half = L >> 1;
  double2* T = smem;
  double2* zs = smem + half;
  const int p = log2_pow2(L);
  const long long r0 = 2LL * blockIdx.x;
  const bool two = r0 + 1 < R;
  const long long qoff = (long long)blockIdx.y * R * m;
  const double* x0 = X + qoff + r0 * m;
  const double* x1 = two ? x0 + m : x0;
  for (int i = threadIdx.x; i < half; i += blockDim.x) T[i] = tw[i];
  __syncthreads();
  auto xin = [&](int i) {
    return i < m ? make_double2(x0[i], two ? x1[i] : 0.0) : make_double2(0.0, 0.0);
  };
  // forward: first stage with the zero upper half
  int q;
  if (p & 1) {   // radix-2, half size L/2: (a0, 0) -> a0, a0 W^b
    for (int b = threadIdx.x; b < half; b += blockDim.x) {
      const double2 a0 = xin(b);
      zs[b] = a0;
      zs[b + half] = cmul(a0, T[b]);
    }
    q = L >> 3;
  } else {       // radix-4, q = L/4, a2 = a3 = 0
    const int q0 = L >> 2;
    for (int j = threadIdx.x; j < q0; j += blockDim.x) {
      const double2 a0 = xin(j), a1 = xin(j + q0);
      const double2 t3 = mul_mi(a1);
      zs[j] = cadd(a0, a1);
      zs[j + q0] = cmul(csub(a0, a1), twv(T, 2 * j, half));
      zs[j + 2 * q0] = cmul(cadd(a0, t3), twv(T, j, half));
      zs[j + 3 * q0] = cmul(csub(a0, t3), twv(T, 3 * j, half));
    }
    q = L >> 4;
  }
  __syncthreads();
  for (; q >= 1; q >>= 2) dif4(zs, L, q, T);
  // inverse: radix-4 stages q = 1, 4, .. below the last; the first takes lam
  const int qlast = (p & 1) ? 0 : (L >> 2);   // final radix-4 stage, or a radix-2 one
  const int qstop = (p & 1) ? (L >> 1) : qlast;
  for (int qq = 1; qq < qstop; qq <<= 2) dit4(zs, L, qq, T, qq == 1 ? lam : nullptr);
  double* Yq = Y + qoff;
  if (p & 1) {   // final radix-2 stage, half size L/2: out[j] = u + v conj(W^j), j < L/2
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const double2 v = cadd(zs[j], cmulc(zs[j + half], T[j]));
      Yq[(long long)j * R + r0] = scale * v.x;
      if (two) Yq[(long long)j * R + r0 + 1] = scale * v.y;
    }
  } else {       // final radix-4 stage q = L/4: outputs j and j + L/4 only
    const int q0 = L >> 2;
    for (int j = threadIdx.x; j < q0; j += blockDim.x) {
      const double2 a0 = zs[j], a1 = zs[j + q0], a2 = zs[j + 2 * q0], a3 = zs[j + 3 * q0];
      const double2 c1 = cmulc(a1, twv(T, 2 * j, half));
      const double2 c2 = cmulc(a2, twv(T, j, half));
      const double2 c3 = cmulc(a3, twv(T, 3 * j, half));
      const double2 o0 = cadd(cadd(a0, c1), cadd(c2, c3));
      const double2 o1 = cadd(csub(a0, c1), mul_pi(csub(c2, c3)));
      Yq[(long long)j * R + r0] = scale * o0.x;
      if (two) Yq[(long long)j * R + r0 + 1] = scale * o0.y;
      if (j + q0 < m) {
        Yq[(long long)(j + q0) * R + r0] = scale * o1.x;
        if (two) Yq[(long long)(j + q0) * R + r0 + 1] = scale * o1.y;
      }
    }
  }
}

}  // namespace

int fft_circulant_size(int m) {
  int L = 1;
  while (L < 2 * m - 1) L <<= 1;
  return L;
}

size_t fft_smem_bytes(int L) { return (size_t)(L + L / 2) * sizeof(double2); }

// threads per transform: one radix-4 butterfly per thread and stage
static int fft_threads(int L) { return std::min(FFT_THREADS, std::max(64, L / 4)); }

int fft_prepare(dski_handle h) {
  for (int k = 0; k < h->d; ++k) {
    const int m = h->m[k];
    const int L = fft_circulant_size(m);
    if (L < 8)   // the transforms take L >= 8 (every grid has m_k >= 4)
      return set_error(DSKI_ERR_ARG, "FFT products need m_k >= 4 (got %d)", m);
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
    k_fft_multiplier<<<1, fft_threads(L), smem, h->stream>>>(h->K64[k].as<double>(), m, L, tw,
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
  k_mode_fft<<<grd, fft_threads(L), fft_smem_bytes(L), h->stream>>>(
      X, h->fft_tw[k].as<double2>(), h->fft_lam[k].as<double>(), Y, m, L, R, scale);
  DSKI_LAUNCHED();
  return DSKI_OK;
}

}  // namespace dski
