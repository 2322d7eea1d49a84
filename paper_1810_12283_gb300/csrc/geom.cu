// Geometry of the D-SKI operator (Sec. 3.1) and the Kronecker factors of
// K_UU (App. A): run once per dski_create / dski_set_hypers.
//
//  * each point's grid parameter t_k = (x_k - lo_k)/h_k, cell c_k = floor(t_k)
//    and fraction f_k = t_k - c_k, in FP64; the S stencil nodes of
//    dimension k are c_k - lead .. c_k - lead + S - 1 (S = 4, lead = 1 for
//    Keys' cubic; S = 6, lead = 2 for the quintic kernel), so a point needs
//    lead <= c_k <= m_k - S + lead;
//  * the flat cell id (first stencil node per dimension, C order over the
//    (m_k - S + 1)-cell grid) is the sort key; a stable LSD radix sort (8-bit
//    digits, deterministic) orders the points by cell, and a CSR cell_start
//    indexes each cell's points;
//  * K_k[a, b] = exp(-((a - b) h_k)^2 / (2 l_k^2)) in FP64, with FP32 and TF32
//    hi/lo copies for the mixed-precision mode products, and (Toeplitz/FFT
//    products) the circulant spectra of kron_fft.cu.
#include <algorithm>
#include <vector>

#include "dski_internal.cuh"
#include "interp.cuh"

namespace dski {
namespace {

struct GeoParams {
  int d, sw, lead;
  int m[DSKI_MAXD];
  int mc[DSKI_MAXD];
  double lo[DSKI_MAXD];
  double h[DSKI_MAXD];
};

__global__ void k_points(const double* __restrict__ X, int n, GeoParams g,
                         uint32_t* __restrict__ key, int* __restrict__ val,
                         double* __restrict__ frac, int* __restrict__ bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t flat = 0;
  bool ok = true;
  for (int k = 0; k < g.d; ++k) {
    const double t = (X[(size_t)i * g.d + k] - g.lo[k]) / g.h[k];
    const double c = floor(t);
    // written so that NaN fails the test
    if (!(c >= (double)g.lead && c <= (double)(g.m[k] - g.sw + g.lead))) {
      ok = false;
      frac[(size_t)i * g.d + k] = 0.0;
      continue;
    }
    flat = flat * (uint32_t)g.mc[k] + (uint32_t)((int)c - g.lead);
    frac[(size_t)i * g.d + k] = t - c;
  }
  if (!ok) {
    atomicAdd(bad, 1);
    flat = 0;
  }
  key[i] = flat;
  val[i] = i;
}

// ---- stable LSD radix sort of (key, value) pairs, 8-bit digits ----------
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;

// Per-tile digit histogram; hist is digit-major [256][ntiles] so that one
// exclusive scan gives every (digit, tile) its output base.
__global__ void k_rs_hist(const uint32_t* __restrict__ keys, int n, int shift,
                          uint32_t* __restrict__ hist, int ntiles) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int base = blockIdx.x * RS_TILE;
  for (int it = 0; it < RS_ITEMS; ++it) {
    const int idx = base + it * RS_THREADS + threadIdx.x;
    if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Single-block exclusive scan of `len` entries (in place).
__global__ void k_scan_excl(uint32_t* __restrict__ a, int len) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  for (int start = 0; start < len; start += blockDim.x) {
    const int idx = start + threadIdx.x;
    const uint32_t v = idx < len ? a[idx] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t t = lane < nw ? warp_tot[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      if (lane < nw) warp_tot[lane] = t;   // inclusive prefix of warp totals
    }
    __syncthreads();
    const uint32_t before = carry + (warp > 0 ? warp_tot[warp - 1] : 0u);
    if (idx < len) a[idx] = before + x - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + x;
    __syncthreads();
  }
}

// Stable scatter: items of a tile are ranked in index order (chunk by chunk,
// warp by warp, lane by lane).
__global__ void k_rs_scatter(const uint32_t* __restrict__ kin, const int* __restrict__ vin,
                             uint32_t* __restrict__ kout, int* __restrict__ vout, int n,
                             int shift, const uint32_t* __restrict__ hist, int ntiles) {
  __shared__ uint32_t base[256];
  __shared__ uint32_t wcnt[RS_WARPS][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  base[threadIdx.x] = hist[(size_t)threadIdx.x * ntiles + blockIdx.x];
  const int tile0 = blockIdx.x * RS_TILE;
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int it = 0; it < RS_ITEMS; ++it) {
    for (int w = 0; w < RS_WARPS; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int idx = tile0 + it * RS_THREADS + threadIdx.x;
    const bool valid = idx < n;
    uint32_t key = 0;
    int val = 0;
    uint32_t digit = 256u;   // sentinel for missing items
    if (valid) {
      key = kin[idx];
      val = vin[idx];
      digit = (key >> shift) & 255u;
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, digit);
    const uint32_t rank = __popc(peers & lt_mask);
    const int leader = __ffs(peers) - 1;
    if (valid && lane == leader) wcnt[warp][digit] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t off = 0;
      for (int w = 0; w < warp; ++w) off += wcnt[w][digit];
      const uint32_t pos = base[digit] + off + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    uint32_t tot = 0;
    for (int w = 0; w < RS_WARPS; ++w) tot += wcnt[w][threadIdx.x];
    base[threadIdx.x] += tot;
    __syncthreads();
  }
}

__global__ void k_apply_sort(const uint32_t* __restrict__ skey, const int* __restrict__ sval,
                             const double* __restrict__ frac_in, int n, int d,
                             int* __restrict__ perm, int* __restrict__ inv_perm,
                             int* __restrict__ cell, double* __restrict__ f64,
                             float* __restrict__ f32) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int i = sval[j];
  perm[j] = i;
  inv_perm[i] = j;
  cell[j] = (int)skey[j];
  for (int k = 0; k < d; ++k) {
    const double f = frac_in[(size_t)i * d + k];
    f64[(size_t)j * d + k] = f;
    f32[(size_t)j * d + k] = (float)f;
  }
}

// Interpolation weights of each sorted point, computed once in FP64: per
// dimension k the S stencil weights w_k[o] and derivative weights
// phi'(.)/h_k, stored as W[j][k][0..S-1] = w, W[j][k][S..2S-1] = dw (2 S d
// values per point), with an FP32 copy rounded from the FP64 values.
template <int S>
__global__ void k_weights(const double* __restrict__ f64, int n, int d, GeoParams g,
                          double* __restrict__ W64, float* __restrict__ W32) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int k = 0; k < d; ++k) {
    double w[S], dw[S];
    stencil_weights<S, double>(f64[(size_t)j * d + k], w, dw);
    const double ih = 1.0 / g.h[k];
    const size_t b = (size_t)j * 2 * S * d + 2 * S * k;
    for (int o = 0; o < S; ++o) {
      W64[b + o] = w[o];
      W64[b + S + o] = dw[o] * ih;
      W32[b + o] = (float)w[o];
      W32[b + S + o] = (float)(dw[o] * ih);
    }
  }
}

// Double-float copy of the FP64 weight table: Wdf[i] = {hi, lo} with
// hi = fl32(W[i]) and lo = fl32(W[i] - hi) (hi + lo = W[i] to ~2^-48).
__global__ void k_split_weights(const double* __restrict__ W, long long count,
                                float2* __restrict__ Wdf) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double w = W[i];
  const float hi = __double2float_rn(w);
  Wdf[i] = make_float2(hi, __double2float_rn(w - (double)hi));
}

// cell_start[c] = first sorted position whose cell is >= c (CSR over cells).
__global__ void k_cell_start(const uint32_t* __restrict__ skey, int n, int ncell,
                             int* __restrict__ start) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int kj = (int)skey[j];
  const int kp = j == 0 ? -1 : (int)skey[j - 1];
  for (int c = kp + 1; c <= kj; ++c) start[c] = j;
  if (j == n - 1)
    for (int c = kj + 1; c <= ncell; ++c) start[c] = n;
}

__device__ __forceinline__ float rna_tf32(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

__global__ void k_factor(int m, double h, double ell, double* __restrict__ K64,
                         float* __restrict__ K32, float* __restrict__ Khi,
                         float* __restrict__ Klo, double* __restrict__ dK64) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * m) return;
  const int a = idx / m, b = idx % m;
  const double r = (double)(a - b) * h;
  const double q = r * r / (ell * ell);
  const double v = exp(-0.5 * q);
  K64[idx] = v;
  dK64[idx] = v * q;
  K32[idx] = (float)v;
  const float hi = rna_tf32((float)v);
  Khi[idx] = hi;
  Klo[idx] = rna_tf32((float)(v - (double)hi));
}

}  // namespace

int build_geometry(dski_handle h, const double* X_dev) {
  const int n = h->n, d = h->d;
  cudaStream_t st = h->stream;
  GeoParams g{};
  g.d = d;
  g.sw = h->sw;
  g.lead = h->lead;
  for (int k = 0; k < d; ++k) {
    g.m[k] = h->m[k];
    g.mc[k] = h->mc[k];
    g.lo[k] = h->lo[k];
    g.h[k] = h->h[k];
  }
  const int ntiles = (n + RS_TILE - 1) / RS_TILE;
  // scratch: keys x2, vals x2, frac, hist, bad flag
  const size_t off_k1 = 0;
  const size_t off_k2 = off_k1 + 256 * (((size_t)n * 4 + 255) / 256);
  const size_t off_v1 = off_k2 + 256 * (((size_t)n * 4 + 255) / 256);
  const size_t off_v2 = off_v1 + 256 * (((size_t)n * 4 + 255) / 256);
  const size_t off_fr = off_v2 + 256 * (((size_t)n * 4 + 255) / 256);
  const size_t off_hs = off_fr + 256 * (((size_t)n * d * 8 + 255) / 256);
  const size_t off_bad = off_hs + 256 * (((size_t)256 * ntiles * 4 + 255) / 256);
  const size_t total = off_bad + 256;
  DevBuf tmp;
  if (tmp.ensure(total) != DSKI_OK) return DSKI_ERR_ALLOC;
  char* base = tmp.as<char>();
  uint32_t* k1 = (uint32_t*)(base + off_k1);
  uint32_t* k2 = (uint32_t*)(base + off_k2);
  int* v1 = (int*)(base + off_v1);
  int* v2 = (int*)(base + off_v2);
  double* fr = (double*)(base + off_fr);
  uint32_t* hist = (uint32_t*)(base + off_hs);
  int* bad = (int*)(base + off_bad);

  int rc = DSKI_OK;
  do {
    if (cudaMemsetAsync(bad, 0, sizeof(int), st) != cudaSuccess) { rc = DSKI_ERR_CUDA; break; }
    k_points<<<(n + 255) / 256, 256, 0, st>>>(X_dev, n, g, k1, v1, fr, bad);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess) { rc = DSKI_ERR_CUDA; break; }
    int nbad = 0;
    if (cudaMemcpyAsync(&nbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) { rc = DSKI_ERR_CUDA; break; }
    if (nbad > 0) {
      rc = set_error(DSKI_ERR_OUT_OF_GRID,
                     "%d point(s) lack a full %d^d stencil (need %d <= floor((x-lo)/h) <= m-%d)",
                     nbad, h->sw, h->lead, h->sw - h->lead);
      break;
    }
    // number of 8-bit passes needed for keys < ncell
    int passes = 0;
    for (uint64_t top = (uint64_t)std::max(h->ncell - 1, 1); top > 0; top >>= 8) ++passes;
    uint32_t *kin = k1, *kout = k2;
    int *vi = v1, *vo = v2;
    for (int p = 0; p < passes; ++p) {
      const int shift = 8 * p;
      k_rs_hist<<<ntiles, RS_THREADS, 0, st>>>(kin, n, shift, hist, ntiles);
      k_scan_excl<<<1, 1024, 0, st>>>(hist, 256 * ntiles);
      k_rs_scatter<<<ntiles, RS_THREADS, 0, st>>>(kin, vi, kout, vo, n, shift, hist, ntiles);
      count_launches(3);
      std::swap(kin, kout);
      std::swap(vi, vo);
    }
    if (cudaGetLastError() != cudaSuccess) { rc = DSKI_ERR_CUDA; break; }
    if (h->perm.ensure((size_t)n * 4) || h->inv_perm.ensure((size_t)n * 4) ||
        h->cell.ensure((size_t)n * 4) || h->cell_start.ensure((size_t)(h->ncell + 1) * 4) ||
        h->frac64.ensure((size_t)n * d * 8) || h->frac32.ensure((size_t)n * d * 4) ||
        h->W64.ensure((size_t)n * d * 2 * h->sw * 8) ||
        h->W32.ensure((size_t)n * d * 2 * h->sw * 4)) {
      rc = DSKI_ERR_ALLOC;
      break;
    }
    k_apply_sort<<<(n + 255) / 256, 256, 0, st>>>(kin, vi, fr, n, d, h->perm.as<int>(),
                                                  h->inv_perm.as<int>(), h->cell.as<int>(),
                                                  h->frac64.as<double>(), h->frac32.as<float>());
    k_cell_start<<<(n + 255) / 256, 256, 0, st>>>(kin, n, h->ncell, h->cell_start.as<int>());
    with_stencil(h, [&](auto S) {
      k_weights<decltype(S)::value><<<(n + 255) / 256, 256, 0, st>>>(h->frac64.as<double>(), n, d, g,
                                                      h->W64.as<double>(), h->W32.as<float>());
    });
    count_launches(3);
    if (h->prec == DSKI_FP64_TC && d == 2 && h->sw == 4) {
      const long long cnt = (long long)n * d * 2 * h->sw;
      if (h->Wdf.ensure((size_t)cnt * sizeof(float2))) {
        rc = DSKI_ERR_ALLOC;
        break;
      }
      k_split_weights<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(h->W64.as<double>(), cnt,
                                                                    h->Wdf.as<float2>());
      count_launches(1);
    }
    if (cudaGetLastError() != cudaSuccess) { rc = DSKI_ERR_CUDA; break; }
    if (cudaStreamSynchronize(st) != cudaSuccess) { rc = DSKI_ERR_CUDA; break; }
  } while (0);
  tmp.release();
  if (rc == DSKI_ERR_CUDA) return set_error(rc, "geometry kernels failed: %s",
                                            cudaGetErrorString(cudaGetLastError()));
  if (rc == DSKI_ERR_ALLOC) return set_error(rc, "device allocation failed in dski_create");
  return rc;
}

int build_factors(dski_handle h) {
  for (int k = 0; k < h->d; ++k) {
    const int m = h->m[k];
    const size_t mm = (size_t)m * m;
    if (h->K64[k].ensure(mm * 8) || h->K32[k].ensure(mm * 4) || h->Khi[k].ensure(mm * 4) ||
        h->Klo[k].ensure(mm * 4) || h->dK64[k].ensure(mm * 8))
      return set_error(DSKI_ERR_ALLOC, "device allocation failed for Kronecker factors");
    k_factor<<<(unsigned)((mm + 255) / 256), 256, 0, h->stream>>>(
        m, h->h[k], h->ell[k], h->K64[k].as<double>(), h->K32[k].as<float>(),
        h->Khi[k].as<float>(), h->Klo[k].as<float>(), h->dK64[k].as<double>());
    count_launches(1);
    DSKI_LAUNCHED();
    if (h->prec == DSKI_FP64_TC) {
      if (h->Kdig[k].ensure((size_t)kOzDigits * mm * 2) || h->Kexp[k].ensure((size_t)m * 4))
        return set_error(DSKI_ERR_ALLOC, "device allocation failed for factor digits");
      DSKI_TRY(oz_slice_factor(h, h->K64[k].as<double>(), m, h->Kdig[k].as<uint16_t>(),
                               h->Kexp[k].as<int>()));
    }
  }
  if (h->kuu_fft) DSKI_TRY(fft_prepare(h));
  return DSKI_OK;
}

}  // namespace dski
