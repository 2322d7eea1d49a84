// Kronecker mode products on the tensor cores (tcgen05, sm_103a).
//
// One mode product of the D-SKI grid product h = s_f^2 (K_1 (x) ... (x) K_d) g
// (Sec. 3.1; K_UU is Kronecker because the SE kernel of App. A is a product
// over dimensions) is, for every grid column q,
//   Y_q[j][r] = scale * sum_i K[j][i] X_q[r][i],
// X_q viewed as R x m with the contracted mode contiguous; the output puts the
// contracted mode first (one step of the cyclic mode rotation).  As a GEMM,
// D (M = j, N = r) = A (j x i, K-major) . B (r x i, K-major) -- both operands
// K-major, accumulator 128 x 32 FP32 in TMEM.
//
// Precision: TF32 operands (kind::tf32).  MIXED_3XTF32 splits both operands
// into hi = rna_tf32(x) and lo = rna_tf32(x - hi) and accumulates
// hi.hi + hi.lo + lo.hi (the lo.lo term is below FP32 resolution);
// MIXED_TF32 uses hi.hi only.  K's split is precomputed with the factor.
//
// Pipeline: 128 threads.  Per 32-wide K chunk every thread stages part of the
// A and B tiles into 128B-swizzled shared memory (two stages), one thread
// issues the MMAs and commits them to the stage's mbarrier; a stage is reused
// only after its mbarrier reports the MMAs that read it complete.  Every wait
// is bounded: on time-out the kernel records an error and still frees TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "dski_internal.cuh"
#include "tc_common.cuh"

namespace dski {
namespace {

constexpr int TC_M = 128;
constexpr int TC_N = 32;
constexpr int TC_KC = 32;                       // TF32 elements per 128-byte row
constexpr int A_BYTES = TC_M * 128;             // 16 KB
constexpr int B_BYTES = TC_N * 128;             // 4 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int TC_SMEM = 2 * STAGE_BYTES + 1024 + 64;
constexpr uint32_t WAIT_LIMIT = 1u << 22;

template <int NMMA>
__global__ void __launch_bounds__(128) k_mode_tc_tf32(const float* __restrict__ X,
                                                      const float* __restrict__ Khi,
                                                      const float* __restrict__ Klo,
                                                      float* __restrict__ Y, int m, long long R,
                                                      float scale, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* mbar = (uint64_t*)(smem + 2 * STAGE_BYTES);
  uint32_t* tslot = (uint32_t*)(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = blockIdx.x * TC_M;
  const long long r0 = (long long)blockIdx.y * TC_N;
  const long long qoff = (long long)blockIdx.z * R * m;
  const float* Xq = X + qoff;
  float* Yq = Y + qoff;

  if (warp == 0) tc::tmem_alloc(tslot, TC_N);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = tc::instr_desc(tc::kFmtTF32, TC_M, TC_N);

  const int nk = (m + TC_KC - 1) / TC_KC;
  uint32_t phase[2] = {0u, 0u};
  int ok = 1;
  for (int kc = 0; kc < nk; ++kc) {
    const int st = kc & 1;
    unsigned char* sAh = smem + st * STAGE_BYTES;
    unsigned char* sAl = sAh + A_BYTES;
    unsigned char* sBh = sAl + A_BYTES;
    unsigned char* sBl = sBh + B_BYTES;
    if (kc >= 2) {
      ok &= tc::mbar_wait(&mbar[st], phase[st], WAIT_LIMIT) ? 1 : 0;
      phase[st] ^= 1u;
    }
    if (!__syncthreads_and(ok)) break;
    const int i0 = kc * TC_KC;
    // A: row tid of the tile (j = j0 + tid), 32 K values
    {
      const int j = j0 + tid;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float4 h4, l4;
        float* hv = &h4.x;
        float* lv = &l4.x;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = i0 + 4 * c + e;
          const bool in = j < m && i < m;
          hv[e] = in ? Khi[(long long)j * m + i] : 0.f;
          lv[e] = (NMMA > 1 && in) ? Klo[(long long)j * m + i] : 0.f;
        }
        *(float4*)(sAh + tc::sw128_off(tid, c)) = h4;
        if (NMMA > 1) *(float4*)(sAl + tc::sw128_off(tid, c)) = l4;
      }
    }
    // B: TPR threads per row of the tile (r = r0 + row), 8 / TPR chunks each
    {
      constexpr int TPR = 128 / TC_N;
      constexpr int CPT = 8 / TPR;
      static_assert(TPR * TC_N == 128 && CPT * TPR == 8, "B tile split");
      const int row = tid / TPR;
      const long long r = r0 + row;
      const int c0 = (tid % TPR) * CPT;
#pragma unroll
      for (int c = c0; c < c0 + CPT; ++c) {
        float4 h4, l4;
        float* hv = &h4.x;
        float* lv = &l4.x;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = i0 + 4 * c + e;
          const float x = (r < R && i < m) ? Xq[r * m + i] : 0.f;
          const float hi = tc::rna_tf32(x);
          hv[e] = hi;
          lv[e] = tc::rna_tf32(x - hi);
        }
        *(float4*)(sBh + tc::sw128_off(row, c)) = h4;
        if (NMMA > 1) *(float4*)(sBl + tc::sw128_off(row, c)) = l4;
      }
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t aH = tc::smem_u32(sAh), aL = tc::smem_u32(sAl);
      const uint32_t bH = tc::smem_u32(sBh), bL = tc::smem_u32(sBl);
#pragma unroll
      for (int kk = 0; kk < TC_KC / 8; ++kk) {
        const uint32_t ko = kk * 32;   // 8 TF32 = 32 bytes per MMA
        const uint32_t acc0 = (kc > 0 || kk > 0) ? 1u : 0u;
        tc::mma_tf32(tmem, tc::sw128_desc(aH + ko), tc::sw128_desc(bH + ko), idesc, acc0);
        if (NMMA > 1) {
          tc::mma_tf32(tmem, tc::sw128_desc(aH + ko), tc::sw128_desc(bL + ko), idesc, 1u);
          tc::mma_tf32(tmem, tc::sw128_desc(aL + ko), tc::sw128_desc(bH + ko), idesc, 1u);
        }
      }
      tc::commit(&mbar[st]);
    }
  }
  // the last commit covers every MMA issued before it
  if (ok) {
    const int st = (nk - 1) & 1;
    ok &= tc::mbar_wait(&mbar[st], phase[st], WAIT_LIMIT) ? 1 : 0;
  } else {
    // drain whatever was issued (bounded) before TMEM is released
    const int st = (nk - 1) & 1;
    tc::mbar_wait(&mbar[st], phase[st], WAIT_LIMIT);
  }
  ok = __syncthreads_and(ok);
  tc::fence_after();
  if (ok) {
    const int j = j0 + warp * 32 + lane;
#pragma unroll
    for (int c16 = 0; c16 < TC_N / 16; ++c16) {
      uint32_t v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c16 * 16, v);
      if (j < m) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const long long r = r0 + c16 * 16 + e;
          if (r < R) Yq[(long long)j * R + r] = scale * __uint_as_float(v[e]);
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TC_N);
}

__device__ __forceinline__ uint32_t cluster_rank_tf() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_tf() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

// The same product with the contraction split over a thread-block cluster:
// CTA (j tile of 128, r tile of 32, column q, split ks of 32); K's hi (and
// lo) planes of the split arrive by TMA (128-byte swizzle), the threads
// split their slice of X into TF32 hi / lo, one thread issues 4 (x NMMA)
// MMAs, each thread writes its row's 32 FP32 partials to an L2 workspace,
// and after a cluster barrier every CTA sums a 1/KS share of the tile over
// the splits in a fixed order (deterministic).  Grid (m/128, R/32, s KS),
// cluster (1, 1, KS), KS = ceil(m / 32) <= 8.
constexpr int TS_SMEM = 2 * A_BYTES + 2 * B_BYTES + 1024 + 64;
template <int NMMA>
__global__ void __launch_bounds__(128) k_mode_tc_tf32_split(
    const __grid_constant__ CUtensorMap tHi, const __grid_constant__ CUtensorMap tLo,
    const float* __restrict__ X, float* __restrict__ Y, float* __restrict__ P, int m, long long R,
    int KS, float scale, int* __restrict__ err, uint32_t wait1) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sAh = smem;
  unsigned char* sAl = sAh + A_BYTES;
  unsigned char* sBh = sAl + A_BYTES;
  unsigned char* sBl = sBh + B_BYTES;
  uint64_t* full = (uint64_t*)(sBl + B_BYTES);
  uint64_t* done = full + 1;
  uint32_t* tslot = (uint32_t*)(full + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = blockIdx.x * TC_M;
  const long long r0 = (long long)blockIdx.y * TC_N;
  const int q = blockIdx.z / KS;
  const uint32_t crank = cluster_rank_tf();
  const int i0 = (int)crank * TC_KC;

  if (warp == 0) tc::tmem_alloc(tslot, TC_N);
  if (tid == 0) {
    tc::mbar_init(full, 1);
    tc::mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    tc::mbar_expect_tx(full, (uint32_t)(NMMA > 1 ? 2 * A_BYTES : A_BYTES));
    tc::tma_load_2d(sAh, &tHi, i0, j0, full);
    if (NMMA > 1) tc::tma_load_2d(sAl, &tLo, i0, j0, full);
  }
  // B: thread (row tid / 4, chunks 2 (tid % 4), +1) of the 32 x 32 slice
  {
    const int row = tid >> 2, c0 = (tid & 3) * 2;
    const long long r = r0 + row;
    const float* xr = X + ((long long)q * R + r) * m;
#pragma unroll
    for (int c = c0; c < c0 + 2; ++c) {
      float4 h4, l4;
      float* hv = &h4.x;
      float* lv = &l4.x;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = i0 + 4 * c + e;
        const float x = (r < R && i < m) ? xr[i] : 0.f;
        const float hi = tc::rna_tf32(x);
        hv[e] = hi;
        lv[e] = tc::rna_tf32(x - hi);
      }
      *(float4*)(sBh + tc::sw128_off(row, c)) = h4;
      if (NMMA > 1) *(float4*)(sBl + tc::sw128_off(row, c)) = l4;
    }
  }
  tc::fence_proxy_async();
  __syncthreads();
  constexpr uint32_t idesc = tc::instr_desc(tc::kFmtTF32, TC_M, TC_N);
  int ok = 1;
  if (tid == 0) {
    if (tc::mbar_wait(full, 0, wait1)) {
      tc::fence_after();
      const uint32_t aH = tc::smem_u32(sAh), aL = tc::smem_u32(sAl);
      const uint32_t bH = tc::smem_u32(sBh), bL = tc::smem_u32(sBl);
#pragma unroll
      for (int kk = 0; kk < TC_KC / 8; ++kk) {
        const uint32_t ko = kk * 32;   // 8 TF32 = 32 bytes per MMA
        tc::mma_tf32(tmem, tc::sw128_desc(aH + ko), tc::sw128_desc(bH + ko), idesc, kk > 0 ? 1u : 0u);
        if (NMMA > 1) {
          tc::mma_tf32(tmem, tc::sw128_desc(aH + ko), tc::sw128_desc(bL + ko), idesc, 1u);
          tc::mma_tf32(tmem, tc::sw128_desc(aL + ko), tc::sw128_desc(bH + ko), idesc, 1u);
        }
      }
    } else {
      ok = 0;
      tc::mbar_wait(full, 0, WAIT_LIMIT);   // let the loads land (bounded)
    }
    tc::commit(done);
  }
  __syncthreads();
  int fin = tc::mbar_wait(done, 0, WAIT_LIMIT) ? 1 : 0;
  fin = __syncthreads_and(fin && (tid != 0 || ok));
  tc::fence_after();
  const long long tile = ((long long)q * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  float* Pt = P + tile * KS * (TC_M * TC_N);
  {
    float* Pw = Pt + (long long)crank * (TC_M * TC_N) + warp * 32 + lane;   // (column, row)
#pragma unroll
    for (int c16 = 0; c16 < TC_N / 16; ++c16) {
      uint32_t v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c16 * 16, v);
#pragma unroll
      for (int e = 0; e < 16; ++e) __stcg(Pw + (c16 * 16 + e) * TC_M, fin ? __uint_as_float(v[e]) : 0.f);
    }
  }
  if (!fin && tid == 0) atomicExch(err, 1);
  cluster_sync_tf();   // every split's partials are written
  {
    const int rb = (int)((crank * TC_M) / KS), re = (int)(((crank + 1) * TC_M) / KS);
    const int nr = re - rb;
    const long long MR = (long long)m * R;
    for (int it = tid; it < nr * TC_N; it += 128) {
      const int row = rb + it % nr, col = it / nr;
      const int off = col * TC_M + row;
      float sum = 0.f;
#pragma unroll
      for (int src = 0; src < 8; ++src)
        if (src < KS) sum += __ldcg(Pt + (long long)src * (TC_M * TC_N) + off);
      const int j = j0 + row;
      const long long r = r0 + col;
      if (j < m && r < R) Y[(long long)q * MR + (long long)j * R + r] = scale * sum;
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TC_N);
}

}  // namespace

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// One mode product on the tensor cores (mixed modes).  Returns DSKI_OK or CUDA.
static bool tf32_split_path(int m) { return m % 4 == 0 && m <= 256; }

// budget of the first mbarrier wait of a tensor-core product (see
// dski_set_wait_budget)
static uint32_t first_wait_polls(dski_handle h) {
  return h->wait_budget < 0 ? WAIT_LIMIT : (uint32_t)h->wait_budget;
}

size_t mode_tc_tf32_ws_bytes(int m, long long R, int s) {
  if (!tf32_split_path(m)) return 0;
  const int KS = (m + TC_KC - 1) / TC_KC;
  const long long tiles = (long long)s * ((m + TC_M - 1) / TC_M) * ((R + TC_N - 1) / TC_N);
  return (size_t)tiles * KS * TC_M * TC_N * 4;
}

int mode_tc_tf32(dski_handle h, const float* X, const float* Khi, const float* Klo, float* Y,
                 int m, long long R, int s, float scale, bool three, float* ws) {
  auto enc = tensor_map_encoder();
  if (enc && tf32_split_path(m)) {
    // split contraction over a cluster, K by TMA
    CUtensorMap tHi, tLo;
    const cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)m};
    const cuuint64_t str[1] = {(cuuint64_t)m * 4};
    const cuuint32_t box[2] = {(cuuint32_t)TC_KC, (cuuint32_t)TC_M};
    const cuuint32_t estr[2] = {1, 1};
    for (int t = 0; t < 2; ++t) {
      const CUresult r = enc(t ? &tLo : &tHi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                             const_cast<float*>(t ? Klo : Khi), dims, str, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS)
        return set_error(DSKI_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
    static std::atomic<unsigned long long> attr_split{0};
    if (first_on_device(&attr_split)) {
      cudaFuncSetAttribute(k_mode_tc_tf32_split<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TS_SMEM);
      cudaFuncSetAttribute(k_mode_tc_tf32_split<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, TS_SMEM);
    }
    const int KS = (m + TC_KC - 1) / TC_KC;
    float* part = ws;
    if (!part) {
      if (h->ozP.ensure(mode_tc_tf32_ws_bytes(m, R, s)))
        return set_error(DSKI_ERR_ALLOC, "tensor-core workspace allocation failed");
      part = h->ozP.as<float>();
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)((m + TC_M - 1) / TC_M), (unsigned)((R + TC_N - 1) / TC_N),
                       (unsigned)(s * KS));
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = TS_SMEM;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = (unsigned)KS;
    attr[1].id = cudaLaunchAttributeClusterSchedulingPolicyPreference;
    attr[1].val.clusterSchedulingPolicyPreference = cudaClusterSchedulingPolicyLoadBalancing;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    StageScope sc(h, ST_KRON, h->stream);
    const cudaError_t e =
        three ? cudaLaunchKernelEx(&cfg, k_mode_tc_tf32_split<3>, tHi, tLo, X, Y, part, m, R, KS,
                                   scale, h->dev_err.as<int>(), first_wait_polls(h))
              : cudaLaunchKernelEx(&cfg, k_mode_tc_tf32_split<1>, tHi, tLo, X, Y, part, m, R, KS,
                                   scale, h->dev_err.as<int>(), first_wait_polls(h));
    if (e != cudaSuccess)
      return set_error(DSKI_ERR_CUDA, "TF32 mode product launch: %s", cudaGetErrorString(e));
    return DSKI_OK;
  }
  static std::atomic<unsigned long long> attr_set{0};
  if (first_on_device(&attr_set)) {
    cudaFuncSetAttribute(k_mode_tc_tf32<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    cudaFuncSetAttribute(k_mode_tc_tf32<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  }
  dim3 grd((unsigned)((m + TC_M - 1) / TC_M), (unsigned)((R + TC_N - 1) / TC_N), (unsigned)s);
  StageScope sc(h, ST_KRON, h->stream);
  if (three)
    k_mode_tc_tf32<3><<<grd, 128, TC_SMEM, h->stream>>>(X, Khi, Klo, Y, m, R, scale,
                                                        h->dev_err.as<int>());
  else
    k_mode_tc_tf32<1><<<grd, 128, TC_SMEM, h->stream>>>(X, Khi, Klo, Y, m, R, scale,
                                                        h->dev_err.as<int>());
  DSKI_LAUNCHED();
  return DSKI_OK;
}


namespace {

// ---------------------------------------------------------------------------
// FP64-accurate mode products on the BF16 tensor cores (DSKI_FP64_TC).
//
// Operands are split into S = 8 signed digits relative to a per-row power
// of two (Ozaki-style splitting): for a row with max |x| < 2^e,
// x = 2^(e - P) V with the integer V = round(x 2^(P - e)), |V| < 2^P, P = 62,
// and V = sum_b d_b 2^(8 (S - 1 - b)), |d_0| <= 64, |d_b| <= 128: integers
// exact in BF16, extracted with integer arithmetic on the FP64 bit pattern
// (GB300's FP64 units are ~60x slower than its integer and FP32 units).  A
// digit product is at most 2^14; one CTA contracts 32 terms, so a level sum
//   T_l = sum_{a + b = l} sum_i A_a[j][i] B_b[r][i]   (at most 8 digit pairs)
// stays below 2^22 and accumulates EXACTLY in its FP32 TMEM accumulator.
// Levels 0..S-1 are kept:
//   Y[j][r] = 2^(fA_j + eB_r - 2 P + 8 (S - 1)) sum_l 2^(8 (S - 1 - l)) T_l,
// exact up to the dropped pairs (weight < 2^(-8 S) of the leading term) and
// the operands' rounding to 62 bits of their row maxima: FP64-class accuracy
// (the FP32 product misses by 2^-24, 26x the noise variance on the terrain
// grid).  K's digits are made once per factor.
//
// One kernel per mode product.  CTA (j tile of 128, r tile of 32, column q,
// contraction split ks of 32); the KS splits of one output tile form a
// thread-block cluster.
//   1. TMA brings K's 8 digit planes of the split (64-byte swizzled rows);
//      meanwhile the threads load the split's 32 x 32 slice of X (FP64) and
//      its per-row maximum exponent.
//   2. Cluster barrier; every CTA takes the row maxima over the whole
//      contraction from the cluster's shared memories (distributed shared
//      memory) and writes its slice's digits, 64-byte swizzled, as the B
//      operand.
//   3. One thread issues the 36 digit-pair MMAs per 16-deep step into 8 TMEM
//      level accumulators.
//   4. Each thread folds its row's levels into an exact int64 pair (hi, lo)
//      and writes it to an L2-resident workspace; after a cluster barrier
//      every CTA sums a 1/KS share of the tile over the splits (fixed order:
//      deterministic) and writes FP64.  (Reading the pairs from the other
//      CTAs' shared memory instead ran at ~10 B/clock per SM.)
constexpr int OZ_S = kOzDigits;                  // digits per operand (8)
constexpr int OZ_P = 6 + 8 * (OZ_S - 1);         // fixed-point bits: |V| < 2^OZ_P
static_assert(OZ_P <= 62, "fixed-point range");
constexpr int Z_M = 128, Z_N = 32, Z_KC = 32;    // tile rows, tile columns, split depth
constexpr int Z_A = Z_M * 64;                     // one A digit plane: 128 rows x 64 B
constexpr int Z_B = Z_N * 64;                     // one B digit plane: 32 rows x 64 B
constexpr int Z_STAGE = OZ_S * (Z_A + Z_B);       // 80 KB of operands
constexpr int Z_TILE = Z_M * Z_N;                 // (hi, lo) pairs per split of a tile
constexpr int Z_EXP = Z_STAGE;                    // 2 x 32 ints: row maxima (partial, full)
constexpr int Z_BAR = Z_STAGE + 256;
constexpr int Z_SMEM = Z_STAGE + 256 + 64 + 1024;
constexpr int Z_MAXKS = 8;                        // portable cluster size
constexpr float Z_MAGIC = 12582912.0f;            // 1.5 2^23: t + Z_MAGIC has bits 0x4B400000 + t
static_assert(OZ_S * Z_N <= 256, "TMEM columns");
// exactness of one level: at most OZ_S digit pairs of 2^14 over Z_KC terms
static_assert((long long)OZ_S * Z_KC * 128 * 128 < (1LL << 24), "FP32 level sums must stay exact");

// Biased exponent field of |x| (0 for zero and subnormals).
__device__ __forceinline__ int exp_field(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// V = round(x 2^(OZ_P - e)) as an integer (|V| < 2^OZ_P when |x| < 2^e), from
// the bit pattern alone.
__device__ __forceinline__ long long fixedP(double x, int e) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((u >> 52) & 0x7FF);
  if (E == 0) return 0;   // zero or subnormal: below the last digit
  const unsigned long long mant = (u & ((1ULL << 52) - 1)) | (1ULL << 52);
  // |V| = mant 2^(E - 1075 + OZ_P - e); the shift can be left (by at most
  // OZ_P - 53 when |x| is the row maximum) or right (with rounding)
  const int sh = 1075 - OZ_P + e - E;   // >= 53 - OZ_P because |x| < 2^e
  long long v = 0;
  if (sh <= 0) v = (long long)(mant << (-sh));
  else if (sh < 62) v = (long long)((mant + (1ULL << (sh - 1))) >> sh);
  return (u >> 63) ? -v : v;
}

// The OZ_S balanced base-256 digits of V (|V| < 2^62) as BF16 bit patterns:
// the bytes of V + 0x8080...80, each minus 128, so d_b in [-128, 127] (the
// first in [-64, 63]) and V = sum_b d_b 2^(8 (S - 1 - b)) exactly.  Every
// digit is independent of the others (no carry chain), and its BF16 value
// comes from one exact FP32 add: 0x4B400000 + d is the bit pattern of
// 1.5 2^23 + d.
__device__ __forceinline__ void digits_bf16(long long V, uint16_t (&d)[OZ_S]) {
  static_assert(OZ_S == 8, "one byte per digit of a 64-bit word");
  const unsigned long long u = (unsigned long long)V + 0x8080808080808080ULL;
  const uint32_t w[2] = {(uint32_t)(u >> 32), (uint32_t)u};
#pragma unroll
  for (int b = 0; b < OZ_S; ++b) {
    const uint32_t byte = (w[b >> 2] >> (8 * (3 - (b & 3)))) & 255u;
    const float f = __uint_as_float(0x4B400000u - 128u + byte) - Z_MAGIC;   // = byte - 128
    d[b] = (uint16_t)(__float_as_uint(f) >> 16);
  }
}

// The double nearest (ties away from zero) to (hi 2^32 + lo) 2^ex, by integer
// operations only (GB300's FP64 units are the scarce resource here).
__device__ __forceinline__ double exact_to_double(long long hi, long long lo, int ex) {
  const __int128 W = ((__int128)hi << 32) + (__int128)lo;
  if (W == 0) return 0.0;
  const unsigned long long sgn = W < 0 ? (1ULL << 63) : 0ULL;
  unsigned __int128 A = W < 0 ? (unsigned __int128)(-W) : (unsigned __int128)W;
  const unsigned long long a1 = (unsigned long long)(A >> 64), a0 = (unsigned long long)A;
  const int nb = a1 ? 128 - __clzll((long long)a1) : 64 - __clzll((long long)a0);
  unsigned long long mant;
  int e2;
  if (nb > 53) {
    const int sh = nb - 53;
    A = (A + ((unsigned __int128)1 << (sh - 1))) >> sh;
    mant = (unsigned long long)A;
    e2 = ex + sh;
    if (mant >> 53) {   // rounding carried into a new bit
      mant >>= 1;
      ++e2;
    }
  } else {
    mant = (unsigned long long)A << (53 - nb);
    e2 = ex - (53 - nb);
  }
  const long long be = (long long)e2 + 52 + 1023;   // value = mant 2^e2, mant in [2^52, 2^53)
  if (be <= 0) return 0.0;                          // below the normal range
  if (be >= 2047) return __longlong_as_double((long long)(sgn | (0x7FFULL << 52)));
  return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) |
                                          (mant & ((1ULL << 52) - 1))));
}

// Digits of A (rows x cols, row stride lda): Ad[b][j][i] (BF16 bits, row
// stride mp >= cols, zero beyond cols) and fA[j] with max_i |A[j][i]| <
// 2^fA[j].  One thread per row.
__global__ void k_oz_slice_factor(const double* __restrict__ A, int rows, int cols, int lda, int mp,
                                  uint16_t* __restrict__ Ad, int* __restrict__ fA) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= rows) return;
  int E = 0;
  for (int i = 0; i < cols; ++i) E = max(E, exp_field(A[(long long)j * lda + i]));
  const int e = E - 1022;   // max |A[j][:]| < 2^e
  fA[j] = e;
  for (int i = 0; i < mp; ++i) {
    uint16_t d[OZ_S];
    digits_bf16(i < cols ? fixedP(A[(long long)j * lda + i], e) : 0LL, d);
#pragma unroll
    for (int b = 0; b < OZ_S; ++b) Ad[((long long)b * rows + j) * mp + i] = d[b];
  }
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
// address of the same shared-memory location in cluster CTA `rank`
__device__ __forceinline__ uint32_t map_cluster(uint32_t saddr, uint32_t rank) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(saddr), "r"(rank));
  return ra;
}
__device__ __forceinline__ int ld_cluster_s32(uint32_t a) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}

// Arguments of one product Y_q = scale A X_q^T (see OzGemm).
struct OzKArgs {
  const double* X;
  long long ldx, xq, R;
  const double* xs;
  long long xsq;
  int xsn;
  const int* fA;
  double* Y;
  int ytrans;
  longlong2* P;
  int Mrows, mp, KS;
  double scale;
  int* err;
  uint32_t wait1;   // polls of the first wait (the TMA of A's digit planes)
};

// Y_q[j][r] = scale sum_i A[j][i] xs_q[i] X_q[r][i] (or its transpose): A's
// digit planes by TMA (Mrows x mp), X FP64 rows of stride ldx.  Grid
// (Mrows/128, R/32, s KS), cluster (1, 1, KS), KS = ceil(mp / 32) <= 8, 128
// threads.  P: workspace of one 128 x 32 tile of (hi, lo) pairs per CTA,
// [tile][split][column][row].
__global__ void __launch_bounds__(128) k_oz_mode(const __grid_constant__ CUtensorMap tA,
                                                 const OzKArgs a) {
  const double* __restrict__ X = a.X;
  const int* __restrict__ fA = a.fA;
  double* __restrict__ Y = a.Y;
  longlong2* __restrict__ P = a.P;
  const int KS = a.KS, m = a.mp;
  const long long R = a.R;
  const double scale = a.scale;
  int* __restrict__ err = a.err;
  // programmatic dependent launch: a following product may start its
  // set-up now; it waits (griddepcontrol.wait below) before reading ours
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  int* pmax = (int*)(smem + Z_EXP);        // this split's row maxima (exponent fields)
  int* emax = pmax + Z_N;                  // over the whole contraction: e per row
  uint64_t* full = (uint64_t*)(smem + Z_BAR);
  uint64_t* done = full + 1;
  uint32_t* tslot = (uint32_t*)(full + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = blockIdx.x * Z_M;
  const long long r0 = (long long)blockIdx.y * Z_N;
  const int q = blockIdx.z / KS;
  const uint32_t crank = cluster_rank();   // == blockIdx.z % KS: the contraction split
  const int i0 = (int)crank * Z_KC;

  if (warp == 0) tc::tmem_alloc(tslot, 256);
  if (tid == 0) {
    tc::mbar_init(full, 1);
    tc::mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    tc::mbar_expect_tx(full, (uint32_t)(OZ_S * Z_A));
    for (int b = 0; b < OZ_S; ++b) tc::tma_load_3d(smem + b * Z_A, &tA, i0, j0, b, full);
  }
  // everything above touches only this CTA's resources and A's digit planes
  // (written when the factors were built); X, the workspace and Y may belong
  // to the kernel before this one in the stream
  asm volatile("griddepcontrol.wait;" ::: "memory");

  // 1. this thread's 8 operand values: row rr, columns i0 + 8 c .. + 7
  const int rr = tid >> 2, c = tid & 3;
  double xv[8];
  {
    const long long r = r0 + rr;
    const int ib = i0 + 8 * c;
    const bool in = r < R && ib < m;   // m % 8 == 0: a chunk is all in or all out
    const double2* src = reinterpret_cast<const double2*>(X + q * a.xq + r * a.ldx + ib);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double2 t = in ? src[u] : make_double2(0.0, 0.0);
      xv[2 * u] = t.x;
      xv[2 * u + 1] = t.y;
    }
    if (a.xs) {   // per-contraction-index scale (exact products are not needed: X rounded once)
#pragma unroll
      for (int u = 0; u < 8; ++u) xv[u] *= ib + u < a.xsn ? a.xs[q * a.xsq + ib + u] : 0.0;
    }
  }
  int E = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) E = max(E, exp_field(xv[u]));
  E = max(E, __shfl_xor_sync(0xffffffffu, E, 1));
  E = max(E, __shfl_xor_sync(0xffffffffu, E, 2));
  if (c == 0) pmax[rr] = E;
  cluster_sync();   // every split's row maxima are visible

  // 2. row maxima over the contraction; the slice's digits as the B operand
  const uint32_t sbase = tc::smem_u32(smem);
  if (tid < Z_N) {
    const uint32_t a = tc::smem_u32(pmax + tid);
    int ev[Z_MAXKS];
#pragma unroll
    for (int src = 0; src < Z_MAXKS; ++src)   // all loads in flight before the max
      ev[src] = src < KS ? ld_cluster_s32(map_cluster(a, (uint32_t)src)) : 0;
    int Em = 0;
#pragma unroll
    for (int src = 0; src < Z_MAXKS; ++src) Em = max(Em, ev[src]);
    emax[tid] = Em - 1022;   // max |X[r][:]| < 2^e
  }
  __syncthreads();
  {
    const int e = emax[rr];
    uint16_t dg[8][OZ_S];
#pragma unroll
    for (int u = 0; u < 8; ++u) digits_bf16(fixedP(xv[u], e), dg[u]);
    unsigned char* bB = smem + OZ_S * Z_A;
#pragma unroll
    for (int b = 0; b < OZ_S; ++b) {
      uint4 w;
      w.x = (uint32_t)dg[0][b] | ((uint32_t)dg[1][b] << 16);
      w.y = (uint32_t)dg[2][b] | ((uint32_t)dg[3][b] << 16);
      w.z = (uint32_t)dg[4][b] | ((uint32_t)dg[5][b] << 16);
      w.w = (uint32_t)dg[6][b] | ((uint32_t)dg[7][b] << 16);
      *reinterpret_cast<uint4*>(bB + b * Z_B + tc::sw64_off(rr, c)) = w;
    }
  }
  tc::fence_proxy_async();   // the digits are read by the tensor cores
  __syncthreads();

  // 3. the digit-pair MMAs
  constexpr uint32_t idesc = tc::instr_desc(tc::kFmtBF16, Z_M, Z_N);
  int ok = 1;
  if (tid == 0) {
    if (tc::mbar_wait(full, 0, a.wait1)) {
      tc::fence_after();
      const uint32_t aB = sbase;
      const uint32_t bB = aB + OZ_S * Z_A;
#pragma unroll
      for (int kk = 0; kk < Z_KC / 16; ++kk) {
        const uint32_t ko = kk * 32;   // 16 BF16 = 32 bytes per MMA
#pragma unroll
        for (int l = 0; l < OZ_S; ++l)
#pragma unroll
          for (int p = 0; p <= l; ++p)
            tc::mma_f16(tmem + l * Z_N, tc::sw64_desc(aB + p * Z_A + ko),
                        tc::sw64_desc(bB + (l - p) * Z_B + ko), idesc, (kk > 0 || p > 0) ? 1u : 0u);
      }
    } else {
      ok = 0;
      tc::mbar_wait(full, 0, WAIT_LIMIT);   // let the loads land (bounded) before reuse
    }
    tc::commit(done);   // arrives once every MMA issued above has completed
  }
  __syncthreads();
  int fin = tc::mbar_wait(done, 0, WAIT_LIMIT) ? 1 : 0;
  fin = __syncthreads_and(fin && (tid != 0 || ok));
  tc::fence_after();

  // 4. fold this thread's row into the exact pair
  //   hi = sum_{l < S/2} T_l 2^(8 (S/2 - 1 - l)),  lo = sum_{l >= S/2} T_l 2^(8 (S - 1 - l))
  // (pairs of levels first in int32: |T_l 2^8 + T_l+1| < 2^31) and write it
  // to the workspace, element (column, row): coalesced over the warp's rows
  static_assert(OZ_S == 8, "the fold below is written for 8 levels");
  const long long tile = ((long long)q * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  longlong2* Pt = P + tile * KS * Z_TILE;
  {
    longlong2* Pw = Pt + (long long)crank * Z_TILE + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c16 = 0; c16 < Z_N / 16; ++c16) {
      int pr[4][16];   // level pairs (0,1), (2,3), (4,5), (6,7)
      uint32_t v[2][16];
      tc::tmem_ld16_async(trow + c16 * 16, v[0]);
      tc::tmem_wait_ld(v[0]);
#pragma unroll
      for (int l = 0; l < OZ_S; ++l) {
        // level l + 1 streams in while level l is folded
        if (l + 1 < OZ_S) tc::tmem_ld16_async(trow + (l + 1) * Z_N + c16 * 16, v[(l + 1) & 1]);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          // the exact integer T (|T| < 2^22) from its FP32 value: one add
          const int t = fin ? (int)(__float_as_uint(__uint_as_float(v[l & 1][e]) + Z_MAGIC) -
                                    0x4B400000u)
                            : 0;
          if (l & 1) pr[l >> 1][e] = pr[l >> 1][e] * 256 + t;
          else pr[l >> 1][e] = t;
        }
        if (l + 1 < OZ_S) tc::tmem_wait_ld(v[(l + 1) & 1]);
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const long long hi = (long long)pr[0][e] * 65536 + pr[1][e];
        const long long lo = (long long)pr[2][e] * 65536 + pr[3][e];
        __stcg(Pw + (c16 * 16 + e) * Z_M, make_longlong2(hi, lo));   // L2 only
      }
    }
  }
  if (!fin && tid == 0) atomicExch(err, 1);
  cluster_sync();   // every split's pairs are written (release / acquire at cluster scope)

  // 5. this CTA's share of the tile (rows [rb, re), all columns), summed over
  // the splits in order
  {
    const int rb = (int)((crank * Z_M) / KS), re = (int)(((crank + 1) * Z_M) / KS);
    const int nr = re - rb;
    const long long MR = (long long)a.Mrows * R;
    const int nit = nr * Z_N;
    for (int it0 = 0; it0 < nit; it0 += 2 * 128) {
      longlong2 pv[2][Z_MAXKS];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int it = it0 + k * 128 + tid;
        const int off = it < nit ? (it / nr) * Z_M + rb + it % nr : 0;   // (column, row)
#pragma unroll
        for (int src = 0; src < Z_MAXKS; ++src)
          pv[k][src] = (src < KS && it < nit) ? __ldcg(Pt + (long long)src * Z_TILE + off)
                                             : make_longlong2(0, 0);
      }
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int it = it0 + k * 128 + tid;
        if (it >= nit) continue;
        long long hi = 0, lo = 0;
#pragma unroll
        for (int src = 0; src < Z_MAXKS; ++src) {
          hi += pv[k][src].x;
          lo += pv[k][src].y;
        }
        const int row = rb + it % nr, col = it / nr;
        const int j = j0 + row;
        const long long r = r0 + col;
        if (j >= a.Mrows || r >= R) continue;
        const int ex = fA[j] + emax[col] - 2 * OZ_P + 8 * (OZ_S - 1);   // Y = (hi 2^32 + lo) 2^ex
        const double v = exact_to_double(hi, lo, ex);
        const long long o = a.ytrans ? r * a.Mrows + j : (long long)j * R + r;
        Y[(long long)q * MR + o] = scale == 1.0 ? v : scale * v;
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

}  // namespace

int oz_slice(dski_handle h, const double* A, int rows, int cols, int lda, int mp, uint16_t* Ad,
             int* fA, int stage) {
  StageScope sc(h, stage, h->stream);
  k_oz_slice_factor<<<(rows + 127) / 128, 128, 0, h->stream>>>(A, rows, cols, lda, mp, Ad, fA);
  DSKI_LAUNCHED();
  return DSKI_OK;
}

int oz_slice_factor(dski_handle h, const double* K, int m, uint16_t* Ad, int* fA) {
  return oz_slice(h, K, m, m, m, m, Ad, fA, ST_KRON);
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult qr{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &qr) == cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// Y_q = scale A X_q^T on the tensor cores (FP64-accurate; see OzGemm).
int oz_gemm(dski_handle h, const OzGemm& g, int stage) {
  if (g.mp % 8 != 0 || g.mp > 256 || g.mp < 8 || g.Mrows < 1 || g.R < 1 || g.s < 1 ||
      g.ldx < g.mp || g.ldx % 2 != 0)
    return set_error(DSKI_ERR_ARG, "FP64_TC product: contraction %d (needs %% 8 == 0, <= 256)", g.mp);
  auto enc = tensor_map_encoder();
  if (!enc) return set_error(DSKI_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  CUtensorMap tA;
  {
    const cuuint64_t dims[3] = {(cuuint64_t)g.mp, (cuuint64_t)g.Mrows, (cuuint64_t)OZ_S};
    const cuuint64_t str[2] = {(cuuint64_t)g.mp * 2, (cuuint64_t)g.Mrows * g.mp * 2};
    const cuuint32_t box[3] = {(cuuint32_t)Z_KC, (cuuint32_t)Z_M, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(&tA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(g.Ad),
                           dims, str, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      return set_error(DSKI_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  }
  static std::atomic<unsigned long long> attr_set{0};
  if (first_on_device(&attr_set))
    cudaFuncSetAttribute(k_oz_mode, cudaFuncAttributeMaxDynamicSharedMemorySize, Z_SMEM);
  OzKArgs a{};
  a.X = g.X;
  a.ldx = g.ldx;
  a.xq = g.xq;
  a.R = g.R;
  a.xs = g.xs;
  a.xsq = g.xsq;
  a.xsn = g.xsn;
  a.fA = g.fA;
  a.Y = g.Y;
  a.ytrans = g.ytrans ? 1 : 0;
  a.Mrows = g.Mrows;
  a.mp = g.mp;
  a.KS = (g.mp + Z_KC - 1) / Z_KC;   // <= 8
  a.scale = g.scale;
  a.err = h->dev_err.as<int>();
  a.wait1 = first_wait_polls(h);
  const long long tiles = (long long)g.s * ((g.Mrows + Z_M - 1) / Z_M) * ((g.R + Z_N - 1) / Z_N);
  DevBuf& ws = g.workspace ? *g.workspace : h->ozP;
  if (ws.ensure((size_t)tiles * a.KS * Z_TILE * sizeof(longlong2)))
    return set_error(DSKI_ERR_ALLOC, "FP64_TC workspace allocation failed");
  a.P = ws.as<longlong2>();
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)((g.Mrows + Z_M - 1) / Z_M), (unsigned)((g.R + Z_N - 1) / Z_N),
                     (unsigned)(g.s * a.KS));
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = Z_SMEM;
  cfg.stream = h->stream;
  cudaLaunchAttribute attr[3];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = (unsigned)a.KS;
  // let a cluster's CTAs share SMs, so that every cluster of a product can
  // be resident at once
  attr[1].id = cudaLaunchAttributeClusterSchedulingPolicyPreference;
  attr[1].val.clusterSchedulingPolicyPreference = cudaClusterSchedulingPolicyLoadBalancing;
  // programmatic dependent launch (the kernel waits before reading inputs)
  attr[2].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[2].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 3;
  StageScope sc(h, stage, h->stream);
  if (cudaLaunchKernelEx(&cfg, k_oz_mode, tA, a) != cudaSuccess)
    return set_error(DSKI_ERR_CUDA, "FP64_TC product launch: %s",
                     cudaGetErrorString(cudaGetLastError()));
  return DSKI_OK;
}

// One mode product Y_q[j][r] = scale sum_i K[j][i] X_q[r][i] (FP64_TC).
int mode_tc_oz(dski_handle h, const double* X, const uint16_t* Ad, const int* fA, double* Y,
               int m, long long R, int s, double scale) {
  if (m % 8 != 0 || m > 256)
    return set_error(DSKI_ERR_ARG, "FP64_TC mode products need m_k %% 8 == 0 and m_k <= 256 (got %d)", m);
  OzGemm g{};
  g.Ad = Ad;
  g.fA = fA;
  g.Mrows = m;
  g.mp = m;
  g.X = X;
  g.ldx = m;
  g.xq = R * m;
  g.R = R;
  g.Y = Y;
  g.scale = scale;
  g.s = s;
  return oz_gemm(h, g, ST_KRON);
}

}  // namespace dski
