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

}  // namespace

// One mode product on the tensor cores (mixed modes).  Returns DSKI_OK or CUDA.
int mode_tc_tf32(dski_handle h, const float* X, const float* Khi, const float* Klo, float* Y,
                 int m, long long R, int s, float scale, bool three) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_mode_tc_tf32<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    cudaFuncSetAttribute(k_mode_tc_tf32<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    attr_set = true;
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
// Both operands are split into S = 6 signed 7-bit digits relative to a
// per-row power of two (Ozaki-style splitting): for a row with max |x| <
// 2^e, x = 2^e sum_b d_b 2^(-6 - 7 b) up to rounding at 2^(e - 41), d_b
// integers in [-64, 64] (exact in BF16), extracted with integer arithmetic.  A product of digits is at most 2^12 in magnitude and a sum of
// m <= 256 of them, over the <= 6 digit pairs (a, b) of one level a + b, stays
// below 2^23, so every level accumulates EXACTLY in the FP32 TMEM
// accumulator.  Levels 0..S-1 are kept (one TMEM accumulator each) and
// combined in FP64:
//   Y[j][r] = 2^(fA_j + eB_r - 12) sum_l 2^(-7 l) T_l[j][r],
// (summed exactly in two int64 halves), which drops only the digit pairs of
// weight < 2^(-7 S) -- a relative error of about 2^-56 of |K| |X|, below FP64
// rounding in the 256-term sums
// (the FP32 product misses by 2^-24, 26x the noise variance on the terrain
// grid).
// K's digits are made once per factor; X's digits by a row-parallel kernel
// before each mode product.
constexpr int OZ_S = kOzDigits;                  // digits per operand (8)
constexpr int OZ_P = 6 + 7 * (OZ_S - 1);         // fixed-point bits: |V| < 2^OZ_P
static_assert(OZ_P <= 62 && OZ_P - 53 <= 8, "fixed-point range");
constexpr int OZ_M = 128, OZ_N = 32, OZ_KC = 64;   // 64 BF16 = one 128-byte row
constexpr int OZ_A_BYTES = OZ_M * 128;           // 16 KB per digit
constexpr int OZ_B_BYTES = OZ_N * 128;           // 4 KB per digit
constexpr int OZ_SMEM = OZ_S * (OZ_A_BYTES + OZ_B_BYTES) + 1024 + 256;
constexpr int OZ_TMEM_COLS = 256;                // >= OZ_S * OZ_N, power of two
static_assert(OZ_S * OZ_N <= OZ_TMEM_COLS, "TMEM columns");
// exactness of one level: at most OZ_S digit pairs of 64 x 64, over K <= 256 terms
static_assert((long long)OZ_S * 256 * 64 * 64 <= (1LL << 24), "FP32 level sums must stay exact");

// Biased exponent field of |x| (0 for zero and subnormals).
__device__ __forceinline__ int exp_field(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// V = round(x 2^(OZ_P - e)) as an integer (|V| < 2^OZ_P when |x| < 2^e), from
// the bit pattern alone: GB300's FP64 units are ~60x slower than its
// integer and FP32 units, so the splitting avoids FP64 arithmetic.
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

// OZ_S signed 7-bit digits of V (weights 2^(7 (S-1)), ..., 2^7, 2^0), each
// in [-64, 64]: round-to-nearest at every step leaves |remainder| <= 2^(k-1).
__device__ __forceinline__ void digitsS(long long V, float (&d)[OZ_S]) {
#pragma unroll
  for (int b = 0; b < OZ_S - 1; ++b) {
    const int k = 7 * (OZ_S - 1 - b);
    const long long q = (V + (1LL << (k - 1))) >> k;
    d[b] = (float)(int)q;
    V -= q << k;
  }
  d[OZ_S - 1] = (float)(int)V;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  // exact: a, b are integers in [-64, 64]
  const uint32_t ua = __float_as_uint(a) >> 16, ub = __float_as_uint(b) >> 16;
  return ua | (ub << 16);
}

// Digits of K (m x m, row-major): Ad[b][j][i] (BF16 bits) and fA[j] with
// max_i |K[j][i]| < 2^fA[j].  One thread per row.
__global__ void k_oz_slice_factor(const double* __restrict__ K, int m,
                                  uint16_t* __restrict__ Ad, int* __restrict__ fA) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  int E = 0;
  for (int i = 0; i < m; ++i) E = max(E, exp_field(K[(long long)j * m + i]));
  const int e = E - 1022;   // max |K[j][:]| < 2^e
  fA[j] = e;
  for (int i = 0; i < m; ++i) {
    float d[OZ_S];
    digitsS(fixedP(K[(long long)j * m + i], e), d);
#pragma unroll
    for (int b = 0; b < OZ_S; ++b)
      Ad[((long long)b * m + j) * m + i] = (uint16_t)(__float_as_uint(d[b]) >> 16);
  }
}

// Digits of the rows of X (s grid columns, each R x m): Bd[q][b][r][i] (BF16
// bits) and eB[q][r] with max_i |X_q[r][i]| < 2^eB.  One warp per row.
__global__ void __launch_bounds__(256) k_oz_slice_rows(const double* __restrict__ X, long long R,
                                                       int m, long long rows,
                                                       uint16_t* __restrict__ Bd,
                                                       int* __restrict__ eB) {
  const long long gr = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // q R + r
  const int lane = threadIdx.x & 31;
  if (gr >= rows) return;   // whole warp
  const long long q = gr / R, r = gr % R;
  const double* xr = X + gr * m;
  int E = 0;
  for (int i = lane; i < m; i += 32) E = max(E, exp_field(xr[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
  const int e = E - 1022;
  if (lane == 0) eB[gr] = e;
  for (int i = lane; i < m; i += 32) {
    float d[OZ_S];
    digitsS(fixedP(xr[i], e), d);
#pragma unroll
    for (int b = 0; b < OZ_S; ++b)
      Bd[((q * OZ_S + b) * R + r) * m + i] = (uint16_t)(__float_as_uint(d[b]) >> 16);
  }
}

__global__ void __launch_bounds__(128) k_mode_tc_oz(const uint16_t* __restrict__ Bd,
                                                    const int* __restrict__ eBg,
                                                    const uint16_t* __restrict__ Ad,
                                                    const int* __restrict__ fA,
                                                    double* __restrict__ Y, int m, long long R,
                                                    double scale, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;                                  // OZ_S digit tiles of A
  unsigned char* sB = smem + OZ_S * OZ_A_BYTES;              // OZ_S digit tiles of B
  uint64_t* mbar = (uint64_t*)(sB + OZ_S * OZ_B_BYTES);
  uint32_t* tslot = (uint32_t*)(mbar + 1);
  int* eB = (int*)(tslot + 4);                               // OZ_N row exponents
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = blockIdx.x * OZ_M;
  const long long r0 = (long long)blockIdx.y * OZ_N;
  const long long q = blockIdx.z;
  double* Yq = Y + q * R * m;
  const uint16_t* Bq = Bd + q * OZ_S * R * m;

  if (warp == 0) tc::tmem_alloc(tslot, OZ_TMEM_COLS);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < OZ_N) eB[tid] = (r0 + tid < R) ? eBg[q * R + r0 + tid] : 0;
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = tc::instr_desc(tc::kFmtBF16, OZ_M, OZ_N);

  const int nk = (m + OZ_KC - 1) / OZ_KC;
  uint32_t phase = 0u;
  int ok = 1;
  for (int kc = 0; kc < nk; ++kc) {
    if (kc > 0) {
      ok &= tc::mbar_wait(&mbar[0], phase, WAIT_LIMIT) ? 1 : 0;
      phase ^= 1u;
    }
    if (!__syncthreads_and(ok)) break;
    const int i0 = kc * OZ_KC;
    // A digits: row tid, 8 chunks of 8 BF16 per digit (m % 8 == 0)
    {
      const int j = j0 + tid;
#pragma unroll
      for (int b = 0; b < OZ_S; ++b) {
        unsigned char* dst = sA + b * OZ_A_BYTES;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int i = i0 + 8 * c;
          uint4 v = make_uint4(0, 0, 0, 0);
          if (j < m && i < m) v = *(const uint4*)(Ad + ((long long)b * m + j) * m + i);
          *(uint4*)(dst + tc::sw128_off(tid, c)) = v;
        }
      }
    }
    // B digits: row tid / 4 of the tile, 2 chunks of 8 BF16 per digit
    {
      const int row = tid >> 2, part = tid & 3;
      const long long r = r0 + row;
#pragma unroll
      for (int b = 0; b < OZ_S; ++b) {
        unsigned char* dst = sB + b * OZ_B_BYTES;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int c = part * 2 + cc;
          const int i = i0 + 8 * c;
          uint4 v = make_uint4(0, 0, 0, 0);
          if (r < R && i < m) v = *(const uint4*)(Bq + ((long long)b * R + r) * m + i);
          *(uint4*)(dst + tc::sw128_off(row, c)) = v;
        }
      }
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
#pragma unroll
      for (int kk = 0; kk < OZ_KC / 16; ++kk) {
        const uint32_t ko = kk * 32;   // 16 BF16 = 32 bytes per MMA
#pragma unroll
        for (int l = 0; l < OZ_S; ++l)
#pragma unroll
          for (int a = 0; a <= l; ++a) {
            const int b = l - a;
            const uint32_t acc = (kc > 0 || kk > 0 || a > 0) ? 1u : 0u;
            tc::mma_f16(tmem + l * OZ_N, tc::sw128_desc(tc::smem_u32(sA + a * OZ_A_BYTES) + ko),
                        tc::sw128_desc(tc::smem_u32(sB + b * OZ_B_BYTES) + ko), idesc, acc);
          }
      }
      tc::commit(&mbar[0]);
    }
  }
  tc::mbar_wait(&mbar[0], phase, WAIT_LIMIT) ? (void)0 : (void)(ok = 0);
  ok = __syncthreads_and(ok);
  tc::fence_after();
  if (ok) {
    const int jl = warp * 32 + lane;
    const int j = j0 + jl;
    const int fj = j < m ? fA[j] : 0;
#pragma unroll
    for (int c16 = 0; c16 < OZ_N / 16; ++c16) {
      // levels are exact integers below 2^24 (level l has <= l + 1 digit
      // pairs): combine them exactly in two int64 halves,
      //   hi = sum_{l < H} T_l 2^(7 (H-1-l)),  lo = sum_{l >= H} T_l 2^(7 (S-1-l)),
      // sum_l T_l 2^(-7 l) = 2^(-7 (S-1)) (hi 2^(7 (S-H)) + lo)
      constexpr int H = OZ_S / 2;
      long long hi[16], lo[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) hi[e] = lo[e] = 0;
#pragma unroll
      for (int l = 0; l < OZ_S; ++l) {
        uint32_t v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + l * OZ_N + c16 * 16, v);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const long long t = (long long)__float2int_rz(__uint_as_float(v[e]));
          if (l < H) hi[e] = hi[e] * 128 + t;
          else lo[e] = lo[e] * 128 + t;
        }
      }
      double acc[16];
#pragma unroll
      for (int e = 0; e < 16; ++e)
        acc[e] = fma((double)hi[e], (double)(1LL << (7 * (OZ_S - H))), (double)lo[e]);
      if (j < m) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int rl = c16 * 16 + e;
          const long long r = r0 + rl;
          // Y = scale acc 2^(fA + eB - 2 P + 7 (S - 1)); power of two from its bits
          const int ex = fj + eB[rl] - 2 * OZ_P + 7 * (OZ_S - 1);
          const double p2 = ex > -1023 ? __longlong_as_double((long long)(ex + 1023) << 52) : 0.0;
          if (r < R) Yq[(long long)j * R + r] = scale * ((double)acc[e] * p2);
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, OZ_TMEM_COLS);
}

}  // namespace

int oz_slice_factor(dski_handle h, const double* K, int m, uint16_t* Ad, int* fA) {
  StageScope sc(h, ST_KRON, h->stream);
  k_oz_slice_factor<<<(m + 127) / 128, 128, 0, h->stream>>>(K, m, Ad, fA);
  DSKI_LAUNCHED();
  return DSKI_OK;
}

int mode_tc_oz(dski_handle h, const double* X, const uint16_t* Ad, const int* fA, double* Y,
               int m, long long R, int s, double scale) {
  if (m % 8 != 0 || m > 256)
    return set_error(DSKI_ERR_ARG, "FP64_TC mode products need m_k %% 8 == 0 and m_k <= 256 (got %d)", m);
  const long long rows = (long long)s * R;
  if (h->ozB.ensure((size_t)rows * m * OZ_S * 2) || h->ozE.ensure((size_t)rows * 4))
    return set_error(DSKI_ERR_ALLOC, "FP64_TC digit workspace allocation failed");
  {
    StageScope sc(h, ST_KRON, h->stream);
    k_oz_slice_rows<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, h->stream>>>(
        X, R, m, rows, h->ozB.as<uint16_t>(), h->ozE.as<int>());
  }
  DSKI_LAUNCHED();
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_mode_tc_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
    attr_set = true;
  }
  dim3 grd((unsigned)((m + OZ_M - 1) / OZ_M), (unsigned)((R + OZ_N - 1) / OZ_N), (unsigned)s);
  StageScope sc(h, ST_KRON, h->stream);
  k_mode_tc_oz<<<grd, 128, OZ_SMEM, h->stream>>>(h->ozB.as<uint16_t>(), h->ozE.as<int>(), Ad, fA, Y,
                                                 m, R, scale, h->dev_err.as<int>());
  DSKI_LAUNCHED();
  return DSKI_OK;
}

}  // namespace dski
