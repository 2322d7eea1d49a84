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
// Both operands are split into S = 8 signed 7-bit digits relative to a
// per-row power of two (Ozaki-style splitting): for a row with max |x| <
// 2^e, x = 2^e sum_b d_b 2^(-6 - 7 b) up to rounding at 2^(e - 55), d_b
// integers in [-64, 64] (exact in BF16), extracted with integer arithmetic.
// A product of digits is at most 2^12 in magnitude and a sum of m <= 256 of
// them, over the <= 8 digit pairs (a, b) of one level a + b, stays within
// 2^23, so every level accumulates EXACTLY in the FP32 TMEM accumulator.
// Levels 0..S-1 are kept (one TMEM accumulator each) and combined in FP64:
//   Y[j][r] = 2^(fA_j + eB_r - 12) sum_l 2^(-7 l) T_l[j][r],
// (summed exactly in two int64 halves), which drops only the digit pairs of
// weight < 2^(-7 S) -- a relative error of about 2^-53 of |K| |X|, at FP64
// rounding in the 256-term sums (the FP32 product misses by 2^-24, 26x the
// noise variance on the terrain grid).
// K's digits are made once per factor; X's digits by a row-parallel kernel
// before each mode product.
constexpr int OZ_S = kOzDigits;                  // digits per operand (8)
constexpr int OZ_P = 6 + 7 * (OZ_S - 1);         // fixed-point bits: |V| < 2^OZ_P
static_assert(OZ_P <= 62 && OZ_P - 53 <= 8, "fixed-point range");
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

// One split of the contraction: the exact FP32 level sums
//   T_l[j][r] = sum_{a + b = l} sum_{i in split} A_a[j][i] B_b[r][i]
// of a 128 x 32 output tile, written as int32 to P[q][split][l][j][r].  The
// digit planes stream in by TMA (64-byte rows, 64-byte swizzle, box 32 wide)
// through two stages; one thread issues the loads and the 36 MMAs per
// 16-deep step; stages are recycled when their MMAs commit.  Splitting the
// contraction over CTAs puts 64 CTAs on a 256 x 256 mode product.
constexpr int Z_M = 128, Z_N = 32, Z_KC = 32;    // 32 BF16 = one 64-byte row
constexpr int Z_A = Z_M * 64;                     // 8 KB per digit plane
constexpr int Z_B = Z_N * 64;                     // 2 KB per digit plane
constexpr int Z_STAGE = OZ_S * (Z_A + Z_B);       // 80 KB
constexpr int Z_SMEM = 2 * Z_STAGE + 1024 + 128;
static_assert(OZ_S * Z_N <= 256, "TMEM columns");

__global__ void __launch_bounds__(128) k_oz_gemm(const __grid_constant__ CUtensorMap tA,
                                                 const __grid_constant__ CUtensorMap tB,
                                                 int* __restrict__ P, int m, long long R,
                                                 int KS, int kper, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + 2 * Z_STAGE);
  uint64_t* empty = full + 2;
  uint64_t* done = full + 4;
  uint32_t* tslot = (uint32_t*)(full + 5);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = blockIdx.x * Z_M;
  const int r0 = blockIdx.y * Z_N;
  const int z = blockIdx.z, q = z / KS, ks = z % KS;
  const int k_begin = ks * kper;
  const int k_end = min(m, k_begin + kper);
  const int nch = (k_end - k_begin + Z_KC - 1) / Z_KC;   // >= 1 by construction

  if (warp == 0) tc::tmem_alloc(tslot, 256);
  if (tid == 0) {
    for (int i = 0; i < 5; ++i) tc::mbar_init(&full[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = tc::instr_desc(tc::kFmtBF16, Z_M, Z_N);

  int ok = 1;
  if (tid == 0) {
    int issued = 0, consumed = 0;
    auto issue = [&](int c) {
      const int st = c & 1;
      unsigned char* base = smem + st * Z_STAGE;
      tc::mbar_expect_tx(&full[st], (uint32_t)Z_STAGE);
      const int i0 = k_begin + c * Z_KC;
      for (int b = 0; b < OZ_S; ++b) {
        tc::tma_load_3d(base + b * Z_A, &tA, i0, j0, b, &full[st]);
        tc::tma_load_4d(base + OZ_S * Z_A + b * Z_B, &tB, i0, r0, b, q, &full[st]);
      }
      issued = c + 1;
    };
    issue(0);
    if (nch > 1) issue(1);
    for (int c = 0; c < nch; ++c) {
      const int st = c & 1;
      const uint32_t ph = (uint32_t)((c >> 1) & 1);
      if (!tc::mbar_wait(&full[st], ph, WAIT_LIMIT)) {
        ok = 0;
        break;
      }
      consumed = c + 1;
      tc::fence_after();
      const uint32_t aB = tc::smem_u32(smem + st * Z_STAGE);
      const uint32_t bB = aB + OZ_S * Z_A;
#pragma unroll
      for (int kk = 0; kk < Z_KC / 16; ++kk) {
        const uint32_t ko = kk * 32;   // 16 BF16 = 32 bytes per MMA
#pragma unroll
        for (int l = 0; l < OZ_S; ++l)
#pragma unroll
          for (int a = 0; a <= l; ++a) {
            const uint32_t acc = (c > 0 || kk > 0 || a > 0) ? 1u : 0u;
            tc::mma_f16(tmem + l * Z_N, tc::sw64_desc(aB + a * Z_A + ko),
                        tc::sw64_desc(bB + (l - a) * Z_B + ko), idesc, acc);
          }
      }
      tc::commit(&empty[st]);
      if (c + 2 < nch) {
        if (!tc::mbar_wait(&empty[st], ph, WAIT_LIMIT)) {
          ok = 0;
          break;
        }
        issue(c + 2);
      }
    }
    tc::commit(done);   // arrives once every MMA issued above has completed
    // after a timeout, let the loads still in flight land before the CTA
    // leaves (bounded as well)
    for (int c = consumed; c < issued; ++c)
      tc::mbar_wait(&full[c & 1], (uint32_t)((c >> 1) & 1), WAIT_LIMIT);
  }
  __syncthreads();
  int fin = tc::mbar_wait(done, 0, WAIT_LIMIT) ? 1 : 0;
  fin = __syncthreads_and(fin && (tid != 0 || ok));
  tc::fence_after();
  if (fin) {
    const int j = j0 + warp * 32 + lane;
    int* Pz = P + (long long)z * OZ_S * m * R;
    const bool vec = (R & 3) == 0;   // rows 16-byte aligned
#pragma unroll 1
    for (int l = 0; l < OZ_S; ++l) {
#pragma unroll
      for (int c16 = 0; c16 < Z_N / 16; ++c16) {
        uint32_t v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + l * Z_N + c16 * 16, v);
        const long long rc = r0 + c16 * 16;
        if (j < m) {
          int* row = Pz + ((long long)l * m + j) * R + rc;
          if (vec && rc + 16 <= R) {
#pragma unroll
            for (int e = 0; e < 16; e += 4)
              *reinterpret_cast<int4*>(row + e) =
                  make_int4(__float2int_rz(__uint_as_float(v[e])),
                            __float2int_rz(__uint_as_float(v[e + 1])),
                            __float2int_rz(__uint_as_float(v[e + 2])),
                            __float2int_rz(__uint_as_float(v[e + 3])));
          } else {
#pragma unroll
            for (int e = 0; e < 16; ++e)
              if (rc + e < R) row[e] = __float2int_rz(__uint_as_float(v[e]));
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// Y[q][j][r] = scale 2^(fA_j + eB_qr - 2 P + 7 (S - 1)) sum_l 2^(7 (S-1-l)) sum_split T_l,
// the level sums combined exactly in two int64 halves.
__global__ void k_oz_combine(const int* __restrict__ P, const int* __restrict__ fA,
                             const int* __restrict__ eB, double* __restrict__ Y, int m,
                             long long R, int KS, int s, double scale) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)m * R;
  if (idx >= per * s) return;
  const long long q = idx / per, jr = idx % per;
  const int j = (int)(jr / R);
  const long long r = jr % R;
  constexpr int H = OZ_S / 2;
  long long hi = 0, lo = 0;
#pragma unroll
  for (int l = 0; l < OZ_S; ++l) {
    long long t = 0;
    for (int k = 0; k < KS; ++k) t += P[(((q * KS + k) * OZ_S + l) * m) * R + jr];
    if (l < H) hi = hi * 128 + t;
    else lo = lo * 128 + t;
  }
  const double acc = fma((double)hi, (double)(1LL << (7 * (OZ_S - H))), (double)lo);
  const int ex = fA[j] + eB[q * R + r] - 2 * OZ_P + 7 * (OZ_S - 1);
  const double p2 = ex > -1023 ? __longlong_as_double((long long)(ex + 1023) << 52) : 0.0;
  Y[q * per + jr] = scale * (acc * p2);
}

}  // namespace

int oz_slice_factor(dski_handle h, const double* K, int m, uint16_t* Ad, int* fA) {
  StageScope sc(h, ST_KRON, h->stream);
  k_oz_slice_factor<<<(m + 127) / 128, 128, 0, h->stream>>>(K, m, Ad, fA);
  DSKI_LAUNCHED();
  return DSKI_OK;
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

// BF16 digit planes as a TMA tensor: dims (innermost first) and byte
// strides of the outer dims; box Z_KC x rows x 1 (x 1), 64-byte swizzle.
static int encode_digits(CUtensorMap* map, const void* base, int rank, const cuuint64_t* dims,
                         const cuuint64_t* strides, cuuint32_t box_rows) {
  auto enc = tensor_map_encoder();
  if (!enc) return set_error(DSKI_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  cuuint32_t box[4] = {(cuuint32_t)Z_KC, box_rows, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank,
                         const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(DSKI_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return DSKI_OK;
}

int mode_tc_oz(dski_handle h, const double* X, const uint16_t* Ad, const int* fA, double* Y,
               int m, long long R, int s, double scale) {
  if (m % 8 != 0 || m > 256)
    return set_error(DSKI_ERR_ARG, "FP64_TC mode products need m_k %% 8 == 0 and m_k <= 256 (got %d)", m);
  const long long rows = (long long)s * R;
  // contraction split: up to 4 splits of >= 64 (whole 32-wide chunks each)
  int KS = std::max(1, std::min(4, m / 64)), kper = m;
  for (;; --KS) {   // every split must start inside [0, m)
    kper = ((m + KS - 1) / KS + Z_KC - 1) / Z_KC * Z_KC;
    if (KS == 1 || (long long)(KS - 1) * kper < m) break;
  }
  if (h->ozB.ensure((size_t)rows * m * OZ_S * 2) || h->ozE.ensure((size_t)rows * 4) ||
      h->ozP.ensure((size_t)s * KS * OZ_S * m * R * 4))
    return set_error(DSKI_ERR_ALLOC, "FP64_TC digit workspace allocation failed");
  {
    StageScope sc(h, ST_KRON, h->stream);
    k_oz_slice_rows<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, h->stream>>>(
        X, R, m, rows, h->ozB.as<uint16_t>(), h->ozE.as<int>());
  }
  DSKI_LAUNCHED();
  CUtensorMap tA, tB;
  {
    const cuuint64_t dims[3] = {(cuuint64_t)m, (cuuint64_t)m, (cuuint64_t)OZ_S};
    const cuuint64_t str[2] = {(cuuint64_t)m * 2, (cuuint64_t)m * m * 2};
    DSKI_TRY(encode_digits(&tA, Ad, 3, dims, str, Z_M));
  }
  {
    const cuuint64_t dims[4] = {(cuuint64_t)m, (cuuint64_t)R, (cuuint64_t)OZ_S, (cuuint64_t)s};
    const cuuint64_t str[3] = {(cuuint64_t)m * 2, (cuuint64_t)R * m * 2,
                               (cuuint64_t)OZ_S * R * m * 2};
    DSKI_TRY(encode_digits(&tB, h->ozB.ptr, 4, dims, str, Z_N));
  }
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, Z_SMEM);
    attr_set = true;
  }
  dim3 grd((unsigned)((m + Z_M - 1) / Z_M), (unsigned)((R + Z_N - 1) / Z_N), (unsigned)(s * KS));
  {
    StageScope sc(h, ST_KRON, h->stream, 2);
    k_oz_gemm<<<grd, 128, Z_SMEM, h->stream>>>(tA, tB, h->ozP.as<int>(), m, R, KS, kper,
                                                h->dev_err.as<int>());
    const long long tot = (long long)s * m * R;
    k_oz_combine<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(
        h->ozP.as<int>(), fA, h->ozE.as<int>(), Y, m, R, KS, s, scale);
  }
  DSKI_LAUNCHED();
  return DSKI_OK;
}

}  // namespace dski
