// The QR-form preconditioner of Sec. 3.3 applied through the grid.
//
// After r pivoted-Cholesky steps the factor satisfies K[:, P] = L L_P^T
// (P the pivot rows, L_P = L[P, :] lower triangular), so L = K[:, P] L_P^-T.
// In D-SKI, K[:, P] = B K_UU B[P]^T = B H with H = K_UU B[P]^T, and because
// K_UU is Kronecker and each row of B a tensor product of 1-D stencils, every
// column of H is a rank-1 Kronecker product:
//   H[:, k] = s_f^2 (x)_dim h_{k,dim},  h_{k,dim} = K_dim[:, S_{k,dim}] a_{k,dim}
// (S the pivot's four stencil nodes, a its weights or derivative weights).
// With [D^-1/2 L; I] = [Q1; Q2] R, Q1 = D^-1/2 B H T, T = L_P^-T R^-1, and
//   M^-1 r = D^-1/2 (y - Q1 Q1^T y), y = D^-1/2 r
//          = D^-1 (r - B H S H^T B^T D^-1 r),   S = T T^T.
// One apply is a scatter, two grid contractions of M r FMAs each, an r x r
// product and a gather -- instead of two passes over the N x r matrix Q1.
// (The grid buffer gridB of the MVM is free during the apply and holds h'.)
// On the terrain system (M = 65,536 grid nodes, N = 300,000 rows, r = 100)
// that is 13 M FP64 FMAs and L2-resident data against 60 M FMAs over 240 MB.
// Used for d = 2 with M < N and FP64 vectors.
#include <algorithm>
#include <cmath>

#include "solve_internal.cuh"

namespace dski {
namespace {

// h_{k,dim}[u] = sum_o K_dim[u][f + o] a[o] for pivot k (one block per (k, dim)).
__global__ void k_pivot_factors(const int* __restrict__ piv, const int* __restrict__ cell,
                                const double* __restrict__ wt, int d, int mc0, int mc1, int mc2,
                                const double* __restrict__ K0, const double* __restrict__ K1,
                                const double* __restrict__ K2, int m0, int m1, int m2,
                                double sf2, int r, int S, double* __restrict__ Hf) {
  const int k = blockIdx.x, dim = blockIdx.y;
  const int e = piv[k];
  const int j = e / (d + 1), c = e % (d + 1);
  int f[3] = {0, 0, 0};
  {
    int t = cell[j];
    const int mc[3] = {mc0, mc1, mc2};
    for (int q = d - 1; q >= 0; --q) {
      f[q] = t % mc[q];
      t /= mc[q];
    }
  }
  const int m = dim == 0 ? m0 : (dim == 1 ? m1 : m2);
  const double* K = dim == 0 ? K0 : (dim == 1 ? K1 : K2);
  // the point's S weights in this dimension (derivative weights for its
  // gradient row), from the per-point table of 2 S values per dimension
  const double* a = wt + (long long)j * 2 * S * d + 2 * S * dim + (c == dim + 1 ? S : 0);
  // offset of this dimension's block inside Hf: sum of r * m over earlier dims
  long long off = 0;
  if (dim >= 1) off += (long long)r * m0;
  if (dim >= 2) off += (long long)r * m1;
  const double sc = dim == 0 ? sf2 : 1.0;
  for (int u = threadIdx.x; u < m; u += blockDim.x) {
    double v = 0.0;
    for (int o = 0; o < S; ++o) v += K[(long long)u * m + f[dim] + o] * a[o];
    Hf[off + (long long)k * m + u] = sc * v;
  }
}

// LP = L[piv, :] (r x r) gathered from the column-major N x r factor.
__global__ void k_gather_lp(const double* __restrict__ L, long long N, const int* __restrict__ piv,
                            int r, double* __restrict__ LP) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= r * r) return;
  const int k = idx / r, t = idx % r;
  LP[idx] = L[(long long)t * N + piv[k]];   // LP[k][t]
}

// S = T T^T with T = LP^-T Rinv (Rinv = R1^-1 R2^-1, upper), one block.
// W is global scratch; LP^-1 by forward substitution (a column per thread).
__global__ void k_grid_s(const double* __restrict__ LP, const double* __restrict__ R1i,
                         const double* __restrict__ R2i, int r, double* __restrict__ S,
                         double* __restrict__ W) {
  // W: 3 r^2 doubles of global scratch (LPinv, Rinv, T)
  double* LPi = W;
  double* Ri = W + r * r;
  double* T = W + 2 * r * r;
  // LP^-1 (lower): column c by forward substitution
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    for (int i = 0; i < r; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      if (i >= c) {
        for (int k = c; k < i; ++k) v -= LP[i * r + k] * LPi[k * r + c];
        v /= LP[i * r + i];
      } else {
        v = 0.0;
      }
      LPi[i * r + c] = v;
    }
  }
  __syncthreads();
  // Rinv = R1i R2i (both upper)
  for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
    const int a = idx / r, b = idx % r;
    double v = 0.0;
    for (int k = a; k <= b; ++k) v += R1i[a * r + k] * R2i[k * r + b];
    Ri[idx] = a <= b ? v : 0.0;
  }
  __syncthreads();
  // T = LPi^T Ri : T[a][b] = sum_k LPi[k][a] Ri[k][b]
  for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
    const int a = idx / r, b = idx % r;
    double v = 0.0;
    for (int k = 0; k < r; ++k) v += LPi[k * r + a] * Ri[k * r + b];
    T[idx] = v;
  }
  __syncthreads();
  // S = T T^T
  for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
    const int a = idx / r, b = idx % r;
    double v = 0.0;
    for (int k = 0; k < r; ++k) v += T[a * r + k] * T[b * r + k];
    S[idx] = v;
  }
}

// Batched C[q][j][i2] = sum_i A'[q][j][i] B[q][i2][i] (row-major, contraction
// contiguous) with A' = A, or A'[j][i] = x_q[i] A[i][j] (XSCALE: A stored
// transposed, k-major, and scaled on the fly by the per-column vector x).
// FP64: an 8 x 8 output tile per 64-thread block, one output per thread,
// rows staged through shared memory 64 at a time -- small blocks so that the
// ~6.5 M FMAs spread over every SM with enough warps resident to hide
// latency (GB300 runs ~1.6 FP64 FMA per clock per SM).
constexpr int GT = 8;
template <bool XSCALE>
__global__ void __launch_bounds__(GT * GT) k_gemm_nt(const double* __restrict__ A, long long sA,
                                                 const double* __restrict__ B, long long sB,
                                                 double* __restrict__ C, long long sC, int J,
                                                 int I2, int K, const double* __restrict__ x,
                                                 int ldA) {
  constexpr int T = GT, BK = 64;
  __shared__ double As[T][BK + 1];
  __shared__ double Bs[T][BK + 1];
  const int tx = threadIdx.x % T, ty = threadIdx.x / T;
  const int j0 = blockIdx.y * T, n0 = blockIdx.x * T;
  const double* Aq = A + blockIdx.z * sA;
  const double* Bq = B + blockIdx.z * sB;
  const double* xq = XSCALE ? x + (long long)blockIdx.z * K : nullptr;
  double* Cq = C + blockIdx.z * sC;
  double acc = 0.0;
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int idx = threadIdx.x; idx < T * BK; idx += T * T) {
      const int jj = idx / BK, kk = idx % BK;
      const int j = j0 + jj, k = k0 + kk;
      double a = 0.0;
      if (j < J && k < K) a = XSCALE ? xq[k] * Aq[(long long)k * ldA + j] : Aq[(long long)j * K + k];
      As[jj][kk] = a;
      const int n = n0 + jj;
      Bs[jj][kk] = (n < I2 && k < K) ? Bq[(long long)n * K + k] : 0.0;
    }
    __syncthreads();
#pragma unroll 16
    for (int kk = 0; kk < BK; ++kk) acc = fma(As[ty][kk], Bs[tx][kk], acc);
    __syncthreads();
  }
  const int j = j0 + ty, n = n0 + tx;
  if (j < J && n < I2) Cq[(long long)j * I2 + n] = acc;
}

// c[q][k] = sum_u0 H0[k][u0] Y[q][k][u0]: one warp per (q, k).
__global__ void k_grid_c(const double* __restrict__ H0, const double* __restrict__ Y, int r,
                         int m0, int nq, double* __restrict__ c) {
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (wid >= nq * r) return;
  const int q = wid / r, k = wid % r;
  const double* y = Y + ((long long)q * r + k) * m0;
  const double* hk = H0 + (long long)k * m0;
  double v = 0.0;
  for (int u = lane; u < m0; u += 32) v = fma(hk[u], y[u], v);
  v = warp_sum(v);
  if (lane == 0) c[(long long)q * r + k] = v;
}

// x[q] = S c[q]: one warp per (q, output row).
__global__ void k_grid_x(const double* __restrict__ S, const double* __restrict__ c, int r,
                         int nq, double* __restrict__ x) {
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (wid >= nq * r) return;
  const int q = wid / r, a = wid % r;
  double v = 0.0;
  for (int b = lane; b < r; b += 32) v = fma(S[a * r + b], c[(long long)q * r + b], v);
  v = warp_sum(v);
  if (lane == 0) x[(long long)q * r + a] = v;
}

// Y (cols x rp) = X^T (X: rows x cols), zero in columns rows..rp-1.
__global__ void k_transpose_pad(const double* __restrict__ X, int rows, int cols, int rp,
                                double* __restrict__ Y) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= cols * rp) return;
  const int b = idx / rp, a = idx % rp;
  Y[idx] = a < rows ? X[(long long)a * cols + b] : 0.0;
}

__global__ void k_transpose(const double* __restrict__ X, int rows, int cols,
                            double* __restrict__ Y) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int a = idx / cols, b = idx % cols;
  Y[(long long)b * rows + a] = X[idx];
}

}  // namespace

int grid_precond_build(dski_handle h, pivchol_handle pc, const int* piv_dev, const double* R1i,
                       const double* R2i) {
  const int r = pc->rank;
  // every mode: the PCG's r and z are FP64 in the mixed modes too, and the
  // grid form runs in FP64 (its scatter and gather read the FP64 weights)
  if (!(h->d == 2 && (long long)h->M < h->N && r >= 1)) return DSKI_OK;
  const int m0 = h->m[0], m1 = h->m[1];
  cudaStream_t st = h->stream;
  DevBuf LP, W;
  if (pc->Hf.ensure((size_t)r * (m0 + m1) * 8) || pc->H1T.ensure((size_t)r * m1 * 8) ||
      pc->Sg.ensure((size_t)r * r * 8) || LP.ensure((size_t)r * r * 8) ||
      W.ensure((size_t)3 * r * r * 8))
    return set_error(DSKI_ERR_ALLOC, "pivchol_build: allocation of the grid preconditioner failed");
  int rc = DSKI_OK;
  {
    StageScope sc(h, ST_PIVCHOL, st, 5);
    k_pivot_factors<<<dim3(r, 2), 256, 0, st>>>(
        piv_dev, h->cell.as<int>(), h->W64.as<double>(), 2, h->mc[0], h->mc[1], 1,
        h->K64[0].as<double>(), h->K64[1].as<double>(), nullptr, m0, m1, 1, h->sf * h->sf, r,
        h->sw, pc->Hf.as<double>());
    k_transpose<<<(r * m1 + 255) / 256, 256, 0, st>>>(pc->Hf.as<double>() + (size_t)r * m0, r, m1,
                                                      pc->H1T.as<double>());
    k_gather_lp<<<(r * r + 255) / 256, 256, 0, st>>>(pc->L.as<double>(), h->N, piv_dev, r,
                                                     LP.as<double>());
    k_grid_s<<<1, 256, 0, st>>>(LP.as<double>(), R1i, R2i, r, pc->Sg.as<double>(),
                                W.as<double>());
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    rc = set_error(DSKI_ERR_CUDA, "pivchol_build: grid preconditioner: %s",
                   cudaGetErrorString(cudaGetLastError()));
  LP.release();
  W.release();
  if (rc == DSKI_OK) pc->grid_form = true;
  // FP64_TC: digit planes for the two products of the apply
  if (rc == DSKI_OK && h->prec == DSKI_FP64_TC && r <= 256 && m1 % 8 == 0 && m1 <= 256 &&
      m1 >= kOzMinM) {
    const int rp = (r + 7) / 8 * 8;
    if (pc->ozH1.ensure((size_t)kOzDigits * r * m1 * 2) ||
        pc->ozH1T.ensure((size_t)kOzDigits * m1 * rp * 2) ||
        pc->ozE.ensure((size_t)(r + m1) * 4) || pc->H0Tp.ensure((size_t)m0 * rp * 8))
      return set_error(DSKI_ERR_ALLOC, "pivchol_build: FP64_TC preconditioner allocation failed");
    const double* H1 = pc->Hf.as<double>() + (size_t)r * m0;
    DSKI_TRY(oz_slice(h, H1, r, m1, m1, m1, pc->ozH1.as<uint16_t>(), pc->ozE.as<int>(),
                      ST_PIVCHOL));
    DSKI_TRY(oz_slice(h, pc->H1T.as<double>(), m1, r, r, rp, pc->ozH1T.as<uint16_t>(),
                      pc->ozE.as<int>() + r, ST_PIVCHOL));
    {
      StageScope sc(h, ST_PIVCHOL, st);
      k_transpose_pad<<<(m0 * rp + 255) / 256, 256, 0, st>>>(pc->Hf.as<double>(), r, m0, rp,
                                                              pc->H0Tp.as<double>());
    }
    DSKI_LAUNCHED();
    pc->rp = rp;
    pc->oz = true;
  }
  return rc;
}

// Z = M^-1 R for s columns (internal layout) through the grid form.
int grid_precond_apply(dski_handle h, pivchol_handle pc, const double* R, double* Z, int s,
                       const CgUpdate* up, double* dpart_rz, const CgFinish* fin) {
  if ((up || dpart_rz || fin) && s > 4)
    return set_error(DSKI_ERR_ARG, "fused CG steps in the preconditioner need s <= 4");
  const int r = pc->rank;
  const int m0 = h->m[0], m1 = h->m[1];
  const long long M = h->M, N = h->N;
  cudaStream_t st = h->stream;
  for (int c0 = 0; c0 < s; c0 += 4) {
    const int q = std::min(4, s - c0);
    double* g = wbuf(h->s_vec[11], (size_t)M * 4);
    if (pc->gwork.ensure((size_t)4 * ((size_t)r * m0 + 2 * (size_t)r) * 8))
      return set_error(DSKI_ERR_ALLOC, "preconditioner workspace allocation failed");
    double* Yb = pc->gwork.as<double>();                  // q x r x m0
    double* cb = Yb + (size_t)4 * r * m0;                 // q x r
    double* xb = cb + (size_t)4 * r;                      // q x r
    double* hp = wbuf(h->gridB, (size_t)M * 4);           // q x M
    if (!g || !hp) return DSKI_ERR_ALLOC;
    // g = B^T D^-1 R
    DSKI_TRY(scatter_scaled(h, R + (size_t)c0 * N, g, q, true, nullptr, 1.0 / pc->nv,
                            1.0 / pc->ng, up));
    if (pc->oz) {
      // the two products on the tensor cores (FP64-accurate digit products)
      OzGemm g1;   // Y[q][k][u0] = sum_u1 H1[k][u1] g[q][u0][u1]
      g1.Ad = pc->ozH1.as<uint16_t>();
      g1.fA = pc->ozE.as<int>();
      g1.Mrows = r;
      g1.mp = m1;
      g1.X = g;
      g1.ldx = m1;
      g1.xq = M;
      g1.R = m0;
      g1.Y = Yb;
      g1.s = q;
      DSKI_TRY(oz_gemm(h, g1, ST_PRECOND));
      {
        // two launches spread over ~13 SMs each: one block doing both ran the
        // 36k FP64 FMAs on a single SM (~3x slower at GB300's FP64 rate)
        StageScope sc(h, ST_PRECOND, st, 2);
        k_grid_c<<<(q * r * 32 + 255) / 256, 256, 0, st>>>(pc->Hf.as<double>(), Yb, r, m0, q, cb);
        k_grid_x<<<(q * r * 32 + 255) / 256, 256, 0, st>>>(pc->Sg.as<double>(), cb, r, q, xb);
      }
      DSKI_LAUNCHED();
      OzGemm g2;   // h'[q][u0][u1] = sum_k H1T[u1][k] x_k H0T[u0][k]
      g2.Ad = pc->ozH1T.as<uint16_t>();
      g2.fA = pc->ozE.as<int>() + r;
      g2.Mrows = m1;
      g2.mp = pc->rp;
      g2.X = pc->H0Tp.as<double>();
      g2.ldx = pc->rp;
      g2.xq = 0;
      g2.R = m0;
      g2.xs = xb;
      g2.xsq = r;
      g2.xsn = r;
      g2.Y = hp;
      g2.ytrans = true;
      g2.s = q;
      DSKI_TRY(oz_gemm(h, g2, ST_PRECOND));
    } else {
      StageScope sc(h, ST_PRECOND, st, 4);
      // Y[q][k][u0] = sum_u1 H1[k][u1] g[q][u0][u1]
      k_gemm_nt<false><<<dim3((m0 + GT - 1) / GT, (r + GT - 1) / GT, q), GT * GT, 0, st>>>(
          pc->Hf.as<double>() + (size_t)r * m0, 0, g, M, Yb, (long long)r * m0, r, m0, m1,
          nullptr, 0);
      k_grid_c<<<(q * r * 32 + 255) / 256, 256, 0, st>>>(pc->Hf.as<double>(), Yb, r, m0, q, cb);
      k_grid_x<<<(q * r * 32 + 255) / 256, 256, 0, st>>>(pc->Sg.as<double>(), cb, r, q, xb);
      // h'[q][u0][u1] = sum_k x_k H0[k][u0] H1[k][u1]
      k_gemm_nt<true><<<dim3((m1 + GT - 1) / GT, (m0 + GT - 1) / GT, q), GT * GT, 0, st>>>(
          pc->Hf.as<double>(), 0, pc->H1T.as<double>(), 0, hp, M, m0, m1, r, xb, m0);
    }
    DSKI_LAUNCHED();
    // Z = (R - B h') ./ noise
    // (FP64 even in FP64_TC: r - B h' cancels in the top eigen-directions,
    // amplifying the gather's rounding by ~lambda_max / sigma^2; its
    // double-float form took 22% more PCG iterations on the terrain solve)
    DSKI_TRY(gather_scaled(h, hp, R + (size_t)c0 * N, Z + (size_t)c0 * N, q, -1.0 / pc->nv,
                           -1.0 / pc->ng, 1.0 / pc->nv, 1.0 / pc->ng, ST_PRECOND, dpart_rz, fin));
  }
  return DSKI_OK;
}

}  // namespace dski
