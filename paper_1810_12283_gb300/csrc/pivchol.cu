// Truncated pivoted Cholesky of the noise-free D-SKI matrix and the QR-form
// preconditioner of Sec. 3.3.
//
// The D-SKI matrix is K = B K_UU B^T with K_UU = s_f^2 K_1 (x) ... (x) K_d.
// Because K_UU is a Kronecker product and every row of B is a tensor product
// of per-dimension S-point stencils (S = 4 cubic, 6 quintic), entries of K
// factor over dimensions:
//   K[(i,c), (j,c')] = s_f^2 prod_k  a_ik^(c)T  K_k[S_ik, S_jk]  a_jk^(c'),
// where S_ik are the S stencil nodes of point i in dimension k and a_ik^(c)
// its interpolation weights (derivative weights / h_k in dimension c-1 when
// c >= 1).  On a regular grid K_k is Toeplitz, K_k[u, v] = kappa_k(|u - v|),
// so the diagonal needs only the S x S block kappa_k(|o - o'|) and a pivot
// row needs only kappa_k at the offsets between two stencils: the method of
// Sec. 3.3 (only the diagonal and the pivot rows are formed) at O(d S^2) per
// entry, without forming the grid.
//
// Greedy pivoting: the pivot is the largest residual diagonal entry; ties go
// to the lowest row index in the caller's block order.  After r steps (or
// when the residual trace drops below 1e-14 of the initial trace) the
// preconditioner M = D + L L^T is put in the QR-stable form
//   [D^-1/2 L; I] = [Q1; Q2] R
// by two CholeskyQR passes in FP64 (R = R2 R1), and
//   log|M| = sum log D + 2 sum log diag(R).
#include <algorithm>
#include <cmath>
#include <new>

#include "interp.cuh"
#include "solve_internal.cuh"

namespace dski {
namespace {

struct PcGeo {
  int d, n;
  long long N;
  int m[DSKI_MAXD];
  int mc[DSKI_MAXD];
  double invh[DSKI_MAXD];
  double sf2;
  const double* kap[DSKI_MAXD];   // first row of K_k: kappa_k(delta), delta = 0..m_k-1
};

struct PcState {
  int pivot;      // internal row of the next pivot
  int stop;       // 1 once the factorisation stopped
  int steps;      // columns produced
  int pad;
  double trace0;  // initial trace
  double dpiv;    // residual diagonal at the pivot
  double trace;   // current residual trace
};

struct ArgMax {
  double v;
  long long u;   // caller block-order index (tie-break)
  long long e;   // internal row
};

__device__ __forceinline__ bool better(const ArgMax& a, const ArgMax& b) {
  return a.v > b.v || (a.v == b.v && a.u < b.u);
}

__device__ __forceinline__ void cell_coords(const PcGeo& g, int cell, int f[DSKI_MAXD]) {
  for (int k = g.d - 1; k >= 0; --k) {
    f[k] = cell % g.mc[k];
    cell /= g.mc[k];
  }
}

// Block-wide argmax + sum; thread 0 writes the block's partials.
__device__ void block_argmax_sum(ArgMax best, double tr, ArgMax* sh, double* shs,
                                 ArgMax* part_a, double* part_s) {
  sh[threadIdx.x] = best;
  shs[threadIdx.x] = tr;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      if (better(sh[threadIdx.x + o], sh[threadIdx.x])) sh[threadIdx.x] = sh[threadIdx.x + o];
      shs[threadIdx.x] += shs[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part_a[blockIdx.x] = sh[0];
    part_s[blockIdx.x] = shs[0];
  }
}

// Last block: reduce the partials in block order and set the next pivot.
__device__ void finish_pivot(int nblocks, const ArgMax* part_a, const double* part_s,
                             PcState* st, int step, int* piv_list, int first, int pivot_done) {
  if (threadIdx.x != 0) return;
  ArgMax b = part_a[0];
  double tr = part_s[0];
  for (int i = 1; i < nblocks; ++i) {
    if (better(part_a[i], b)) b = part_a[i];
    tr += part_s[i];
  }
  if (first) {
    st->trace0 = tr;
    st->steps = 0;
    st->stop = 0;
  } else {
    piv_list[step] = pivot_done;
    st->steps = step + 1;
  }
  st->trace = tr;
  st->pivot = (int)b.e;
  st->dpiv = b.v;
  if (!(b.v > 0.0) || !(tr > 1e-14 * st->trace0)) st->stop = 1;
}

template <int D, int S>
__device__ __forceinline__ void point_weights(const PcGeo& g, const double* frac, long long j,
                                              double w[D][S], double dw[D][S]) {
#pragma unroll
  for (int k = 0; k < D; ++k) {
    stencil_weights<S, double>(frac[j * D + k], w[k], dw[k]);
#pragma unroll
    for (int o = 0; o < S; ++o) dw[k][o] *= g.invh[k];
  }
}

template <int D, int S>
__global__ void __launch_bounds__(256) k_pc_diag(PcGeo g, const int* __restrict__ cell,
                                                 const double* __restrict__ frac,
                                                 const int* __restrict__ perm,
                                                 double* __restrict__ Dg, ArgMax* part_a,
                                                 double* part_s, unsigned* ticket,
                                                 PcState* st) {
  __shared__ ArgMax sh[256];
  __shared__ double shs[256];
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  ArgMax best{-1.0, 0x7fffffffffffffffLL, 0};
  double tr = 0.0;
  if (j < g.n) {
    double w[D][S], dw[D][S];
    point_weights<D, S>(g, frac, j, w, dw);
    double qw[D], qd[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      double a = 0.0, b = 0.0;
#pragma unroll
      for (int o = 0; o < S; ++o)
#pragma unroll
        for (int o2 = 0; o2 < S; ++o2) {
          const double kv = g.kap[k][o > o2 ? o - o2 : o2 - o];
          a += w[k][o] * kv * w[k][o2];
          b += dw[k][o] * kv * dw[k][o2];
        }
      qw[k] = a;
      qd[k] = b;
    }
    const int pi = perm[j];
#pragma unroll
    for (int c = 0; c <= D; ++c) {
      double v = g.sf2;
#pragma unroll
      for (int k = 0; k < D; ++k) v *= (c == k + 1) ? qd[k] : qw[k];
      const long long e = j * (D + 1) + c;
      Dg[e] = v;
      tr += v;
      const ArgMax cand{v, (long long)c * g.n + pi, e};
      if (better(cand, best)) best = cand;
    }
  }
  block_argmax_sum(best, tr, sh, shs, part_a, part_s);
  if (last_block(ticket, gridDim.x)) finish_pivot(gridDim.x, part_a, part_s, st, 0, nullptr, 1, 0);
}

template <int D, int S>
__global__ void __launch_bounds__(256) k_pc_step(PcGeo g, const int* __restrict__ cell,
                                                 const double* __restrict__ frac,
                                                 const int* __restrict__ perm,
                                                 double* __restrict__ Dg, double* __restrict__ L,
                                                 int step, ArgMax* part_a, double* part_s,
                                                 unsigned* ticket, PcState* st,
                                                 int* piv_list) {
  __shared__ ArgMax sh[256];
  __shared__ double shs[256];
  __shared__ double Lp[128];
  __shared__ double ap[D][S];
  __shared__ int fp[D];
  if (st->stop) return;   // uniform across the grid: written by an earlier launch
  const long long ep = st->pivot;
  const double dp = st->dpiv;
  const long long jp = ep / (D + 1);
  const int cp = (int)(ep % (D + 1));
  for (int t = threadIdx.x; t < step; t += blockDim.x) Lp[t] = L[(long long)t * g.N + ep];
  if (threadIdx.x == 0) {
    int f[DSKI_MAXD];
    cell_coords(g, cell[jp], f);
    double w[D][S], dw[D][S];
    point_weights<D, S>(g, frac, jp, w, dw);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      fp[k] = f[k];
#pragma unroll
      for (int o = 0; o < S; ++o) ap[k][o] = (cp == k + 1) ? dw[k][o] : w[k][o];
    }
  }
  __syncthreads();
  const double inv_sq = 1.0 / sqrt(dp);
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  ArgMax best{-1.0, 0x7fffffffffffffffLL, 0};
  double tr = 0.0;
  if (j < g.n) {
    int f[DSKI_MAXD];
    cell_coords(g, cell[j], f);
    double w[D][S], dw[D][S];
    point_weights<D, S>(g, frac, j, w, dw);
    double Wk[D], Dk[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      double a = 0.0, b = 0.0;
#pragma unroll
      for (int o = 0; o < S; ++o) {
        double hk = 0.0;
#pragma unroll
        for (int o2 = 0; o2 < S; ++o2) {
          const int delta = abs(f[k] + o - fp[k] - o2);
          hk += g.kap[k][delta] * ap[k][o2];
        }
        a += w[k][o] * hk;
        b += dw[k][o] * hk;
      }
      Wk[k] = a;
      Dk[k] = b;
    }
    const int pi = perm[j];
#pragma unroll
    for (int c = 0; c <= D; ++c) {
      double row = g.sf2;
#pragma unroll
      for (int k = 0; k < D; ++k) row *= (c == k + 1) ? Dk[k] : Wk[k];
      const long long e = j * (D + 1) + c;
      double acc = row;
      for (int t = 0; t < step; ++t) acc -= L[(long long)t * g.N + e] * Lp[t];
      const double col = acc * inv_sq;
      L[(long long)step * g.N + e] = col;
      double dn = Dg[e];
      dn = (e == ep || dn <= 0.0) ? 0.0 : dn - col * col;
      if (dn < 0.0) dn = 0.0;
      Dg[e] = dn;
      tr += dn;
      const ArgMax cand{dn, (long long)c * g.n + pi, e};
      if (better(cand, best)) best = cand;
    }
  }
  block_argmax_sum(best, tr, sh, shs, part_a, part_s);
  if (last_block(ticket, gridDim.x))
    finish_pivot(gridDim.x, part_a, part_s, st, step, piv_list, 0, (int)ep);
}

// In-place Cholesky G = R^T R (upper R) of an r x r SPD matrix, optionally
// after G += I (add_identity) and G += T^T T (T upper triangular, may be
// NULL); also R^-1 and sum log diag(R).  One block; G in dynamic shared
// memory (r <= 128).  flag is set to 1 if G is not numerically PD.
__global__ void k_small_chol(const double* __restrict__ Gin, int r, int add_identity,
                             const double* __restrict__ T, double* __restrict__ R,
                             double* __restrict__ Rinv, double* __restrict__ logdiag,
                             int* __restrict__ flag) {
  extern __shared__ double G[];   // r x r
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
    const int a = idx / r, b = idx % r;
    double v = Gin[idx];
    if (add_identity && a == b) v += 1.0;
    if (T) {
      double t = 0.0;
      for (int k = 0; k <= min(a, b); ++k) t += T[k * r + a] * T[k * r + b];
      v += t;
    }
    G[idx] = v;
  }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (threadIdx.x == 0) {
      const double djj = G[j * r + j];
      if (!(djj > 0.0) || !isfinite(djj)) bad = 1;
      G[j * r + j] = sqrt(fmax(djj, 1e-300));
    }
    __syncthreads();
    const double rjj = G[j * r + j];
    for (int k = j + 1 + threadIdx.x; k < r; k += blockDim.x) G[j * r + k] /= rjj;
    __syncthreads();
    // trailing update G[a][b] -= R[j][a] R[j][b] for j < a <= b
    const int rem = r - j - 1;
    for (int idx = threadIdx.x; idx < rem * rem; idx += blockDim.x) {
      const int a = j + 1 + idx / rem, b = j + 1 + idx % rem;
      if (b >= a) G[a * r + b] -= G[j * r + a] * G[j * r + b];
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
    const int a = idx / r, b = idx % r;
    R[idx] = b >= a ? G[idx] : 0.0;
  }
  // R^-1 by back substitution, one column per thread
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    for (int i = r - 1; i >= 0; --i) {
      double v = (i == c) ? 1.0 : 0.0;
      if (i <= c) {
        for (int k = i + 1; k <= c; ++k) v -= G[i * r + k] * Rinv[k * r + c];
        v /= G[i * r + i];
      }
      Rinv[i * r + c] = (i <= c) ? v : 0.0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < r; ++i) s += log(G[i * r + i]);
    *logdiag = s;
    if (bad) *flag = 1;
  }
}

__global__ void k_inv_sqrt_noise(int n, int d, double nv, double ng, double* __restrict__ dis,
                                 double* __restrict__ ds) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * (d + 1)) return;
  const double v = (e % (d + 1)) == 0 ? nv : ng;
  dis[e] = 1.0 / sqrt(v);
  ds[e] = sqrt(v);
}

// the diagonal, then `rank` pivot steps (each stops itself once the
// factorisation has stopped)
template <int D, int S>
void launch_pc(dski_handle h, const PcGeo& g, unsigned nb, int rank, double* Dg, double* L,
               ArgMax* part_a, double* part_s, unsigned* tk, PcState* stt, int* piv_list,
               cudaStream_t st) {
  k_pc_diag<D, S><<<nb, 256, 0, st>>>(g, h->cell.as<int>(), h->frac64.as<double>(),
                                      h->perm.as<int>(), Dg, part_a, part_s, tk, stt);
  for (int k = 0; k < rank; ++k)
    k_pc_step<D, S><<<nb, 256, 0, st>>>(g, h->cell.as<int>(), h->frac64.as<double>(),
                                        h->perm.as<int>(), Dg, L, k, part_a, part_s, tk, stt,
                                        piv_list);
}

PcGeo make_pcgeo(dski_handle h) {
  PcGeo g{};
  g.d = h->d;
  g.n = h->n;
  g.N = h->N;
  for (int k = 0; k < DSKI_MAXD; ++k) {
    g.m[k] = k < h->d ? h->m[k] : 1;
    g.mc[k] = k < h->d ? h->mc[k] : 1;
    g.invh[k] = k < h->d ? 1.0 / h->h[k] : 1.0;
    g.kap[k] = k < h->d ? h->K64[k].as<double>() : nullptr;
  }
  g.sf2 = h->sf * h->sf;
  return g;
}

// layout of the build's state buffer
constexpr size_t kPivOff = 64;                  // PcState fits in 64 bytes
constexpr size_t kFlagOff = kPivOff + 128 * 4;  // pivots of up to 128 steps
constexpr size_t kSmallOff = kFlagOff + 64;     // r x r matrices (8-byte aligned)
static_assert(sizeof(PcState) <= kPivOff, "PcState grew");

void free_pc(pivchol_handle pc) {
  if (!pc) return;
  pc->L.release();
  pc->Q1.release();
  pc->Qh.release();
  pc->Ql.release();
  pc->Hf.release();
  pc->H1T.release();
  pc->Sg.release();
  pc->ozH1.release();
  pc->ozH1T.release();
  pc->ozE.release();
  pc->H0Tp.release();
  pc->gwork.release();
  pc->dis.release();
  pc->ds.release();
  delete pc;
}

}  // namespace

// CholeskyQR2 of [D^-1/2 L; I]: Q1 = D^-1/2 L R1^-1 R2^-1, log|M|.
static int qr_form(dski_handle h, pivchol_handle pc, int* flag_dev, double* small,
                   const int* piv_dev) {
  const int r = pc->rank;
  const long long N = h->N;
  cudaStream_t st = h->stream;
  double* G = small;               // r x r
  double* R1 = G + r * r;
  double* R1i = R1 + r * r;
  double* R2 = R1i + r * r;
  double* R2i = R2 + r * r;
  double* ld = R2i + r * r;        // 2 log-diag sums
  DevBuf Q1a;
  if (Q1a.ensure((size_t)N * r * 8) || pc->Q1.ensure((size_t)N * r * 8))
    return set_error(DSKI_ERR_ALLOC, "pivchol_build: allocation of Q1 failed");
  const size_t smem = (size_t)r * r * 8;
  cudaFuncSetAttribute(k_small_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int rc = DSKI_OK;
  do {
    // pass 1: G = L^T D^-1 L (+ I inside the factorisation)
    double* dinv = wbuf(h->s_vec[8], (size_t)N);
    if (!dinv) { rc = DSKI_ERR_ALLOC; break; }
    // dinv = dis .* dis
    rc = ts_nn(h, pc->dis.as<double>(), 1.0, pc->dis.as<double>(), 0.0, nullptr, 0, nullptr, 1,
               dinv, nullptr);
    if (rc) break;
    rc = ts_tn(h, pc->L.as<double>(), r, pc->L.as<double>(), r, dinv, G);
    if (rc) break;
    {
      StageScope sc(h, ST_PIVCHOL, st);
      k_small_chol<<<1, 256, smem, st>>>(G, r, 1, nullptr, R1, R1i, ld, flag_dev);
    }
    DSKI_LAUNCHED();
    rc = ts_nn(h, nullptr, 0.0, nullptr, 1.0, pc->L.as<double>(), r, R1i, r, Q1a.as<double>(),
               pc->dis.as<double>());
    if (rc) break;
    // pass 2: G2 = Q1a^T Q1a + R1^-T R1^-1
    rc = ts_tn(h, Q1a.as<double>(), r, Q1a.as<double>(), r, nullptr, G);
    if (rc) break;
    {
      StageScope sc(h, ST_PIVCHOL, st);
      k_small_chol<<<1, 256, smem, st>>>(G, r, 0, R1i, R2, R2i, ld + 1, flag_dev);
    }
    DSKI_LAUNCHED();
    rc = ts_nn(h, nullptr, 0.0, nullptr, 1.0, Q1a.as<double>(), r, R2i, r, pc->Q1.as<double>(),
               nullptr);
    if (rc) break;
    double hld[2] = {0, 0};
    if (cudaMemcpyAsync(hld, ld, sizeof(hld), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = set_error(DSKI_ERR_CUDA, "pivchol_build: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    pc->logdetM += 2.0 * (hld[0] + hld[1]);
    rc = grid_precond_build(h, pc, piv_dev, R1i, R2i);
    if (rc) break;
    // the FP32 (MIXED) modes apply Q1 in double-float arithmetic; FP64 and
    // FP64_TC keep it in FP64: the QR-form apply cancels in the top
    // eigen-directions, amplifying its rounding by ~1 + lambda_max / sigma^2
    // (2^-44 double-float stalled PCG at 1.5e-6 where FP64 reached 2.5e-9)
    // (the grid form, where it applies, replaces the Q1 apply in every mode)
    if (!f64_vectors(h) && !pc->grid_form) {
      rc = split_q1(h, pc);
      if (rc) break;
    }
  } while (0);
  cudaStreamSynchronize(st);
  Q1a.release();
  return rc;
}

}  // namespace dski

using namespace dski;

extern "C" int pivchol_build(dski_handle h, int rank, pivchol_handle* out, int* rank_achieved) {
  clear_error();
  if (!out) return set_error(DSKI_ERR_ARG, "pivchol_build: out is NULL");
  *out = nullptr;
  if (!h) return set_error(DSKI_ERR_ARG, "pivchol_build: NULL handle");
  if (rank < 1 || rank > 128) return set_error(DSKI_ERR_ARG, "pivchol_build: rank must be in 1..128");
  const long long N = h->N;
  rank = (int)std::min<long long>(rank, N);
  pivchol_handle pc = new (std::nothrow) pivchol_();
  if (!pc) return set_error(DSKI_ERR_ALLOC, "pivchol_build: host allocation failed");
  pc->h = h;
  pc->N = h->N;
  pc->nv = h->nv;
  pc->ng = h->ng;
  cudaStream_t st = h->stream;
  const int nb = (int)((h->n + 255) / 256);
  DevBuf Dg, state;
  int rc = DSKI_OK;
  do {
    if (pc->L.ensure((size_t)N * rank * 8) || pc->dis.ensure((size_t)N * 8) ||
        pc->ds.ensure((size_t)N * 8) || Dg.ensure((size_t)N * 8) ||
        state.ensure(kSmallOff + 6 * 128 * 128 * 8 + 64)) {
      rc = set_error(DSKI_ERR_ALLOC, "pivchol_build: device allocation failed");
      break;
    }
    PcState* stt = (PcState*)state.ptr;
    int* piv_list = (int*)((char*)state.ptr + kPivOff);
    int* flag = (int*)((char*)state.ptr + kFlagOff);
    double* small = (double*)((char*)state.ptr + kSmallOff);
    double* part = wbuf(h->s_part, (size_t)nb * 4);
    unsigned* tk = tickets(h, 1);
    if (!part || !tk) { rc = set_error(DSKI_ERR_ALLOC, "pivchol_build: workspace"); break; }
    ArgMax* part_a = (ArgMax*)part;
    double* part_s = part + (size_t)nb * 3;
    if (cudaMemsetAsync(state.ptr, 0, kSmallOff, st) != cudaSuccess) {
      rc = set_error(DSKI_ERR_CUDA, "pivchol_build: memset failed");
      break;
    }
    const PcGeo g = make_pcgeo(h);
    {
      StageScope sc(h, ST_PIVCHOL, st, 1 + rank);
      with_stencil(h, [&](auto Sc) {
        constexpr int S = decltype(Sc)::value;
        switch (h->d) {
          case 1: launch_pc<1, S>(h, g, nb, rank, Dg.as<double>(), pc->L.as<double>(), part_a, part_s, tk, stt, piv_list, st); break;
          case 2: launch_pc<2, S>(h, g, nb, rank, Dg.as<double>(), pc->L.as<double>(), part_a, part_s, tk, stt, piv_list, st); break;
          default: launch_pc<3, S>(h, g, nb, rank, Dg.as<double>(), pc->L.as<double>(), part_a, part_s, tk, stt, piv_list, st); break;
        }
      });
    }
    if (cudaGetLastError() != cudaSuccess) { rc = set_error(DSKI_ERR_CUDA, "pivchol_build: launch failed"); break; }
    {
      StageScope sc(h, ST_PIVCHOL, st);
      k_inv_sqrt_noise<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(h->n, h->d, h->nv, h->ng,
                                                                      pc->dis.as<double>(),
                                                                      pc->ds.as<double>());
    }
    PcState hs{};
    std::vector<int> piv(rank);
    if (cudaMemcpyAsync(&hs, stt, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(piv.data(), piv_list, rank * sizeof(int), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = set_error(DSKI_ERR_CUDA, "pivchol_build: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    pc->rank = hs.steps;
    pc->piv.assign(piv.begin(), piv.begin() + hs.steps);
    pc->logdetM = (double)h->n * std::log(h->nv) + (double)h->n * h->d * std::log(h->ng);
    if (pc->rank > 0) {
      if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) { rc = DSKI_ERR_CUDA; break; }
      rc = qr_form(h, pc, flag, small, piv_list);
      if (rc) break;
      int hflag = 0;
      if (cudaMemcpy(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = set_error(DSKI_ERR_CUDA, "pivchol_build: flag read failed");
        break;
      }
      if (hflag) {
        rc = set_error(DSKI_ERR_BREAKDOWN, "pivchol_build: r x r Gram matrix not positive definite");
        break;
      }
    }
  } while (0);
  Dg.release();
  state.release();
  if (rc != DSKI_OK) {
    free_pc(pc);
    return rc;
  }
  *out = pc;
  if (rank_achieved) *rank_achieved = pc->rank;
  return DSKI_OK;
}

extern "C" int pivchol_export(pivchol_handle pc, double* L_dev, int* pivots_host) {
  clear_error();
  if (!pc) return set_error(DSKI_ERR_ARG, "pivchol_export: NULL preconditioner");
  dski_handle h = pc->h;
  if (pivots_host) {
    std::vector<int> perm(h->n);
    if (cudaMemcpyAsync(perm.data(), h->perm.ptr, h->n * sizeof(int), cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      return set_error(DSKI_ERR_CUDA, "pivchol_export: %s", cudaGetErrorString(cudaGetLastError()));
    for (int k = 0; k < pc->rank; ++k) {
      const int e = pc->piv[k];
      const int j = e / (h->d + 1), c = e % (h->d + 1);
      pivots_host[k] = c * h->n + perm[j];
    }
  }
  if (L_dev && pc->rank > 0) DSKI_TRY(permute_out(h, pc->L.ptr, L_dev, pc->rank, true, h->stream));
  if (cudaStreamSynchronize(h->stream) != cudaSuccess)
    return set_error(DSKI_ERR_CUDA, "pivchol_export: %s", cudaGetErrorString(cudaGetLastError()));
  return DSKI_OK;
}

extern "C" double pivchol_logdet(pivchol_handle pc) { return pc ? pc->logdetM : NAN; }

extern "C" void pivchol_destroy(pivchol_handle pc) {
  if (!pc) return;
  cudaStreamSynchronize(pc->h->stream);
  free_pc(pc);
}
