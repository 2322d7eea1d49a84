// Many independent D-SKI systems solved by PCG in one persistent launch
// (Sec. 2 conjugate gradients, Sec. 3.3 preconditioning, with the MVM
// K~ v = B K_UU B^T v + D v of Sec. 3.1 and B = [W; dW] of Eq. 4).
//
// One CTA solves one system from start to finish and then takes the next
// system from a device work queue: an atomic counter over a list ordered by
// estimated cost per iteration, largest first.  The system's grid vector
// (M doubles) and its Kronecker factors K_k (m_k x m_k doubles) stay in the
// CTA's shared memory for the whole solve; the point vectors, the stencil
// weights and the preconditioner's Q1 are read from global memory (L2).
// Every step is FP64 on the SIMT units: at these sizes (grids of a few
// thousand nodes, a few thousand points) a system is far too small to fill
// the tensor cores or the GPU, and many of them side by side fill the SMs.
//
// Per iteration, in one CTA (rows e = j (d + 1) + c of the point-sorted,
// point-interleaved layout):
//   A  p = z + beta p for every point's rows, then scatter G = B^T p
//      (sum-factorised stencil, shared-memory atomics; each thread takes a
//      contiguous run of points, so the lanes of a warp hit distant cells)
//   K  G = sf^2 (K_1 x ... x K_d) G, one mode at a time, in place: a warp
//      holds one fibre (lane i its entries i and i + 32), broadcasts entry j
//      by shuffle and accumulates row i of K_k
//   C  q = B G + D p (the gather, sum-factorised in reverse) and p^T q
//   U  x += alpha p, r -= alpha q, ||r||^2 and c = Q1^T D^-1/2 r
//   P  z = D^-1/2 (D^-1/2 r - Q1 c) and r^T z
// with one block reduction (fixed order) after C, U and P.  When the
// recursive residual meets rtol the true residual b - K~ x is formed with
// the same FP64 operator and the solve restarts from it if it misses
// (as dski_pcg_solve does).  The scatter's shared-memory atomics add in no
// fixed order, so results may differ between runs in their last bits.
//
// There is no grid-wide synchronisation and no spin-wait: CTAs share only
// the work-queue counter.  maxit bounds every solve.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "solve_internal.cuh"

namespace dski {
namespace {

constexpr int BT = 256;            // threads per CTA
constexpr int BW = BT / 32;        // warps per CTA
constexpr int RMAX = 32;           // largest preconditioner rank
constexpr int MMAX = 64;           // largest m_k (two fibre entries per lane)
constexpr int MAX_RESTARTS = 64;

// One system, as the kernel sees it (device pointers into its handle and
// preconditioner, and its slice of the launch's workspace).  Plain data: a
// CTA copies it to shared memory.
struct BInst {
  int n, d, N, S, M, rank;
  int m[DSKI_MAXD], mc[DSKI_MAXD];
  double nv, ng, sf2;
  const int* perm;     // sorted position -> original point
  const int* cell;     // flat cell id per sorted point
  const double* W;     // 2 S d stencil weights per sorted point
  const double* K[DSKI_MAXD];
  const double* Q1;    // N x rank, column-major (NULL: no preconditioner)
  const double* dis;   // D^-1/2 per internal row
  const double* b;     // user layout (block order)
  double* x;           // user layout: initial guess in, solution out
  double* ws;          // 6 N doubles: b, x, r, z, p, q (internal layout)
};

struct BOut {
  int iters;
  int status;
  int restarts;
  int pad;
  double relres;
  double seconds;
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Sum of NV per-thread values over the CTA, in a fixed order (warp
// butterflies, then the warps in order); the totals land in tot[0..NV).
// red holds BW x NV doubles.  All threads must call it.
template <int NV>
__device__ __forceinline__ void block_sums(double (&v)[NV], double* red, double* tot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double s = warp_sum(v[k]);
    if (lane == 0) red[w * NV + k] = s;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += BT) {
    double s = 0.0;
    for (int q = 0; q < BW; ++q) s += red[q * NV + k];
    tot[k] = s;
  }
  __syncthreads();
}

// First grid node of sorted point j's stencil (C-order flat index).
template <int D>
__device__ __forceinline__ int stencil_base(const BInst& I, int j) {
  int id = I.cell[j];
  if (D == 1) return id;
  if (D == 2) {
    const int c1 = id % I.mc[1], c0 = id / I.mc[1];
    return c0 * I.m[1] + c1;
  }
  const int c2 = id % I.mc[2];
  id /= I.mc[2];
  const int c1 = id % I.mc[1], c0 = id / I.mc[1];
  return (c0 * I.m[1] + c1) * I.m[2] + c2;
}

// Stage A: G += B^T v for one point (values v[0..D]): node (o_1..o_d) gets
// prod_k w_k v_0 + sum_c (dw_c prod_{k != c} w_k) v_c, sum-factorised one
// dimension at a time.
template <int D, int S>
__device__ __forceinline__ void scatter_point(const double* w, const double* v, double* G,
                                              int base, const int* m) {
  if (D == 1) {
#pragma unroll
    for (int a = 0; a < S; ++a) atomicAdd(G + base + a, fma(w[a], v[0], w[S + a] * v[1]));
  } else if (D == 2) {
    const double* w1 = w + 2 * S;
#pragma unroll
    for (int a = 0; a < S; ++a) {
      const double A = fma(w[a], v[0], w[S + a] * v[1]);
      const double B = w[a] * v[2];
#pragma unroll
      for (int b = 0; b < S; ++b)
        atomicAdd(G + base + a * m[1] + b, fma(w1[b], A, w1[S + b] * B));
    }
  } else {
    const double* w1 = w + 2 * S;
    const double* w2 = w + 4 * S;
    const int st0 = m[1] * m[2];
#pragma unroll 1
    for (int a = 0; a < S; ++a) {
      const double A = fma(w[a], v[0], w[S + a] * v[1]);
      const double B = w[a] * v[2];
      const double C = w[a] * v[3];
#pragma unroll
      for (int b = 0; b < S; ++b) {
        const double P = fma(w1[b], A, w1[S + b] * B);
        const double Q = w1[b] * C;
        double* g = G + base + a * st0 + b * m[2];
#pragma unroll
        for (int c = 0; c < S; ++c) atomicAdd(g + c, fma(w2[c], P, w2[S + c] * Q));
      }
    }
  }
}

// Stage C: out[0..D] = (B G) for one point: the value row and the d
// derivative rows, the transpose of scatter_point's factorisation.
template <int D, int S>
__device__ __forceinline__ void gather_point(const double* w, const double* G, int base,
                                             const int* m, double* out) {
  if (D == 1) {
    double o0 = 0, o1 = 0;
#pragma unroll
    for (int a = 0; a < S; ++a) {
      const double g = G[base + a];
      o0 = fma(w[a], g, o0);
      o1 = fma(w[S + a], g, o1);
    }
    out[0] = o0;
    out[1] = o1;
  } else if (D == 2) {
    const double* w1 = w + 2 * S;
    double o0 = 0, o1 = 0, o2 = 0;
#pragma unroll
    for (int a = 0; a < S; ++a) {
      const double* g = G + base + a * m[1];
      double t = 0, u = 0;
#pragma unroll
      for (int b = 0; b < S; ++b) {
        t = fma(w1[b], g[b], t);
        u = fma(w1[S + b], g[b], u);
      }
      o0 = fma(w[a], t, o0);
      o1 = fma(w[S + a], t, o1);
      o2 = fma(w[a], u, o2);
    }
    out[0] = o0;
    out[1] = o1;
    out[2] = o2;
  } else {
    const double* w1 = w + 2 * S;
    const double* w2 = w + 4 * S;
    const int st0 = m[1] * m[2];
    double o0 = 0, o1 = 0, o2 = 0, o3 = 0;
#pragma unroll 1
    for (int a = 0; a < S; ++a) {
      double A = 0, B = 0, C = 0;
#pragma unroll
      for (int b = 0; b < S; ++b) {
        const double* g = G + base + a * st0 + b * m[2];
        double t = 0, u = 0;
#pragma unroll
        for (int c = 0; c < S; ++c) {
          t = fma(w2[c], g[c], t);
          u = fma(w2[S + c], g[c], u);
        }
        A = fma(w1[b], t, A);
        B = fma(w1[S + b], t, B);
        C = fma(w1[b], u, C);
      }
      o0 = fma(w[a], A, o0);
      o1 = fma(w[S + a], A, o1);
      o2 = fma(w[a], B, o2);
      o3 = fma(w[a], C, o3);
    }
    out[0] = o0;
    out[1] = o1;
    out[2] = o2;
    out[3] = o3;
  }
}

// Stage K: G <- sf^2 (K_1 x ... x K_d) G in place.  For mode k a fibre is
// the m_k entries that differ only in coordinate k; one warp owns a fibre,
// lane i holds entries i and i + 32, and entry j reaches every lane by
// shuffle while lane i accumulates K_k[i][j] x_j (K_k is symmetric, so row
// j read across the lanes is contiguous).
template <int D>
__device__ __forceinline__ void kron_inplace(const BInst& I, double* G, const double* Ks) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double* K = Ks;
#pragma unroll 1
  for (int k = 0; k < D; ++k) {
    const int mk = I.m[k];
    int stride = 1;
    for (int q = k + 1; q < D; ++q) stride *= I.m[q];
    const int nfib = I.M / mk;
    const double scale = (k == D - 1) ? I.sf2 : 1.0;
    const bool ha = lane < mk, hb = lane + 32 < mk;
    const int j1 = mk < 32 ? mk : 32;
#pragma unroll 1
    for (int f = w; f < nfib; f += BW) {
      const int o = f / stride, u = f - o * stride;
      double* g = G + (size_t)o * mk * stride + u;
      const double xa = ha ? g[lane * stride] : 0.0;
      const double xb = hb ? g[(lane + 32) * stride] : 0.0;
      double ya = 0.0, yb = 0.0;
#pragma unroll 4
      for (int j = 0; j < j1; ++j) {
        const double xj = __shfl_sync(0xffffffffu, xa, j);
        const double* Kr = K + j * mk;
        if (ha) ya = fma(Kr[lane], xj, ya);
        if (hb) yb = fma(Kr[lane + 32], xj, yb);
      }
#pragma unroll 4
      for (int j = 32; j < mk; ++j) {
        const double xj = __shfl_sync(0xffffffffu, xb, j - 32);
        const double* Kr = K + j * mk;
        if (ha) ya = fma(Kr[lane], xj, ya);
        if (hb) yb = fma(Kr[lane + 32], xj, yb);
      }
      // each lane overwrites only the entries it read itself
      if (ha) g[lane * stride] = scale * ya;
      if (hb) g[(lane + 32) * stride] = scale * yb;
    }
    K += mk * mk;
    __syncthreads();
  }
}

// G = 0 (stage A accumulates into it).
__device__ __forceinline__ void grid_clear(double* G, int M) {
  for (int i = threadIdx.x; i < M; i += BT) G[i] = 0.0;
  __syncthreads();
}

// Stage A over the system's points: mode 0 scatters v as it is; mode 1
// first sets v = z (a restart), mode 2 v = z + beta v (the CG direction
// update), writing v back.  Thread t takes points [t c, (t + 1) c).
template <int D, int S>
__device__ __forceinline__ void stage_scatter(const BInst& I, double* G, double* v,
                                              const double* z, double beta, int mode) {
  constexpr int R1 = D + 1, NW = 2 * S * D;
  const int n = I.n;
  const int chunk = (n + BT - 1) / BT;
  const int j0 = threadIdx.x * chunk, j1 = min(n, j0 + chunk);
#pragma unroll 1
  for (int j = j0; j < j1; ++j) {
    double vv[R1];
#pragma unroll
    for (int c = 0; c < R1; ++c) {
      const int e = j * R1 + c;
      double val = v[e];
      if (mode == 1) val = z[e];
      else if (mode == 2) val = fma(beta, val, z[e]);
      if (mode) v[e] = val;
      vv[c] = val;
    }
    double w[NW];
    const double* wj = I.W + (size_t)j * NW;
#pragma unroll
    for (int k = 0; k < NW; ++k) w[k] = __ldg(wj + k);
    scatter_point<D, S>(w, vv, G, stencil_base<D>(I, j), I.m);
  }
  __syncthreads();
}

// Stage C over the system's points: q = B G + D v.  resid = false: out = q
// and the thread's part of v^T q is returned; resid = true: out = b - q
// (the true residual, v = x) and the thread's part of ||b - q||^2.
template <int D, int S>
__device__ __forceinline__ double stage_gather(const BInst& I, const double* G, const double* v,
                                               const double* b, double* out, bool resid) {
  constexpr int R1 = D + 1, NW = 2 * S * D;
  double acc = 0.0;
#pragma unroll 1
  for (int j = threadIdx.x; j < I.n; j += BT) {
    double w[NW];
    const double* wj = I.W + (size_t)j * NW;
#pragma unroll
    for (int k = 0; k < NW; ++k) w[k] = __ldg(wj + k);
    double o[R1];
    gather_point<D, S>(w, G, stencil_base<D>(I, j), I.m, o);
#pragma unroll
    for (int c = 0; c < R1; ++c) {
      const int e = j * R1 + c;
      const double ve = v[e];
      const double qe = fma(c == 0 ? I.nv : I.ng, ve, o[c]);
      if (resid) {
        const double re = b[e] - qe;
        out[e] = re;
        acc = fma(re, re, acc);
      } else {
        out[e] = qe;
        acc = fma(ve, qe, acc);
      }
    }
  }
  return acc;
}

// Stage U: with upd, x += alpha p and r -= alpha q; then ||r||^2 (tot[0])
// and, with a preconditioner, c = Q1^T D^-1/2 r (tot[1..rank]).
__device__ __forceinline__ void stage_update(const BInst& I, double* x, double* r, const double* p,
                                             const double* q, double alpha, bool upd, double* red,
                                             double* tot) {
  const int N = I.N;
  if (!I.Q1) {
    double acc[1] = {0.0};
    for (int e = threadIdx.x; e < N; e += BT) {
      double re = r[e];
      if (upd) {
        x[e] = fma(alpha, p[e], x[e]);
        re = fma(-alpha, q[e], re);
        r[e] = re;
      }
      acc[0] = fma(re, re, acc[0]);
    }
    block_sums<1>(acc, red, tot);
    return;
  }
  const int rank = I.rank;
  double acc[RMAX + 1];
#pragma unroll
  for (int k = 0; k <= RMAX; ++k) acc[k] = 0.0;
#pragma unroll 1
  for (int e = threadIdx.x; e < N; e += BT) {
    double re = r[e];
    if (upd) {
      x[e] = fma(alpha, p[e], x[e]);
      re = fma(-alpha, q[e], re);
      r[e] = re;
    }
    acc[0] = fma(re, re, acc[0]);
    const double y = __ldg(I.dis + e) * re;
    const double* qe = I.Q1 + e;
#pragma unroll
    for (int k = 0; k < RMAX; ++k)
      if (k < rank) acc[1 + k] = fma(__ldg(qe + (size_t)k * N), y, acc[1 + k]);
  }
  block_sums<RMAX + 1>(acc, red, tot);
}

// Stage P: z = D^-1/2 (D^-1/2 r - Q1 c) with c = tot[1..rank] from stage U;
// returns r^T z in every thread.
__device__ __forceinline__ double stage_precond(const BInst& I, const double* r, double* z,
                                                double* red, double* tot) {
  const int N = I.N, rank = I.rank;
  double acc[1] = {0.0};
#pragma unroll 1
  for (int e = threadIdx.x; e < N; e += BT) {
    const double de = __ldg(I.dis + e);
    const double re = r[e];
    double s = de * re;
    const double* qe = I.Q1 + e;
#pragma unroll
    for (int k = 0; k < RMAX; ++k)
      if (k < rank) s = fma(-__ldg(qe + (size_t)k * N), tot[1 + k], s);
    const double ze = de * s;
    z[e] = ze;
    acc[0] = fma(re, ze, acc[0]);
  }
  // every thread has read tot[1..rank] before block_sums writes tot[0]
  block_sums<1>(acc, red, tot);
  return tot[0];
}

// The whole PCG of one system in the calling CTA.  G: M doubles and Ks the
// factors (sum m_k^2 doubles) in shared memory; red / tot: reduction scratch.
template <int D, int S>
__device__ __noinline__ void solve_one(const BInst& I, double rtol, int maxit, double* G,
                                       double* Ks, double* red, double* tot, BOut* out) {
  constexpr int R1 = D + 1;
  const unsigned long long t0 = gtimer();
  const int N = I.N, n = I.n;
  double* bI = I.ws;
  double* x = bI + N;
  double* r = x + N;
  double* z = I.Q1 ? r + N : r;   // without a preconditioner z is r
  double* p = r + 2 * (size_t)N;
  double* q = r + 3 * (size_t)N;
  {
    int off = 0;
    for (int k = 0; k < D; ++k) {
      const int mm = I.m[k] * I.m[k];
      for (int i = threadIdx.x; i < mm; i += BT) Ks[off + i] = __ldg(I.K[k] + i);
      off += mm;
    }
  }
  // user (block) order -> internal rows e = j (d + 1) + c
  double acc[1] = {0.0};
  for (int e = threadIdx.x; e < N; e += BT) {
    const int j = e / R1, c = e - j * R1;
    const size_t u = (size_t)c * n + I.perm[j];
    const double be = I.b[u];
    bI[e] = be;
    x[e] = I.x[u];
    acc[0] = fma(be, be, acc[0]);
  }
  block_sums<1>(acc, red, tot);
  const double bn2 = tot[0];
  const double tgt = rtol * rtol * bn2;
  auto true_residual = [&]() -> double {   // r = b - K~ x, returns ||r||^2
    grid_clear(G, I.M);
    stage_scatter<D, S>(I, G, x, nullptr, 0.0, 0);
    kron_inplace<D>(I, G, Ks);
    double a[1] = {stage_gather<D, S>(I, G, x, bI, r, true)};
    block_sums<1>(a, red, tot);
    return tot[0];
  };
  int status = DSKI_OK, it = 0, restarts = 0;
  double rn2 = 0.0;
  if (bn2 == 0.0) {
    for (int e = threadIdx.x; e < N; e += BT) x[e] = 0.0;
    __syncthreads();
  } else {
    rn2 = true_residual();
    for (;;) {
      if (!isfinite(rn2)) { status = DSKI_ERR_BREAKDOWN; break; }
      if (rn2 <= tgt) break;
      if (it >= maxit || restarts > MAX_RESTARTS) { status = DSKI_ERR_NOT_CONVERGED; break; }
      // (re)start from the true residual: z = M^-1 r, p = z
      double rz;
      if (I.Q1) {
        stage_update(I, x, r, p, q, 0.0, false, red, tot);
        rz = stage_precond(I, r, z, red, tot);
      } else {
        rz = rn2;
      }
      double beta = 0.0;
      int mode = 1;
      bool broke = false;
      for (;;) {
        grid_clear(G, I.M);
        stage_scatter<D, S>(I, G, p, z, beta, mode);
        kron_inplace<D>(I, G, Ks);
        double a[1] = {stage_gather<D, S>(I, G, p, nullptr, q, false)};
        block_sums<1>(a, red, tot);
        const double pq = tot[0];
        if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rz)) { broke = true; break; }
        const double alpha = rz / pq;
        stage_update(I, x, r, p, q, alpha, true, red, tot);
        rn2 = tot[0];
        ++it;
        if (rn2 <= tgt || it >= maxit || !isfinite(rn2)) break;
        const double rz1 = I.Q1 ? stage_precond(I, r, z, red, tot) : rn2;
        beta = rz1 / rz;
        rz = rz1;
        mode = 2;
      }
      rn2 = true_residual();
      ++restarts;
      if (broke) { status = DSKI_ERR_BREAKDOWN; break; }
    }
  }
  // internal rows -> user order
  for (int e = threadIdx.x; e < N; e += BT) {
    const int j = e / R1, c = e - j * R1;
    I.x[(size_t)c * n + I.perm[j]] = x[e];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    out->iters = it;
    out->status = status;
    out->restarts = restarts;
    out->relres = bn2 > 0.0 ? sqrt(rn2 / bn2) : 0.0;
    out->seconds = (double)(gtimer() - t0) * 1e-9;
  }
}

// The persistent launch: each CTA takes systems off the queue (order[t] for
// ticket t) until the tickets run out.
__global__ void __launch_bounds__(BT) k_batch_pcg(const BInst* __restrict__ insts,
                                                  const int* __restrict__ order, int count,
                                                  unsigned* queue, BOut* outs, double rtol,
                                                  int maxit) {
  extern __shared__ __align__(16) double smem[];
  __shared__ double red[BW * (RMAX + 1)];
  __shared__ double tot[RMAX + 1];
  __shared__ BInst sI;
  __shared__ int s_task;
  for (;;) {
    if (threadIdx.x == 0) {
      const int t = (int)atomicAdd(queue, 1u);
      s_task = t < count ? order[t] : -1;
      if (s_task >= 0) sI = insts[s_task];
    }
    __syncthreads();
    const int i = s_task;
    if (i < 0) return;
    double* G = smem;
    double* Ks = smem + sI.M;
    BOut* o = outs + i;
    switch (sI.d * 10 + sI.S) {
      case 14: solve_one<1, 4>(sI, rtol, maxit, G, Ks, red, tot, o); break;
      case 24: solve_one<2, 4>(sI, rtol, maxit, G, Ks, red, tot, o); break;
      case 34: solve_one<3, 4>(sI, rtol, maxit, G, Ks, red, tot, o); break;
      case 16: solve_one<1, 6>(sI, rtol, maxit, G, Ks, red, tot, o); break;
      case 26: solve_one<2, 6>(sI, rtol, maxit, G, Ks, red, tot, o); break;
      default: solve_one<3, 6>(sI, rtol, maxit, G, Ks, red, tot, o); break;
    }
    // every thread is done with sI and s_task before thread 0 refills them
    __syncthreads();
  }
}

}  // namespace
}  // namespace dski

using namespace dski;

extern "C" int dski_pcg_solve_batch(int count, const dski_handle* hs, const pivchol_handle* pcs,
                                    const double* const* b, double* const* x, double rtol,
                                    int maxit, int* iters, double* relres, int* status,
                                    double* seconds) {
  clear_error();
  if (count < 1 || !hs || !b || !x)
    return set_error(DSKI_ERR_ARG, "dski_pcg_solve_batch: NULL argument or count < 1");
  if (!(rtol > 0.0) || maxit < 1)
    return set_error(DSKI_ERR_ARG, "dski_pcg_solve_batch: need rtol > 0, maxit >= 1");
  int dev = 0, optin = 0;
  DSKI_CUDA(cudaGetDevice(&dev));
  DSKI_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa{};
  DSKI_CUDA(cudaFuncGetAttributes(&fa, k_batch_pcg));
  const size_t smem_cap = (size_t)optin - fa.sharedSizeBytes;
  std::vector<BInst> bi(count);
  std::vector<double> cost(count);
  std::vector<size_t> off(count);
  size_t wsd = 0, smem = 0;
  for (int i = 0; i < count; ++i) {
    dski_handle h = hs[i];
    pivchol_handle pc = pcs ? pcs[i] : nullptr;
    if (!h || !b[i] || !x[i])
      return set_error(DSKI_ERR_ARG, "dski_pcg_solve_batch: system %d: NULL handle or vector", i);
    if (!f64_vectors(h))
      return set_error(DSKI_ERR_ARG,
                       "dski_pcg_solve_batch: system %d: FP64 vectors needed (FP64 or FP64_TC handle)", i);
    if (h->d < 1 || h->d > DSKI_MAXD || (h->sw != 4 && h->sw != 6))
      return set_error(DSKI_ERR_ARG, "dski_pcg_solve_batch: system %d: unsupported d or stencil", i);
    if (pc && pc->h != h)
      return set_error(DSKI_ERR_ARG, "dski_pcg_solve_batch: system %d: preconditioner of another handle", i);
    if (pc && pc->rank > RMAX)
      return set_error(DSKI_ERR_ARG, "dski_pcg_solve_batch: system %d: preconditioner rank %d above %d",
                       i, pc->rank, RMAX);
    if (pc && (!pc->Q1.ptr || !pc->dis.ptr))
      return set_error(DSKI_ERR_ARG, "dski_pcg_solve_batch: system %d: preconditioner without its QR form", i);
    size_t kk = 0, msum = 0;
    for (int k = 0; k < h->d; ++k) {
      if (h->m[k] > MMAX)
        return set_error(DSKI_ERR_ARG, "dski_pcg_solve_batch: system %d: m_%d = %d above %d", i, k,
                         h->m[k], MMAX);
      kk += (size_t)h->m[k] * h->m[k];
      msum += h->m[k];
    }
    const size_t sm = ((size_t)h->M + kk) * 8;
    if (sm > smem_cap)
      return set_error(DSKI_ERR_ARG,
                       "dski_pcg_solve_batch: system %d: grid and factors need %zu bytes of shared "
                       "memory (at most %zu)", i, sm, smem_cap);
    BInst& I = bi[i];
    I = BInst{};
    I.n = h->n;
    I.d = h->d;
    I.N = h->N;
    I.S = h->sw;
    I.M = h->M;
    I.rank = pc ? pc->rank : 0;
    for (int k = 0; k < DSKI_MAXD; ++k) {
      I.m[k] = h->m[k];
      I.mc[k] = h->mc[k];
      I.K[k] = k < h->d ? h->K64[k].as<double>() : nullptr;
    }
    I.nv = h->nv;
    I.ng = h->ng;
    I.sf2 = h->sf * h->sf;
    I.perm = h->perm.as<int>();
    I.cell = h->cell.as<int>();
    I.W = h->W64.as<double>();
    I.Q1 = pc ? pc->Q1.as<double>() : nullptr;
    I.dis = pc ? pc->dis.as<double>() : nullptr;
    I.b = b[i];
    I.x = x[i];
    off[i] = wsd;
    wsd += 6 * (size_t)h->N;
    smem = std::max(smem, sm);
    // FP64 operations of one iteration: the stencil passes, the mode
    // products, the preconditioner and the vector updates
    double sten = 1.0;
    for (int k = 0; k < h->d; ++k) sten *= h->sw;
    cost[i] = 4.0 * (h->d + 1) * sten * h->n + (double)h->M * (double)msum +
              (double)h->N * (2.0 * I.rank + 12.0);
  }
  // largest estimated cost first (longest-processing-time order)
  std::vector<int> ord(count);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  // the handles' earlier work (geometry, factors, preconditioners) is done
  for (int i = 0; i < count; ++i) DSKI_CUDA(cudaStreamSynchronize(hs[i]->stream));
  cudaStream_t st = hs[0]->stream;
  auto up16 = [](size_t v) { return (v + 15) & ~(size_t)15; };
  const size_t o_inst = up16(wsd * 8);
  const size_t o_ord = up16(o_inst + sizeof(BInst) * count);
  const size_t o_out = up16(o_ord + sizeof(int) * count);
  const size_t o_q = up16(o_out + sizeof(BOut) * count);
  const size_t total = o_q + 16;
  char* mem = nullptr;
  if (cudaMalloc(&mem, total) != cudaSuccess)
    return set_error(DSKI_ERR_ALLOC, "dski_pcg_solve_batch: %zu bytes of workspace", total);
  struct Free {
    char* p;
    ~Free() { cudaFree(p); }
  } fr{mem};
  for (int i = 0; i < count; ++i) bi[i].ws = reinterpret_cast<double*>(mem) + off[i];
  DSKI_CUDA(cudaMemcpyAsync(mem + o_inst, bi.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice, st));
  DSKI_CUDA(cudaMemcpyAsync(mem + o_ord, ord.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st));
  DSKI_CUDA(cudaMemsetAsync(mem + o_q, 0, 16, st));
  static std::atomic<unsigned long long> attr_set{0};
  if (first_on_device(&attr_set))
    DSKI_CUDA(cudaFuncSetAttribute(k_batch_pcg, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem_cap));
  int bps = 0;
  DSKI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_batch_pcg, BT, smem));
  const int grid = std::min(count, std::max(1, bps) * std::max(1, hs[0]->sm_count));
  k_batch_pcg<<<grid, BT, smem, st>>>(reinterpret_cast<const BInst*>(mem + o_inst),
                                      reinterpret_cast<const int*>(mem + o_ord), count,
                                      reinterpret_cast<unsigned*>(mem + o_q),
                                      reinterpret_cast<BOut*>(mem + o_out), rtol, maxit);
  DSKI_LAUNCHED();
  count_launches(1);
  std::vector<BOut> ho(count);
  DSKI_CUDA(cudaMemcpyAsync(ho.data(), mem + o_out, sizeof(BOut) * count, cudaMemcpyDeviceToHost, st));
  DSKI_CUDA(cudaStreamSynchronize(st));
  int bad = 0, first = -1;
  for (int i = 0; i < count; ++i) {
    if (iters) iters[i] = ho[i].iters;
    if (relres) relres[i] = ho[i].relres;
    if (status) status[i] = ho[i].status;
    if (seconds) seconds[i] = ho[i].seconds;
    if (ho[i].status != DSKI_OK) {
      ++bad;
      if (first < 0) first = i;
    }
  }
  if (first >= 0) {
    const int rc = ho[first].status;
    return set_error(rc, "dski_pcg_solve_batch: %d of %d systems failed (first: system %d, %s, "
                     "relres %.3g after %d iterations)", bad, count, first,
                     rc == DSKI_ERR_BREAKDOWN ? "breakdown" : "not converged", ho[first].relres,
                     ho[first].iters);
  }
  return DSKI_OK;
}
