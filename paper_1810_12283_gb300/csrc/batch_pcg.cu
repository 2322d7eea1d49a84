// Many independent D-SKI systems solved by PCG in one persistent launch
// (Sec. 2 conjugate gradients, Sec. 3.3 preconditioning, with the MVM
// K~ v = B K_UU B^T v + D v of Sec. 3.1 and B = [W; dW] of Eq. 4).
//
// The launch is made of thread-block clusters of C CTAs (C = 1, 2, 4 or 8).
// A cluster solves one system from start to finish and then takes the next
// from a device work queue: an atomic counter over a list ordered by
// estimated cost per iteration, largest first.  Every CTA of the cluster
// keeps the system's grid vector (M doubles) and Kronecker factors K_k
// (m_k x m_k doubles) in its shared memory for the whole solve; the point
// vectors, stencil weights and the preconditioner's Q1 stay in global
// memory (L2).  Every step is FP64 on the SIMT units: a system (a grid of a
// few thousand nodes, a few thousand points) is far too small for the
// tensor cores or the whole GPU, and many systems side by side fill the SMs.
//
// CTA c of the cluster owns a contiguous run of the (cell-sorted) points
// and their rows e = j (d + 1) + c', a run of grid "columns" (the flat index
// over dimensions 2..d) and a slab of grid rows (dimension 1).  Per
// iteration:
//   A  p = z + beta p on its rows; scatter its points into its own copy of
//      the grid (sum-factorised stencil, shared-memory atomics)
//   -- cluster barrier
//   R  its columns summed over the C copies (distributed shared memory, in
//      rank order), then mode 1 of the Kronecker product on those columns
//   -- cluster barrier
//   T  its slab's rows fetched from the columns' owners, then modes 2..d on
//      the slab (in place: a warp holds a fibre, lane i entries i and i+32,
//      entry j reaches the lanes by shuffle; sf^2 with the last mode)
//   -- cluster barrier
//   G  the other slabs fetched (every CTA now holds sf^2 (x_k K_k) B^T p);
//      q = B G + D p for its points and its part of p^T q
//   U  x += alpha p, r -= alpha q, ||r||^2 and c = Q1^T D^-1/2 r on its rows
//   P  z = D^-1/2 (D^-1/2 r - Q1 c) and r^T z on its rows
// Each dot product is a block reduction in a fixed order, then a cluster
// barrier and a sum of the C CTAs' totals in rank order, so every CTA holds
// the same scalars.  When the recursive residual meets rtol the true
// residual b - K~ x is formed with the same FP64 operator and the solve
// restarts from it if it misses (as dski_pcg_solve does).  The scatter's
// shared-memory atomics add in no fixed order, so results may differ
// between runs in their last bits.
//
// The only synchronisation is the hardware cluster barrier and
// __syncthreads: there is no spin-wait, and CTAs of different clusters share
// only the work-queue counter.  maxit bounds every solve.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include <cooperative_groups.h>

#include "solve_internal.cuh"

namespace dski {
namespace {

constexpr int BT = 256;            // threads per CTA
constexpr int BW = BT / 32;        // warps per CTA
constexpr int RMAX = 32;           // largest preconditioner rank
constexpr int MMAX = 64;           // largest m_k (two fibre entries per lane)
constexpr int MAX_RESTARTS = 64;
constexpr int kBatchDefaultCluster = 4;   // CTAs per system when the caller passes 0

namespace cg = cooperative_groups;

// One system, as the kernel sees it (device pointers into its handle and
// preconditioner, and its slice of the launch's workspace).  Plain data:
// each CTA copies it to shared memory.
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


__device__ __forceinline__ int split(int total, int C, int c) {
  return (int)(((long long)total * c) / C);
}

// The share of CTA c (of C) in a system: points [j0, j1) and their rows
// [e0, e1); grid columns [k0, k1) of the Mc = M / m_1 columns; the slab of
// dimension-1 rows [r0, r1).
struct Part {
  int c, C;
  int j0, j1, e0, e1;
  int Mc, k0, k1, r0, r1;
};

// Sum of NV per-thread values over the cluster: a block reduction into
// this CTA's buffer part[0..NV), a cluster barrier, then the C buffers added
// in rank order into tot (the same totals in every CTA).  Consecutive calls
// must alternate between two buffers: a buffer is rewritten only after the
// next call's barrier, which every CTA reaches after its reads of it.
template <int NV>
__device__ __forceinline__ void cluster_sums(double (&v)[NV], double* red, double* part,
                                             double* tot, cg::cluster_group& cl, int C) {
  block_sums<NV>(v, red, part);
  cl.sync();
  for (int k = threadIdx.x; k < NV; k += BT) {
    double s = 0.0;
    for (int q = 0; q < C; ++q) s += *cl.map_shared_rank(part + k, q);
    tot[k] = s;
  }
  __syncthreads();
}

// In-place mode product on the fibres (o, u) of G, o in [o0, o0 + no),
// u in [u0, u0 + nu): fibre (o, u) holds the mk entries
// G[(o mk + i) stride + u], replaced by scale sum_j K[i][j] x_j.  A warp owns
// a fibre, lane i holds entries i and i + 32, and entry j reaches every lane
// by shuffle while lane i accumulates K[j][i] x_j (K is symmetric, so row j
// read across the lanes is contiguous).
__device__ __forceinline__ void fibres(double* G, const double* K, int mk, int stride, int o0,
                                       int no, int u0, int nu, double scale) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool ha = lane < mk, hb = lane + 32 < mk;
  const int j1 = mk < 32 ? mk : 32;
  const int nf = no * nu;
#pragma unroll 1
  for (int f = w; f < nf; f += BW) {
    const int oi = f / nu;
    double* g = G + ((size_t)(o0 + oi) * mk) * stride + (u0 + f - oi * nu);
    const double xa = ha ? g[(size_t)lane * stride] : 0.0;
    const double xb = hb ? g[(size_t)(lane + 32) * stride] : 0.0;
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
    if (ha) g[(size_t)lane * stride] = scale * ya;
    if (hb) g[(size_t)(lane + 32) * stride] = scale * yb;
  }
}

// G = 0 (stage A accumulates into it).
__device__ __forceinline__ void grid_clear(double* G, int M) {
  for (int i = threadIdx.x; i < M; i += BT) G[i] = 0.0;
  __syncthreads();
}

// Stage A over this CTA's points: mode 0 scatters v as it is; mode 1 first
// sets v = z (a restart), mode 2 v = z + beta v (the CG direction update),
// writing v back.  Each thread takes a contiguous run of the points, so the
// lanes of a warp work on distant cells.
template <int D, int S>
__device__ __forceinline__ void stage_scatter(const BInst& I, const Part& P, double* G, double* v,
                                              const double* z, double beta, int mode) {
  constexpr int R1 = D + 1, NW = 2 * S * D;
  const int np = P.j1 - P.j0;
  const int chunk = (np + BT - 1) / BT;
  const int j0 = P.j0 + threadIdx.x * chunk, j1 = min(P.j1, j0 + chunk);
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

// G <- sf^2 (K_1 x ... x K_d) B^T v over the cluster (stages A, R, T and the
// fetch of the other slabs); afterwards every CTA holds the whole product.
template <int D, int S>
__device__ __forceinline__ void cluster_kernel_product(const BInst& I, const Part& P, double* G,
                                                       const double* Ks, double* v,
                                                       const double* z, double beta, int mode,
                                                       cg::cluster_group& cl) {
  const int Mc = P.Mc, m0 = I.m[0], C = P.C;
  grid_clear(G, I.M);
  stage_scatter<D, S>(I, P, G, v, z, beta, mode);
  cl.sync();
  // R: this CTA's columns summed over the C copies in rank order, then the
  // first mode on them (fibres along dimension 1: stride Mc)
  {
    const int nk = P.k1 - P.k0, tot = m0 * nk;
    for (int idx = threadIdx.x; idx < tot; idx += BT) {
      const int i0 = idx / nk;
      double* a = G + (size_t)i0 * Mc + P.k0 + (idx - i0 * nk);
      double s = 0.0;
      for (int q = 0; q < C; ++q) s += *cl.map_shared_rank(a, q);
      *a = s;
    }
    __syncthreads();
    fibres(G, Ks, m0, Mc, 0, 1, P.k0, nk, D == 1 ? I.sf2 : 1.0);
    __syncthreads();
  }
  cl.sync();
  // T: this CTA's slab rows from the columns' owners, then modes 2..d on
  // the slab
  {
    const int nr = P.r1 - P.r0;
    for (int q = 0; q < C; ++q) {
      if (q == P.c) continue;
      const int q0 = split(Mc, C, q), nk = split(Mc, C, q + 1) - q0, tot = nr * nk;
      for (int idx = threadIdx.x; idx < tot; idx += BT) {
        const int i = idx / nk;
        double* a = G + (size_t)(P.r0 + i) * Mc + q0 + (idx - i * nk);
        *a = *cl.map_shared_rank(a, q);
      }
    }
    __syncthreads();
    const double* K = Ks + m0 * m0;
    int outer = 1;   // prod of m_k over the dimensions between the first and mode k
    for (int k = 1; k < D; ++k) {
      const int mk = I.m[k];
      int stride = 1;
      for (int q = k + 1; q < D; ++q) stride *= I.m[q];
      fibres(G, K, mk, stride, P.r0 * outer, nr * outer, 0, stride, k == D - 1 ? I.sf2 : 1.0);
      __syncthreads();
      K += mk * mk;
      outer *= mk;
    }
  }
  cl.sync();
  // the other CTAs' slabs
  for (int q = 0; q < C; ++q) {
    if (q == P.c) continue;
    const size_t a0 = (size_t)split(m0, C, q) * Mc, a1 = (size_t)split(m0, C, q + 1) * Mc;
    for (size_t a = a0 + threadIdx.x; a < a1; a += BT) G[a] = *cl.map_shared_rank(G + a, q);
  }
  __syncthreads();
}

// Stage C over this CTA's points: q = B G + D v.  resid = false: out = q
// and the thread's part of v^T q is returned; resid = true: out = b - q
// (the true residual, v = x) and the thread's part of ||b - q||^2.
template <int D, int S>
__device__ __forceinline__ double stage_gather(const BInst& I, const Part& P, const double* G,
                                               const double* v, const double* b, double* out,
                                               bool resid) {
  constexpr int R1 = D + 1, NW = 2 * S * D;
  double acc = 0.0;
#pragma unroll 1
  for (int j = P.j0 + threadIdx.x; j < P.j1; j += BT) {
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

// Stage U on this CTA's rows: with upd, x += alpha p and r -= alpha q; then
// the cluster's ||r||^2 (tot[0]) and, with a preconditioner,
// c = Q1^T D^-1/2 r (tot[1..rank]).
__device__ __forceinline__ void stage_update(const BInst& I, const Part& P, double* x, double* r,
                                             const double* p, const double* q, double alpha,
                                             bool upd, double* red, double* part, double* tot,
                                             cg::cluster_group& cl) {
  if (!I.Q1) {
    double acc[1] = {0.0};
    for (int e = P.e0 + threadIdx.x; e < P.e1; e += BT) {
      double re = r[e];
      if (upd) {
        x[e] = fma(alpha, p[e], x[e]);
        re = fma(-alpha, q[e], re);
        r[e] = re;
      }
      acc[0] = fma(re, re, acc[0]);
    }
    cluster_sums<1>(acc, red, part, tot, cl, P.C);
    return;
  }
  const int N = I.N, rank = I.rank;
  double acc[RMAX + 1];
#pragma unroll
  for (int k = 0; k <= RMAX; ++k) acc[k] = 0.0;
#pragma unroll 1
  for (int e = P.e0 + threadIdx.x; e < P.e1; e += BT) {
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
  cluster_sums<RMAX + 1>(acc, red, part, tot, cl, P.C);
}

// Stage P on this CTA's rows: z = D^-1/2 (D^-1/2 r - Q1 c) with
// c = tot[1..rank] from stage U; returns the cluster's r^T z.
__device__ __forceinline__ double stage_precond(const BInst& I, const Part& P, const double* r,
                                                double* z, double* red, double* part, double* tot,
                                                cg::cluster_group& cl) {
  const int N = I.N, rank = I.rank;
  double acc[1] = {0.0};
#pragma unroll 1
  for (int e = P.e0 + threadIdx.x; e < P.e1; e += BT) {
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
  // every thread has read tot[1..rank] before cluster_sums writes tot[0]
  cluster_sums<1>(acc, red, part, tot, cl, P.C);
  return tot[0];
}

// The whole PCG of one system in the calling cluster.  G: M doubles and Ks
// the factors (sum m_k^2 doubles) in shared memory; red, tot and the two
// partial-sum buffers pbuf: reduction scratch.
template <int D, int S>
__device__ __noinline__ void solve_one(const BInst& I, double rtol, int maxit, double* G,
                                       double* Ks, double* red, double* tot, double* pbuf,
                                       BOut* out) {
  constexpr int R1 = D + 1;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned long long t0 = gtimer();
  Part P;
  P.c = (int)cl.block_rank();
  P.C = (int)cl.num_blocks();
  P.j0 = split(I.n, P.C, P.c);
  P.j1 = split(I.n, P.C, P.c + 1);
  P.e0 = P.j0 * R1;
  P.e1 = P.j1 * R1;
  P.Mc = I.M / I.m[0];
  P.k0 = split(P.Mc, P.C, P.c);
  P.k1 = split(P.Mc, P.C, P.c + 1);
  P.r0 = split(I.m[0], P.C, P.c);
  P.r1 = split(I.m[0], P.C, P.c + 1);
  int rb = 0;   // the partial-sum buffer of the next cluster reduction
  auto part = [&]() { return pbuf + (rb++ & 1) * (RMAX + 1); };
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
  // user (block) order -> internal rows e = j (d + 1) + c, this CTA's rows
  double acc[1] = {0.0};
  for (int e = P.e0 + threadIdx.x; e < P.e1; e += BT) {
    const int j = e / R1, c = e - j * R1;
    const size_t u = (size_t)c * n + I.perm[j];
    const double be = I.b[u];
    bI[e] = be;
    x[e] = I.x[u];
    acc[0] = fma(be, be, acc[0]);
  }
  cluster_sums<1>(acc, red, part(), tot, cl, P.C);
  const double bn2 = tot[0];
  const double tgt = rtol * rtol * bn2;
  auto true_residual = [&]() -> double {   // r = b - K~ x, returns ||r||^2
    cluster_kernel_product<D, S>(I, P, G, Ks, x, nullptr, 0.0, 0, cl);
    double a[1] = {stage_gather<D, S>(I, P, G, x, bI, r, true)};
    cluster_sums<1>(a, red, part(), tot, cl, P.C);
    return tot[0];
  };
  int status = DSKI_OK, it = 0, restarts = 0;
  double rn2 = 0.0;
  if (bn2 == 0.0) {
    for (int e = P.e0 + threadIdx.x; e < P.e1; e += BT) x[e] = 0.0;
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
        stage_update(I, P, x, r, p, q, 0.0, false, red, part(), tot, cl);
        rz = stage_precond(I, P, r, z, red, part(), tot, cl);
      } else {
        rz = rn2;
      }
      double beta = 0.0;
      int mode = 1;
      bool broke = false;
      for (;;) {
        cluster_kernel_product<D, S>(I, P, G, Ks, p, z, beta, mode, cl);
        double a[1] = {stage_gather<D, S>(I, P, G, p, nullptr, q, false)};
        cluster_sums<1>(a, red, part(), tot, cl, P.C);
        const double pq = tot[0];
        if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rz)) { broke = true; break; }
        const double alpha = rz / pq;
        stage_update(I, P, x, r, p, q, alpha, true, red, part(), tot, cl);
        rn2 = tot[0];
        ++it;
        if (rn2 <= tgt || it >= maxit || !isfinite(rn2)) break;
        const double rz1 = I.Q1 ? stage_precond(I, P, r, z, red, part(), tot, cl) : rn2;
        beta = rz1 / rz;
        rz = rz1;
        mode = 2;
      }
      rn2 = true_residual();
      ++restarts;
      if (broke) { status = DSKI_ERR_BREAKDOWN; break; }
    }
  }
  // this CTA's internal rows -> user order
  for (int e = P.e0 + threadIdx.x; e < P.e1; e += BT) {
    const int j = e / R1, c = e - j * R1;
    I.x[(size_t)c * n + I.perm[j]] = x[e];
  }
  __syncthreads();
  if (P.c == 0 && threadIdx.x == 0) {
    out->iters = it;
    out->status = status;
    out->restarts = restarts;
    out->relres = bn2 > 0.0 ? sqrt(rn2 / bn2) : 0.0;
    out->seconds = (double)(gtimer() - t0) * 1e-9;
  }
}

// The persistent launch: each cluster takes systems off the queue (order[t]
// for ticket t, drawn by the cluster's first CTA) until the tickets run out.
__global__ void __launch_bounds__(BT) k_batch_pcg(const BInst* __restrict__ insts,
                                                  const int* __restrict__ order, int count,
                                                  unsigned* queue, BOut* outs, double rtol,
                                                  int maxit) {
  extern __shared__ __align__(16) double smem[];
  __shared__ double red[BW * (RMAX + 1)];
  __shared__ double tot[RMAX + 1];
  __shared__ double pbuf[2 * (RMAX + 1)];
  __shared__ BInst sI;
  __shared__ int s_ticket, s_task;
  cg::cluster_group cl = cg::this_cluster();
  for (;;) {
    if (cl.block_rank() == 0 && threadIdx.x == 0) {
      const int t = (int)atomicAdd(queue, 1u);
      s_ticket = t < count ? order[t] : -1;
    }
    cl.sync();
    if (threadIdx.x == 0) {
      s_task = *cl.map_shared_rank(&s_ticket, 0);
      if (s_task >= 0) sI = insts[s_task];
    }
    // every CTA has read the first CTA's ticket before it can draw the next
    cl.sync();
    const int i = s_task;
    if (i < 0) return;
    double* G = smem;
    double* Ks = smem + sI.M;
    BOut* o = outs + i;
    switch (sI.d * 10 + sI.S) {
      case 14: solve_one<1, 4>(sI, rtol, maxit, G, Ks, red, tot, pbuf, o); break;
      case 24: solve_one<2, 4>(sI, rtol, maxit, G, Ks, red, tot, pbuf, o); break;
      case 34: solve_one<3, 4>(sI, rtol, maxit, G, Ks, red, tot, pbuf, o); break;
      case 16: solve_one<1, 6>(sI, rtol, maxit, G, Ks, red, tot, pbuf, o); break;
      case 26: solve_one<2, 6>(sI, rtol, maxit, G, Ks, red, tot, pbuf, o); break;
      default: solve_one<3, 6>(sI, rtol, maxit, G, Ks, red, tot, pbuf, o); break;
    }
    // no CTA still reads another's shared memory when the next system starts
    cl.sync();
  }
}

}  // namespace
}  // namespace dski

using namespace dski;

extern "C" int dski_pcg_solve_batch(int count, const dski_handle* hs, const pivchol_handle* pcs,
                                    const double* const* b, double* const* x, double rtol,
                                    int maxit, int cluster, int* iters, double* relres,
                                    int* status, double* seconds) {
  clear_error();
  if (count < 1 || !hs || !b || !x)
    return set_error(DSKI_ERR_ARG, "dski_pcg_solve_batch: NULL argument or count < 1");
  if (!(rtol > 0.0) || maxit < 1)
    return set_error(DSKI_ERR_ARG, "dski_pcg_solve_batch: need rtol > 0, maxit >= 1");
  if (cluster != 0 && cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8)
    return set_error(DSKI_ERR_ARG, "dski_pcg_solve_batch: cluster must be 0, 1, 2, 4 or 8");
  const int C = cluster ? cluster : kBatchDefaultCluster;
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
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg{};
  cfg.blockDim = dim3(BT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(C * std::max(1, hs[0]->sm_count / C));
  int ncl = 0;
  DSKI_CUDA(cudaOccupancyMaxActiveClusters(&ncl, k_batch_pcg, &cfg));
  if (ncl < 1)
    return set_error(DSKI_ERR_ARG, "dski_pcg_solve_batch: no cluster of %d CTAs with %zu bytes of "
                     "shared memory each fits on this GPU", C, smem);
  // one cluster per system at most, all resident at once
  cfg.gridDim = dim3(C * std::min(count, ncl));
  const BInst* a_inst = reinterpret_cast<const BInst*>(mem + o_inst);
  const int* a_ord = reinterpret_cast<const int*>(mem + o_ord);
  unsigned* a_q = reinterpret_cast<unsigned*>(mem + o_q);
  BOut* a_out = reinterpret_cast<BOut*>(mem + o_out);
  DSKI_CUDA(cudaLaunchKernelEx(&cfg, k_batch_pcg, a_inst, a_ord, count, a_q, a_out, rtol, maxit));
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
