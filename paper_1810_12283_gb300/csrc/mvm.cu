// The D-SKI MVM of Sec. 3.1:
//   K~ v = B (K_UU (B^T v)) + noise .* v,   B = [W; dW_1; ...; dW_d],
// in three stages on the sorted, point-interleaved internal layout:
//   scatter  g = B^T v   (grid-node-owned pull over the S^d neighbouring
//                         cells: deterministic, no atomics)
//   kron     h = s_f^2 (K_1 (x) ... (x) K_d) g  (d mode products)
//   gather   out = B h + noise .* v   (point-owned, sum-factorised stencil)
// The mode products here are the SIMT path (FP64 DFMA, or FP32 FFMA);
// the tensor-core (3x)TF32 path lives in kron_tc.cu.
#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>

#include "dski_internal.cuh"
#include "interp.cuh"
#include "solve_internal.cuh"

namespace dski {

struct MvmGeo {
  int d;
  int m[DSKI_MAXD];
  int mc[DSKI_MAXD];
  double invh[DSKI_MAXD];
};

template <class T>
const T* wt_table(dski_handle h);
template <>
const double* wt_table<double>(dski_handle h) { return h->W64.as<double>(); }
template <>
const float* wt_table<float>(dski_handle h) { return h->W32.as<float>(); }

static MvmGeo make_geo(dski_handle h) {
  MvmGeo g{};
  g.d = h->d;
  for (int k = 0; k < DSKI_MAXD; ++k) {
    g.m[k] = k < h->d ? h->m[k] : 1;
    g.mc[k] = k < h->d ? h->mc[k] : 1;
    g.invh[k] = k < h->d ? 1.0 / h->h[k] : 1.0;
  }
  return g;
}

namespace {

template <class T>
struct T2v {
  T x, y;
};
// two consecutive values (8-byte aligned for float: one 64-bit load)
__device__ __forceinline__ T2v<float> ld2(const float* p) {
  const float2 f = __ldg(reinterpret_cast<const float2*>(p));
  return {f.x, f.y};
}
__device__ __forceinline__ T2v<double> ld2(const double* p) { return {__ldg(p), __ldg(p + 1)}; }

// ------------------------------------------------------------- scatter ----
// Grid node u receives sum_i [w_i(u) v_i^0 + sum_p dw_{i,p}(u) v_i^p] over the
// points i whose stencil covers u, i.e. whose cell (first stencil node) f
// satisfies u - S + 1 <= f <= u per dimension.  The cells of the last
// dimension are contiguous in sorted order, so each (f_0, .., f_{d-2}) gives
// one range.  For d >= 2 SPLIT lanes share a node, lane `sub` taking the PER
// first-dimension cells f_0 = u_0 - S + 1 + sub PER + i; their partial sums
// are combined in a fixed order (deterministic).
constexpr int scatter_split(int D, int S) { return D > 1 ? (S == 4 ? 4 : 2) : 1; }

template <class T, int D, int CB, int S>
__global__ void __launch_bounds__(256) k_scatter(MvmGeo g, const int* __restrict__ cell_start,
                                                 const int* __restrict__ cell,
                                                 const T* __restrict__ wt,
                                                 const T* __restrict__ v, T* __restrict__ grid,
                                                 int s, long long N, long long M) {
  constexpr int SPLIT = scatter_split(D, S);
  constexpr int PER = D > 1 ? S / SPLIT : 1;
  constexpr int TW = 2 * S;   // table values per point and dimension
  const long long tix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long u = tix / SPLIT;
  const int sub = (int)(tix % SPLIT);
  const bool valid = u < M;
  const int q0 = blockIdx.y * CB;
  int uc[3] = {0, 0, 0};
  {
    long long t = valid ? u : 0;
    for (int k = D - 1; k >= 0; --k) {
      uc[k] = (int)(t % g.m[k]);
      t /= g.m[k];
    }
  }
  T acc[CB];
#pragma unroll
  for (int q = 0; q < CB; ++q) acc[q] = T(0);
  const int L = D - 1;   // last (fastest) dimension
  const int lo_l = max(0, uc[L] - (S - 1)), hi_l = min(uc[L], g.mc[L] - 1);
  int lo1 = 0, hi1 = 0;
  if (D > 2) {
    lo1 = max(0, uc[1] - (S - 1));
    hi1 = min(uc[1], g.mc[1] - 1);
  }
  for (int i0 = 0; i0 < PER; ++i0) {
    int f0 = 0;
    bool active = valid && lo_l <= hi_l;
    if (D > 1) {
      f0 = uc[0] - (S - 1) + sub * PER + i0;
      active = active && f0 >= 0 && f0 <= g.mc[0] - 1;
    }
    if (!active) continue;
    for (int f1 = lo1; f1 <= hi1; ++f1) {
      long long rowbase;
      if (D == 1) rowbase = 0;
      else if (D == 2) rowbase = (long long)f0 * g.mc[1];
      else rowbase = ((long long)f0 * g.mc[1] + f1) * g.mc[2];
      const int js = cell_start[rowbase + lo_l];
      const int je = cell_start[rowbase + hi_l + 1];
      for (int j = js; j < je; ++j) {
        const int fl = (int)(cell[j] - rowbase);
        const int ol = uc[L] - fl;
        // weights of this point at this node from the per-point table
        const T* wj = wt + (long long)j * (TW * D);
        T c[D + 1];
        if (D == 1) {
          c[0] = wj[ol];
          c[1] = wj[S + ol];
        } else if (D == 2) {
          const int o0 = uc[0] - f0;
          const T w0 = wj[o0], dw0 = wj[S + o0], w1 = wj[TW + ol], dw1 = wj[TW + S + ol];
          c[0] = w0 * w1;
          c[1] = dw0 * w1;
          c[D > 1 ? 2 : 0] = w0 * dw1;
        } else {
          const int o0 = uc[0] - f0, o1 = uc[D > 2 ? 1 : 0] - f1;
          const T w0 = wj[o0], dw0 = wj[S + o0], w1 = wj[TW + o1], dw1 = wj[TW + S + o1];
          const T w2 = wj[2 * TW + ol], dw2 = wj[2 * TW + S + ol];
          const T w01 = w0 * w1;
          c[0] = w01 * w2;
          c[1] = dw0 * w1 * w2;
          c[D > 1 ? 2 : 0] = w0 * dw1 * w2;
          c[D > 2 ? 3 : 0] = w01 * dw2;
        }
        const long long e = (long long)j * (D + 1);
#pragma unroll
        for (int q = 0; q < CB; ++q) {
          if (q0 + q < s) {
            const T* vq = v + (long long)(q0 + q) * N + e;
            T a = acc[q];
#pragma unroll
            for (int cc = 0; cc <= D; ++cc) a += c[cc] * vq[cc];
            acc[q] = a;
          }
        }
      }
    }
  }
  // fixed-order combination over the node's lanes: (sub0 + sub1) + (sub2 + sub3)
#pragma unroll
  for (int o = 1; o < SPLIT; o <<= 1)
#pragma unroll
    for (int q = 0; q < CB; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
  if (valid && sub == 0) {
#pragma unroll
    for (int q = 0; q < CB; ++q)
      if (q0 + q < s) grid[(long long)(q0 + q) * M + u] = acc[q];
  }
}

// ------------------------------------------ sum-factorised FP64 scatter ----
// The weight of point j at node u is a product over dimensions, so the node
// sum factors: with o_k = u_k - f_k the point's offset in dimension k
// (0 <= o_k < S),
//   d = 2:  w1[o1] A[o0] + dw1[o1] B[o0],
//           A[o0] = w0[o0] v^0 + dw0[o0] v^1,  B[o0] = w0[o0] v^2;
//   d = 3:  w2[o2] P[o0][o1] + dw2[o2] Q[o0][o1],
//           P = w1[o1] (w0[o0] v^0 + dw0[o0] v^1) + dw1[o1] w0[o0] v^2,
//           Q = w0[o0] w1[o1] v^3.
// A point-parallel pass forms A, B (P, Q) once per point; the node pass then
// costs two FMAs per (node, point) instead of six (eight), which matters on
// GB300 where FP64 arithmetic bounds the scatter.
// PCG fusion: with z != NULL the pass first replaces v by z + beta_q v (the
// CG search-direction update) and writes it back, then forms the products.
template <int D, int S>
__global__ void __launch_bounds__(256) k_scatter_prep(const double* __restrict__ wt,
                                                      double* __restrict__ v, int s,
                                                      int n, long long N, double sv, double sg,
                                                      const double* __restrict__ z,
                                                      const double* __restrict__ beta,
                                                      double* __restrict__ ab, CgUpdate up) {
  constexpr int NC = D == 2 ? 2 * S : 2 * S * S;   // coefficients per point and column
  const long long jt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = jt < n;
  double rsum[4] = {0.0, 0.0, 0.0, 0.0};   // ||r||^2 partials (fused CG update, s <= 4)
  const long long j = live ? jt : 0;
  const double* wj = wt + j * (2 * S * D);
#pragma unroll
  for (int q = 0; q < 4; ++q) {   // s <= 4 on this path
    if (q >= s || !live) break;
    double* vq0 = v + (long long)q * N + j * (D + 1);
    if (z) {
      const double* zq = z + (long long)q * N + j * (D + 1);
      const double be = beta[q];
#pragma unroll
      for (int c = 0; c <= D; ++c) vq0[c] = fma(be, vq0[c], zq[c]);
    }
    if (up.x && up.active[q]) {
      // x += alpha p, r -= alpha q (v is r), ||r||^2
      const long long o = (long long)q * N + j * (D + 1);
      const double al = up.alpha[q];
#pragma unroll
      for (int c = 0; c <= D; ++c) {
        up.x[o + c] = fma(al, up.p[o + c], up.x[o + c]);
        const double ri = fma(-al, up.q[o + c], vq0[c]);
        vq0[c] = ri;
        rsum[q] = fma(ri, ri, rsum[q]);
      }
    }
    double vq[D + 1];
    vq[0] = sv * vq0[0];
#pragma unroll
    for (int c = 1; c <= D; ++c) vq[c] = sg * vq0[c];
    double* o = ab + ((long long)q * n + j) * NC;
    if (D == 2) {
#pragma unroll
      for (int a = 0; a < S; ++a) {
        o[a] = wj[a] * vq[0] + wj[S + a] * vq[1];
        o[S + a] = wj[a] * vq[2];
      }
    } else {
#pragma unroll
      for (int a = 0; a < S; ++a) {
        const double t0 = wj[a] * vq[0] + wj[S + a] * vq[1];
        const double t1 = wj[a] * vq[2];
        const double t2 = wj[a] * vq[D > 2 ? 3 : 0];
#pragma unroll
        for (int b = 0; b < S; ++b) {
          o[a * S + b] = wj[2 * S + b] * t0 + wj[3 * S + b] * t1;
          o[S * S + a * S + b] = wj[2 * S + b] * t2;
        }
      }
    }
  }
  if (up.x) {
    __shared__ double red[8][4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double t = rsum[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) red[w][q] = t;
    }
    __syncthreads();
    if (threadIdx.x < 4 && (int)threadIdx.x < s) {
      double t = 0.0;
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) t += red[ww][threadIdx.x];
      up.dpart[(long long)threadIdx.x * gridDim.x + blockIdx.x] = t;
    }
  }
}


template <int D, int CB, int S>
__global__ void __launch_bounds__(256) k_scatter_ab(MvmGeo g, const int* __restrict__ cell_start,
                                                    const int* __restrict__ cell,
                                                    const double* __restrict__ wt,
                                                    const double* __restrict__ ab,
                                                    double* __restrict__ grid, int s, int n,
                                                    long long M) {
  constexpr int NC = D == 2 ? 2 * S : 2 * S * S;
  constexpr int SPLIT = scatter_split(D, S), PER = S / SPLIT;
  const long long tix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long u = tix / SPLIT;
  const int sub = (int)(tix % SPLIT);
  const bool valid = u < M;
  const int q0 = blockIdx.y * CB;
  int uc[3] = {0, 0, 0};
  {
    long long t = valid ? u : 0;
    for (int k = D - 1; k >= 0; --k) {
      uc[k] = (int)(t % g.m[k]);
      t /= g.m[k];
    }
  }
  double acc[CB];
#pragma unroll
  for (int q = 0; q < CB; ++q) acc[q] = 0.0;
  const int L = D - 1;
  const int lo_l = max(0, uc[L] - (S - 1)), hi_l = min(uc[L], g.mc[L] - 1);
  int lo1 = 0, hi1 = 0;
  if (D > 2) {
    lo1 = max(0, uc[1] - (S - 1));
    hi1 = min(uc[1], g.mc[1] - 1);
  }
  for (int i0 = 0; i0 < PER; ++i0) {
    const int f0 = uc[0] - (S - 1) + sub * PER + i0;
    const int o0 = uc[0] - f0;
    if (!(valid && lo_l <= hi_l && f0 >= 0 && f0 <= g.mc[0] - 1)) continue;
    for (int f1 = lo1; f1 <= hi1; ++f1) {
      const long long rowbase = D == 2 ? (long long)f0 * g.mc[1]
                                       : ((long long)f0 * g.mc[1] + f1) * g.mc[D > 2 ? 2 : 1];
      const int js = cell_start[rowbase + lo_l];
      const int je = cell_start[rowbase + hi_l + 1];
      const int ci = D == 2 ? o0 : o0 * S + (uc[D > 2 ? 1 : 0] - f1);   // coefficient index
      for (int j = js; j < je; ++j) {
        const int ol = uc[L] - (int)(cell[j] - rowbase);
        const double wl = wt[(long long)j * (2 * S * D) + 2 * S * L + ol];
        const double dl = wt[(long long)j * (2 * S * D) + 2 * S * L + S + ol];
#pragma unroll
        for (int q = 0; q < CB; ++q) {
          if (q0 + q < s) {
            const double* c = ab + ((long long)(q0 + q) * n + j) * NC;
            acc[q] = fma(wl, c[ci], fma(dl, c[NC / 2 + ci], acc[q]));
          }
        }
      }
    }
  }
#pragma unroll
  for (int o = 1; o < SPLIT; o <<= 1)
#pragma unroll
    for (int q = 0; q < CB; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
  if (valid && sub == 0) {
#pragma unroll
    for (int q = 0; q < CB; ++q)
      if (q0 + q < s) grid[(long long)(q0 + q) * M + u] = acc[q];
  }
}

// ------------------------------------------------- scatter, d = 2, by cell ----
// Two passes, both deterministic (fixed summation orders, no atomics):
//   1. per cell: S[q][a][b][cell] = sum over the cell's points j of
//        w0_a w1_b v0_j + w0'_a w1_b v1_j + w0_a w1'_b v2_j
//      (the point's contribution to stencil node (c0 + a, c1 + b)); a group
//      of G lanes takes one cell, each lane a stride-G subset of its points
//      (read once, coalesced, sorted by cell), and a fixed butterfly over the
//      group adds the lanes' sums.  G follows the mean points per cell.
//   2. per node: g[q][u0][u1] = sum_{a, b} S[q][a][b][(u0 - a, u1 - b)] over
//      the (up to) 16 cells whose stencil holds the node; consecutive nodes
//      read consecutive cells of one plane.
// Each point is read once (the node-owned pull above reads it 16 times);
// the per-cell planes hold 16 values per cell and column.  Cubic (4-node)
// stencils only; the quintic stencil takes the node-owned pull.
// Optional, as in k_scatter_prep: v0 scaled by sv, v1, v2 by sg; with z,
// p = z + beta p is formed first and written back (fused PCG direction).
template <class T, int CB, int G>
__global__ void __launch_bounds__(256) k_scatter_cells(const int* __restrict__ cell_start,
                                                       const T* __restrict__ frac, T ih0, T ih1,
                                                       T* __restrict__ v,
                                                       T* __restrict__ S, int s, long long N,
                                                       int ncell, T sv, T sg,
                                                       const double* __restrict__ z,
                                                       const double* __restrict__ beta) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = (int)(t / G), g = (int)(t % G);
  const bool live = c < ncell;   // whole groups: ncell groups, G | 32
  const int q0 = blockIdx.y * CB;
  T acc[CB][16];
#pragma unroll
  for (int q = 0; q < CB; ++q)
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[q][k] = T(0);
  // one point's contribution, its values already loaded: the weights from
  // its two cell fractions, the scalings, the sum-factorised stencil
  auto add_point = [&](const T2v<T>& fr, T (&vp)[CB][3]) {
    T w[16];
    keys4<T>(fr.x, w, w + 4);
    keys4<T>(fr.y, w + 8, w + 12);
#pragma unroll
    for (int q = 0; q < CB; ++q) {
      const T v0 = vp[q][0] * sv, v1 = vp[q][1] * (sg * ih0), v2 = vp[q][2] * (sg * ih1);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const T ca = fma(w[a], v0, w[4 + a] * v1);
        const T ea = w[a] * v2;
#pragma unroll
        for (int b = 0; b < 4; ++b)
          acc[q][a * 4 + b] = fma(w[8 + b], ca, fma(w[12 + b], ea, acc[q][a * 4 + b]));
      }
    }
  };
  if (live && !z) {
    // two points per lane and trip, both points' loads issued before either
    // is used: one point per trip left too few loads in flight for HBM
    const int js = cell_start[c], je = cell_start[c + 1];
    int j = js + g;
    for (; j + G < je; j += 2 * G) {
      const T2v<T> fa = ld2(frac + 2 * (long long)j), fb = ld2(frac + 2 * (long long)(j + G));
      T va[CB][3], vb[CB][3];
#pragma unroll
      for (int q = 0; q < CB; ++q) {
        const bool on = q0 + q < s;
        const T* pa = v + (long long)(q0 + q) * N + (long long)j * 3;
        const T* pb = pa + 3 * (long long)G;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          va[q][cc] = on ? pa[cc] : T(0);
          vb[q][cc] = on ? pb[cc] : T(0);
        }
      }
      add_point(fa, va);
      add_point(fb, vb);
    }
    if (j < je) {
      const T2v<T> fa = ld2(frac + 2 * (long long)j);
      T va[CB][3];
#pragma unroll
      for (int q = 0; q < CB; ++q) {
        const bool on = q0 + q < s;
        const T* pa = v + (long long)(q0 + q) * N + (long long)j * 3;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) va[q][cc] = on ? pa[cc] : T(0);
      }
      add_point(fa, va);
    }
  } else if (live) {
    const int js = cell_start[c], je = cell_start[c + 1];
    for (int j = js + g; j < je; j += G) {
      // the point's weights from its two cell fractions (the 12 bytes of
      // geometry a point carries, instead of a 64-byte weight table):
      // w[0..3] = phi, w[4..7] = phi' in dimension 0, w[8..15] likewise in 1;
      // the 1/h of the derivative weights scales the point's gradient values
      T w[16];
      const T2v<T> fr = ld2(frac + 2 * (long long)j);
      keys4<T>(fr.x, w, w + 4);
      keys4<T>(fr.y, w + 8, w + 12);
#pragma unroll
      for (int q = 0; q < CB; ++q) {
        if (q0 + q >= s) break;
        T* vj = v + (long long)(q0 + q) * N + (long long)j * 3;
        T v0 = vj[0], v1 = vj[1], v2 = vj[2];
        if (z) {   // p = z + beta p (double vectors only)
          const double* zj = z + (long long)(q0 + q) * N + (long long)j * 3;
          const double be = beta[q0 + q];
          v0 = (T)fma(be, (double)v0, zj[0]);
          v1 = (T)fma(be, (double)v1, zj[1]);
          v2 = (T)fma(be, (double)v2, zj[2]);
          vj[0] = v0;
          vj[1] = v1;
          vj[2] = v2;
        }
        v0 *= sv;
        v1 *= sg * ih0;   // dW_0 = phi'(dimension 0) / h_0
        v2 *= sg * ih1;   // dW_1 = phi'(dimension 1) / h_1
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const T ca = fma(w[a], v0, w[4 + a] * v1);   // sum-factorised over dimension 0
          const T ea = w[a] * v2;
#pragma unroll
          for (int b = 0; b < 4; ++b)
            acc[q][a * 4 + b] = fma(w[8 + b], ca, fma(w[12 + b], ea, acc[q][a * 4 + b]));
        }
      }
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < CB; ++q)
#pragma unroll
      for (int k = 0; k < 16; ++k) acc[q][k] += __shfl_xor_sync(0xffffffffu, acc[q][k], o);
  if (!live) return;
#pragma unroll
  for (int q = 0; q < CB; ++q) {
    if (q0 + q >= s) break;
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (k % G == g) S[((long long)(q0 + q) * 16 + k) * ncell + c] = acc[q][k];
  }
}

template <class T, int CB>
__global__ void __launch_bounds__(256) k_scatter_nodes(MvmGeo geo, const T* __restrict__ S,
                                                       T* __restrict__ grid, int s, long long M,
                                                       int ncell) {
  const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= M) return;
  const int u0 = (int)(u / geo.m[1]), u1 = (int)(u % geo.m[1]);
  const int q0 = blockIdx.y * CB;
  T acc[CB];
#pragma unroll
  for (int q = 0; q < CB; ++q) acc[q] = T(0);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int c0 = u0 - a;
    if (c0 < 0 || c0 >= geo.mc[0]) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c1 = u1 - b;
      if (c1 < 0 || c1 >= geo.mc[1]) continue;
      const long long cell = (long long)c0 * geo.mc[1] + c1;
#pragma unroll
      for (int q = 0; q < CB; ++q)
        if (q0 + q < s) acc[q] += S[((long long)(q0 + q) * 16 + a * 4 + b) * ncell + cell];
    }
  }
#pragma unroll
  for (int q = 0; q < CB; ++q)
    if (q0 + q < s) grid[(long long)(q0 + q) * M + u] = acc[q];
}

// ------------------------------- FP64_TC scatter, d = 2, double-float ----
// k_scatter_cells' two passes at FP64-class accuracy on the FP32 units
// (GB300 runs FP32 ~60x faster than FP64), after a point-parallel pass that
// does each point's FP64 work with every lane busy:
//   0. per point (k_scatter_split_df): the CG steps a pass may carry, in
//      FP64 -- p = z + beta p (written back), or x += alpha p, r -= alpha q
//      (r written back) with per-block partial sums of ||r||^2 (column q at
//      dpart[q gridDim.x + block]) -- then each value split into a
//      double-float pair hi + lo (split_trunc, < 2^-47) and v^0 scaled by
//      sv, v^1..2 by sg in double-float;
//   1. per cell (k_scatter_cells_df): the 16 stencil sums of the cell's
//      points with the weights as pairs (Wdf), every product and sum an
//      error-free transformation (FMA exact product, TwoSum), so each sum
//      carries ~2^-48 relative error of the magnitudes it adds (FP64:
//      2^-53); G lanes per cell, a fixed butterfly adds the lanes;
//   2. per node (k_scatter_nodes_df): the 16 cells' sums in a fixed order,
//      rounded once to FP64.
// Column q = blockIdx.y in every pass.
__device__ __forceinline__ void df_prod(float ah, float al, float bh, float bl, float& ph,
                                        float& pl) {
  const float p = ah * bh;
  const float e = fmaf(ah, bh, -p);
  const float t = fmaf(ah, bl, fmaf(al, bh, e));
  ph = p + t;              // |t| << |p|: Fast2Sum renormalises exactly
  pl = t - (ph - p);
}

// x = hi + lo + e with |e| < 2^-47 |x|: hi is x truncated to a 24-bit
// significand and lo the next 24 bits of x's significand (truncated), both
// assembled from the bit pattern with integer operations.  split_d's
// conversions and subtraction run on GB300's FP64 pipe, which bound the
// point pass (ncu: 64% busy); these need none.  Outside 2^-79 <= |x| <
// 2^128 (where hi or lo would leave FP32's normal range): split_d.
__device__ __forceinline__ void split_trunc(double x, float& hi, float& lo) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const int E = (int)((hw >> 20) & 0x7FF);
  if (E < 944 || E > 1150) {
    split_d(x, hi, lo);
    return;
  }
  const unsigned sign = hw & 0x80000000u;
  hi = __uint_as_float(sign | ((unsigned)(E - 896) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
  const unsigned r24 = (lw & 0x1FFFFFFFu) >> 5;
  if (r24 == 0) {
    lo = 0.f;
    return;
  }
  const int lz = __clz(r24) - 8;   // leading zeros within the 24 bits
  lo = __uint_as_float(sign | ((unsigned)(E - 920 - lz) << 23) | ((r24 << lz) & 0x7FFFFFu));
}

// sv, sg as double-float pairs (split on the host); scaled: apply them
__global__ void __launch_bounds__(256) k_scatter_split_df(
    double* __restrict__ v, float2* __restrict__ Vdf, int n, long long N, bool scaled, float2 svp,
    float2 sgp, const double* __restrict__ z, const double* __restrict__ beta, CgUpdate up) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  const bool live = j < n;
  const bool upd = up.x != nullptr && up.active[q] != 0;
  double rs = 0.0;
  if (live) {
    const long long o = (long long)q * N + (long long)j * 3;
    double vv[3] = {v[o], v[o + 1], v[o + 2]};
    if (z) {
      const double be = beta[q];
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        vv[cc] = fma(be, vv[cc], z[o + cc]);
        v[o + cc] = vv[cc];
      }
    }
    if (upd) {
      const double alpha = up.alpha[q];
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        up.x[o + cc] = fma(alpha, up.p[o + cc], up.x[o + cc]);
        vv[cc] = fma(-alpha, up.q[o + cc], vv[cc]);
        v[o + cc] = vv[cc];
        rs = fma(vv[cc], vv[cc], rs);
      }
    }
    float2* out = Vdf + ((long long)q * n + j) * 3;
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      float hi, lo;
      split_trunc(vv[cc], hi, lo);
      if (scaled) {   // v^0 sv, v^1..2 sg, in double-float
        const float2 sc = cc == 0 ? svp : sgp;
        df_prod(hi, lo, sc.x, sc.y, hi, lo);
      }
      out[cc] = make_float2(hi, lo);
    }
  }
  if (up.x) {
    __shared__ double red[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double t = rs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[w] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = 0.0;
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) b += red[ww];
      up.dpart[(long long)q * gridDim.x + blockIdx.x] = b;
    }
  }
}

template <int G>
__global__ void __launch_bounds__(256) k_scatter_cells_df(const int* __restrict__ cell_start,
                                                          const float2* __restrict__ Wdf,
                                                          const float2* __restrict__ Vdf, int n,
                                                          float2* __restrict__ S, int ncell) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = (int)(t / G), g = (int)(t % G);
  const bool live = c < ncell;   // whole groups: G | 32
  const int q = blockIdx.y;
  float ah[16], al[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    ah[k] = 0.f;
    al[k] = 0.f;
  }
  if (live) {
    const int js = cell_start[c], je = cell_start[c + 1];
    for (int j = js + g; j < je; j += G) {
      const float2* vj = Vdf + ((long long)q * n + j) * 3;
      const float2 v0 = vj[0], v1 = vj[1], v2 = vj[2];
      float2 w[16];   // w0[0..3], dw0[0..3] (dimension 0), w1, dw1 (dimension 1)
      const float4* w4 = reinterpret_cast<const float4*>(Wdf + (long long)j * 16);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float4 x = __ldg(w4 + k);
        w[2 * k] = make_float2(x.x, x.y);
        w[2 * k + 1] = make_float2(x.z, x.w);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        // A = w0_a v0 + dw0_a v1, B = w0_a v2 (sum-factorised over dimension 0)
        float Ah, Al, Bh, Bl;
        df_prod(w[a].x, w[a].y, v0.x, v0.y, Ah, Al);
        df_fma(w[4 + a].x, w[4 + a].y, v1.x, v1.y, Ah, Al);
        {
          float sh, se;
          two_sum(Ah, Al, sh, se);
          Ah = sh;
          Al = se;
        }
        df_prod(w[a].x, w[a].y, v2.x, v2.y, Bh, Bl);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          df_fma(w[8 + b].x, w[8 + b].y, Ah, Al, ah[a * 4 + b], al[a * 4 + b]);
          df_fma(w[12 + b].x, w[12 + b].y, Bh, Bl, ah[a * 4 + b], al[a * 4 + b]);
        }
      }
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float oh = __shfl_xor_sync(0xffffffffu, ah[k], o);
      const float ol = __shfl_xor_sync(0xffffffffu, al[k], o);
      df_add(ah[k], al[k], oh, ol);
    }
  if (!live) return;
#pragma unroll
  for (int k = 0; k < 16; ++k)
    if (k % G == g) {
      float sh, se;
      two_sum(ah[k], al[k], sh, se);
      S[((long long)q * 16 + k) * ncell + c] = make_float2(sh, se);
    }
}

// Per node: the 16 cells whose stencils hold it, added in double-float in
// a fixed order, rounded once to FP64.  Column q = blockIdx.y.
__global__ void __launch_bounds__(256) k_scatter_nodes_df(MvmGeo geo, const float2* __restrict__ S,
                                                          double* __restrict__ grid, long long M,
                                                          int ncell) {
  const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= M) return;
  const int q = blockIdx.y;
  const int u0 = (int)(u / geo.m[1]), u1 = (int)(u % geo.m[1]);
  float sh = 0.f, sl = 0.f;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int c0 = u0 - a;
    if (c0 < 0 || c0 >= geo.mc[0]) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c1 = u1 - b;
      if (c1 < 0 || c1 >= geo.mc[1]) continue;
      const float2 x = S[((long long)q * 16 + a * 4 + b) * ncell + (long long)c0 * geo.mc[1] + c1];
      df_add(sh, sl, x.x, x.y);
    }
  }
  grid[(long long)q * M + u] = (double)sh + (double)sl;
}

template <class T, int CB, int G>
void launch_scatter_cells(dski_handle h, T* v, T* S, int s, T sv, T sg, const double* z,
                          const double* beta, cudaStream_t st) {
  static_assert(std::is_same<T, float>::value, "the per-cell scatter reads the FP32 fractions");
  const int ncell = h->mc[0] * h->mc[1];
  const long long threads = (long long)ncell * G;
  const dim3 grd((unsigned)((threads + 255) / 256), (unsigned)((s + CB - 1) / CB));
  k_scatter_cells<T, CB, G><<<grd, 256, 0, st>>>(h->cell_start.as<int>(), h->frac32.as<float>(),
                                                  (T)(1.0 / h->h[0]), (T)(1.0 / h->h[1]), v, S,
                                                  s, h->N, ncell, sv, sg, z, beta);
}

// The gather's optional CG work: per-block partial sums of v^T out per
// column (fixed tree) to dpart[q gridDim.x + block], and a folded CG
// finisher: the last block completes the partial sums (fixed block order)
// and updates the device scalars.  All threads of every block call it.
template <int CB>
__device__ __forceinline__ void gather_partials(const double (&dsum)[CB], double* dpart, int q0,
                                                int s, CgFinish fin) {
  if (!dpart) return;
  __shared__ double red[8][CB];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < CB; ++q) {
    double t = dsum[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[w][q] = t;
  }
  __syncthreads();
  if (threadIdx.x < CB && q0 + (int)threadIdx.x < s) {
    double t = 0.0;
    for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) t += red[ww][threadIdx.x];
    dpart[(long long)(q0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
  }
  if (fin.kind >= 0 && last_block(fin.ticket, gridDim.x * gridDim.y)) {
    __shared__ double sh[32];
    __shared__ double tot[CG_MAXS];
    if (fin.kind == 0) {
      sum_columns(dpart, gridDim.x, fin.cs.s, 1, 0, tot, sh);
      alpha_finish(tot, fin.cs);
    } else {
      sum_columns(fin.part2, fin.nb2 > 0 ? fin.nb2 : (int)gridDim.x, fin.cs.s, 1, 0, tot, sh);
      update_finish(tot, fin.cs, sh);
      __syncthreads();   // active flags settled before beta reads them
      sum_columns(dpart, gridDim.x, fin.cs.s, 1, 0, tot, sh);
      beta_finish(tot, fin.cs, 0);
    }
  }
}

// -------------------------------------------------------------- gather ----
// out_j^0 = av sum_u w_j(u) h(u) + nv v_j^0,
// out_j^p = ag sum_u dw_{j,p}(u) h(u) + ng v_j^p,
// evaluated dimension by dimension over the S^d stencil (av = ag = 1 and
// nv, ng the noise for the MVM; other values for the preconditioner).
template <class T, int D, int CB, int S>
__global__ void __launch_bounds__(256) k_gather(MvmGeo g, const int* __restrict__ cell,
                                                const T* __restrict__ wt,
                                                const T* __restrict__ grid,
                                                const T* __restrict__ v, T* __restrict__ out,
                                                int s, int n, long long N, long long M, T nv,
                                                T ng, T av, T ag, double* __restrict__ dpart,
                                                CgFinish fin) {
  const int jt = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = jt < n;
  const int j = live ? jt : n - 1;   // dead threads redo the last point, write nothing
  const int q0 = blockIdx.y * CB;
  double dsum[CB];
#pragma unroll
  for (int q = 0; q < CB; ++q) dsum[q] = 0.0;
  int f[3] = {0, 0, 0};
  {
    int t = cell[j];
    for (int k = D - 1; k >= 0; --k) {
      f[k] = t % g.mc[k];
      t /= g.mc[k];
    }
  }
  T w[D][S], dw[D][S];
  if constexpr (std::is_same<T, float>::value) {
    // FP32: the weights from the point's D cell fractions (wt is the FP32
    // fraction array, n x D) -- the geometry the byte model counts, instead
    // of a 2 S D-value weight table per point
#pragma unroll
    for (int k = 0; k < D; ++k) {
      stencil_weights<S, T>(__ldg(wt + (long long)j * D + k), w[k], dw[k]);
      const T ih = (T)g.invh[k];
#pragma unroll
      for (int o = 0; o < S; ++o) dw[k][o] *= ih;
    }
  } else {
    const T* wj = wt + (long long)j * (2 * S * D);
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int o = 0; o < S; ++o) {
        w[k][o] = wj[2 * S * k + o];
        dw[k][o] = wj[2 * S * k + S + o];
      }
  }
  long long base = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) base = base * g.m[k] + f[k];
  const long long e = (long long)j * (D + 1);
#pragma unroll
  for (int q = 0; q < CB; ++q) {
    if (q0 + q >= s) break;
    const T* hq = grid + (long long)(q0 + q) * M + base;
    T r[D + 1];
#pragma unroll
    for (int cc = 0; cc <= D; ++cc) r[cc] = T(0);
    if (D == 1) {
#pragma unroll
      for (int a = 0; a < S; ++a) {
        const T x = hq[a];
        r[0] += w[0][a] * x;
        r[1] += dw[0][a] * x;
      }
    } else if (D == 2) {
      const int s1 = g.m[D > 1 ? 1 : 0];
#pragma unroll
      for (int a = 0; a < S; ++a) {
        T rw = T(0), rd = T(0);
#pragma unroll
        for (int b = 0; b < S; ++b) {
          const T x = hq[(long long)a * s1 + b];
          rw += w[D > 1 ? 1 : 0][b] * x;
          rd += dw[D > 1 ? 1 : 0][b] * x;
        }
        r[0] += w[0][a] * rw;
        r[1] += dw[0][a] * rw;
        r[D > 1 ? 2 : 0] += w[0][a] * rd;
      }
    } else {
      const long long s1 = (long long)g.m[1] * g.m[2];
      const int s2 = g.m[2];
#pragma unroll
      for (int a = 0; a < S; ++a) {
        T aw = T(0), ad1 = T(0), ad2 = T(0);
#pragma unroll
        for (int b = 0; b < S; ++b) {
          T lw = T(0), ld = T(0);
#pragma unroll
          for (int c2 = 0; c2 < S; ++c2) {
            const T x = hq[a * s1 + (long long)b * s2 + c2];
            lw += w[D > 2 ? 2 : 0][c2] * x;
            ld += dw[D > 2 ? 2 : 0][c2] * x;
          }
          aw += w[D > 1 ? 1 : 0][b] * lw;
          ad1 += dw[D > 1 ? 1 : 0][b] * lw;
          ad2 += w[D > 1 ? 1 : 0][b] * ld;
        }
        r[0] += w[0][a] * aw;
        r[1] += dw[0][a] * aw;
        r[D > 1 ? 2 : 0] += w[0][a] * ad1;
        r[D > 2 ? 3 : 0] += w[0][a] * ad2;
      }
    }
    const T* vq = v + (long long)(q0 + q) * N + e;
    T* oq = out + (long long)(q0 + q) * N + e;
    T o[D + 1];
    o[0] = av * r[0] + nv * vq[0];
#pragma unroll
    for (int cc = 1; cc <= D; ++cc) o[cc] = ag * r[cc] + ng * vq[cc];
    if (live) {
#pragma unroll
      for (int cc = 0; cc <= D; ++cc) oq[cc] = o[cc];
      if (dpart)
#pragma unroll
        for (int cc = 0; cc <= D; ++cc) dsum[q] = fma((double)vq[cc], (double)o[cc], dsum[q]);
    }
  }
  gather_partials<CB>(dsum, dpart, q0, s, fin);
}

// ----------------------------------------------- FP32 gather, d = 2 ----
// The MIXED modes' gather without partial sums (cubic stencil): two
// consecutive points per thread, every load of both points (cells,
// fractions, the 2 x 16 grid values, v) issued before either point's sums,
// since one point per thread left too few loads in flight for HBM.  The
// weights come from the FP32 fractions; the sums are k_gather's.  Column
// q = blockIdx.y.
__global__ void __launch_bounds__(256) k_gather2_f32(MvmGeo g, const int* __restrict__ cell,
                                                     const float* __restrict__ frac,
                                                     const float* __restrict__ grid,
                                                     const float* __restrict__ v,
                                                     float* __restrict__ out, int n, long long N,
                                                     long long M, float nv, float ng, float av,
                                                     float ag) {
  const int j0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (j0 >= n) return;
  const bool two = j0 + 1 < n;
  const int jp[2] = {j0, two ? j0 + 1 : j0};
  const int q = blockIdx.y;
  const int m1 = g.m[1], mc1 = g.mc[1];
  float x[2][16], fr[2][2], vv[2][3];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int c = __ldg(cell + jp[u]);
    const T2v<float> f = ld2(frac + 2 * (long long)jp[u]);
    fr[u][0] = f.x;
    fr[u][1] = f.y;
    const int f0 = c / mc1, f1 = c - f0 * mc1;
    const float* hq = grid + (long long)q * M + (long long)f0 * m1 + f1;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) x[u][a * 4 + b] = __ldg(hq + (long long)a * m1 + b);
    const float* vq = v + (long long)q * N + (long long)jp[u] * 3;
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) vv[u][cc] = vq[cc];
  }
  const float ih0 = (float)g.invh[0], ih1 = (float)g.invh[1];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    if (u == 1 && !two) break;
    float w0[4], dw0[4], w1[4], dw1[4];
    stencil_weights<4, float>(fr[u][0], w0, dw0);
    stencil_weights<4, float>(fr[u][1], w1, dw1);
    float r0 = 0.f, r1 = 0.f, r2 = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      float rw = 0.f, rd = 0.f;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        rw += w1[b] * x[u][a * 4 + b];
        rd += dw1[b] * x[u][a * 4 + b];
      }
      r0 += w0[a] * rw;
      r1 += dw0[a] * rw;
      r2 += w0[a] * rd;
    }
    float* oq = out + (long long)q * N + (long long)jp[u] * 3;
    oq[0] = av * r0 + nv * vv[u][0];
    oq[1] = ag * (r1 * ih0) + ng * vv[u][1];
    oq[2] = ag * (r2 * ih1) + ng * vv[u][2];
  }
}

// ------------------------------- FP64_TC gather, d = 2, double-float ----
// The gather's stencil sums on the FP32 units at FP64-class accuracy: the
// grid (FP64) is first split in place into double-float pairs (split_trunc;
// 8 bytes per node either way), then each point
// forms its value and two derivative sums from the pairs and its weights
// (Wdf) with error-free products and TwoSum sums (~2^-48 of the magnitudes
// added), rounds each once to FP64 and finishes in FP64 exactly as k_gather:
// out^0 = av r^0 + nv v^0, out^p = ag r^p + ng v^p, the partial sums of
// v^T out and the folded CG finisher.  Column q = blockIdx.y.
__global__ void __launch_bounds__(256) k_grid_split_df(double* __restrict__ grid, long long count) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float hi, lo;
  split_trunc(grid[i], hi, lo);
  reinterpret_cast<float2*>(grid)[i] = make_float2(hi, lo);
}

__global__ void __launch_bounds__(256) k_gather_df(MvmGeo g, const int* __restrict__ cell,
                                                   const float2* __restrict__ Wdf,
                                                   const float2* __restrict__ G,
                                                   const double* __restrict__ v,
                                                   double* __restrict__ out, int s, int n,
                                                   long long N, long long M, double nv, double ng,
                                                   double av, double ag, double* __restrict__ dpart,
                                                   CgFinish fin) {
  const int jt = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = jt < n;
  const int j = live ? jt : n - 1;   // dead threads redo the last point, write nothing
  const int q = blockIdx.y;
  double dsum[1] = {0.0};
  const int t = cell[j];
  const int f0 = t / g.mc[1], f1 = t - f0 * g.mc[1];
  const int m1 = g.m[1];
  const float2* hq = G + (long long)q * M + (long long)f0 * m1 + f1;
  float2 w[16];   // w0[0..3], dw0[0..3], w1[0..3], dw1[0..3]
  const float4* w4 = reinterpret_cast<const float4*>(Wdf + (long long)j * 16);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 x = __ldg(w4 + k);
    w[2 * k] = make_float2(x.x, x.y);
    w[2 * k + 1] = make_float2(x.z, x.w);
  }
  float r0h = 0.f, r0l = 0.f, r1h = 0.f, r1l = 0.f, r2h = 0.f, r2l = 0.f;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    float th = 0.f, tl = 0.f, uh = 0.f, ul = 0.f;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float2 x = hq[(long long)a * m1 + b];
      df_fma(w[8 + b].x, w[8 + b].y, x.x, x.y, th, tl);
      df_fma(w[12 + b].x, w[12 + b].y, x.x, x.y, uh, ul);
    }
    float sh, se;
    two_sum(th, tl, sh, se);
    th = sh;
    tl = se;
    two_sum(uh, ul, sh, se);
    uh = sh;
    ul = se;
    df_fma(w[a].x, w[a].y, th, tl, r0h, r0l);
    df_fma(w[4 + a].x, w[4 + a].y, th, tl, r1h, r1l);
    df_fma(w[a].x, w[a].y, uh, ul, r2h, r2l);
  }
  const double r[3] = {(double)r0h + (double)r0l, (double)r1h + (double)r1l,
                       (double)r2h + (double)r2l};
  const long long e = (long long)q * N + (long long)j * 3;
  const double o0 = av * r[0] + nv * v[e];
  const double o1 = ag * r[1] + ng * v[e + 1];
  const double o2 = ag * r[2] + ng * v[e + 2];
  if (live) {
    out[e] = o0;
    out[e + 1] = o1;
    out[e + 2] = o2;
    if (dpart) dsum[0] = fma(v[e], o0, fma(v[e + 1], o1, v[e + 2] * o2));
  }
  gather_partials<1>(dsum, dpart, q, s, fin);
}

// --------------------------------------------------- SIMT mode product ----
// Y[q][j][r] = scale * sum_i X[q][r][i] K[j][i]  (K symmetric m x m,
// X viewed as R x m with the contracted mode contiguous; the output has the
// contracted mode first: one step of the cyclic mode rotation).
template <class T, int TM, int TN>
__global__ void __launch_bounds__(256) k_mode_simt(const T* __restrict__ X,
                                                   const T* __restrict__ K, T* __restrict__ Y,
                                                   int m, long long R, T scale) {
  constexpr int BM = 16 * TM, BN = 16 * TN, BK = 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int j0 = blockIdx.y * BM;
  const long long r0 = (long long)blockIdx.x * BN;
  const long long qoff = (long long)blockIdx.z * R * m;
  const T* Xq = X + qoff;
  T* Yq = Y + qoff;
  T acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = T(0);
  for (int i0 = 0; i0 < m; i0 += BK) {
    for (int idx = threadIdx.x; idx < BM * BK; idx += 256) {
      const int jj = idx / BK, ii = idx % BK;
      const int gj = j0 + jj, gi = i0 + ii;
      As[ii][jj] = (gj < m && gi < m) ? K[(long long)gj * m + gi] : T(0);
    }
    for (int idx = threadIdx.x; idx < BN * BK; idx += 256) {
      const int rr = idx / BK, ii = idx % BK;
      const long long gr = r0 + rr;
      const int gi = i0 + ii;
      Bs[ii][rr] = (gr < R && gi < m) ? Xq[gr * m + gi] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int ii = 0; ii < BK; ++ii) {
      T a[TM], b[TN];
#pragma unroll
      for (int x = 0; x < TM; ++x) a[x] = As[ii][ty * TM + x];
#pragma unroll
      for (int y = 0; y < TN; ++y) b[y] = Bs[ii][tx * TN + y];
#pragma unroll
      for (int x = 0; x < TM; ++x)
#pragma unroll
        for (int y = 0; y < TN; ++y) acc[x][y] += a[x] * b[y];
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < TM; ++x) {
    const int gj = j0 + ty * TM + x;
    if (gj >= m) continue;
#pragma unroll
    for (int y = 0; y < TN; ++y) {
      const long long gr = r0 + tx * TN + y;
      if (gr < R) Yq[(long long)gj * R + gr] = scale * acc[x][y];
    }
  }
}

template <class T>
__global__ void k_perm_in(const int* __restrict__ perm, const T* __restrict__ vu,
                          T* __restrict__ vi, int n, int d, long long N, int s) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int i = perm[j];
  for (int q = 0; q < s; ++q)
    for (int c = 0; c <= d; ++c)
      vi[q * N + (long long)j * (d + 1) + c] = vu[q * N + (long long)c * n + i];
}

template <class T>
__global__ void k_perm_out(const int* __restrict__ perm, const T* __restrict__ vi,
                           T* __restrict__ vu, int n, int d, long long N, int s) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int i = perm[j];
  for (int q = 0; q < s; ++q)
    for (int c = 0; c <= d; ++c)
      vu[q * N + (long long)c * n + i] = vi[q * N + (long long)j * (d + 1) + c];
}

template <class T, int D, int CB, int S>
void launch_scatter(dski_handle h, const MvmGeo& g, const T* wt, const T* v, T* grid, int s,
                    cudaStream_t st) {
  const long long threads = (long long)h->M * scatter_split(D, S);
  dim3 grd((unsigned)((threads + 255) / 256), (unsigned)((s + CB - 1) / CB));
  StageScope sc(h, ST_SCATTER, st);
  k_scatter<T, D, CB, S><<<grd, 256, 0, st>>>(g, h->cell_start.as<int>(), h->cell.as<int>(), wt,
                                              v, grid, s, (long long)h->N, (long long)h->M);
}

struct GatherScale {
  double av = 1.0, ag = 1.0;   // multiply B h on value / gradient rows
  double nv = 0.0, ng = 0.0;   // multiply v on value / gradient rows
  int stage = ST_GATHER;
  double* dpart = nullptr;     // per-block partial sums of v^T out (FP64 only)
  CgFinish fin{};              // finisher folded into the last block (with dpart)
  // the grid is the caller's scratch: FP64_TC (d = 2, cubic) may split it
  // in place and take the double-float gather
  bool grid_scratch = false;
};

template <class T, int D, int CB, int S>
void launch_gather(dski_handle h, const MvmGeo& g, const T* wt, const T* grid, const T* v,
                   T* out, int s, cudaStream_t st, const GatherScale& gs) {
  // FP32 gathers evaluate the weights from the FP32 fractions
  if constexpr (std::is_same<T, float>::value) wt = h->frac32.as<float>();
  if constexpr (std::is_same<T, float>::value && D == 2 && S == 4) {
    if (!gs.dpart) {
      StageScope sc(h, gs.stage, st);
      const unsigned nt = (unsigned)((h->n + 1) / 2);
      k_gather2_f32<<<dim3((nt + 255) / 256, (unsigned)s), 256, 0, st>>>(
          g, h->cell.as<int>(), wt, grid, v, out, h->n, (long long)h->N, (long long)h->M,
          (float)gs.nv, (float)gs.ng, (float)gs.av, (float)gs.ag);
      return;
    }
  }
  if constexpr (std::is_same<T, double>::value && D == 2 && S == 4) {
    if (gs.grid_scratch && df_scatter_path(h, true)) {
      StageScope sc(h, gs.stage, st, 2);
      const long long cnt = (long long)h->M * s;
      double* gw = const_cast<double*>(grid);
      k_grid_split_df<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(gw, cnt);
      k_gather_df<<<dim3((unsigned)((h->n + 255) / 256), (unsigned)s), 256, 0, st>>>(
          g, h->cell.as<int>(), h->Wdf.as<float2>(), reinterpret_cast<const float2*>(gw), v, out,
          s, h->n, (long long)h->N, (long long)h->M, gs.nv, gs.ng, gs.av, gs.ag, gs.dpart,
          gs.fin);
      return;
    }
  }
  dim3 grd((unsigned)((h->n + 255) / 256), (unsigned)((s + CB - 1) / CB));
  StageScope sc(h, gs.stage, st);
  k_gather<T, D, CB, S><<<grd, 256, 0, st>>>(g, h->cell.as<int>(), wt, grid, v, out, s, h->n,
                                          (long long)h->N, (long long)h->M, (T)gs.nv, (T)gs.ng,
                                          (T)gs.av, (T)gs.ag, gs.dpart, gs.fin);
}

template <class T, int D>
void scatter_dispatch(dski_handle h, const MvmGeo& g, const T* wt, const T* v, T* grid, int s,
                      cudaStream_t st) {
  with_stencil(h, [&](auto Sc) {
    constexpr int S = decltype(Sc)::value;
    if (s == 1) launch_scatter<T, D, 1, S>(h, g, wt, v, grid, s, st);
    else if (s <= 4) launch_scatter<T, D, 4, S>(h, g, wt, v, grid, s, st);
    else launch_scatter<T, D, 8, S>(h, g, wt, v, grid, s, st);
  });
}

template <class T, int D>
void gather_dispatch(dski_handle h, const MvmGeo& g, const T* wt, const T* grid, const T* v,
                     T* out, int s, cudaStream_t st, const GatherScale* gsp = nullptr) {
  GatherScale gs;
  if (gsp) {
    gs = *gsp;
  } else {
    gs.nv = h->nv;
    gs.ng = h->ng;
  }
  with_stencil(h, [&](auto Sc) {
    constexpr int S = decltype(Sc)::value;
    if (s == 1) launch_gather<T, D, 1, S>(h, g, wt, grid, v, out, s, st, gs);
    else if (s <= 4) launch_gather<T, D, 4, S>(h, g, wt, grid, v, out, s, st, gs);
    else launch_gather<T, D, 8, S>(h, g, wt, grid, v, out, s, st, gs);
  });
}

template <class T>
void mode_simt_variant(int v, const T* X, const T* K, T* Y, int m, long long R, int s, T scale,
                       cudaStream_t st) {
  const int b = v == 0 ? 64 : (v == 1 ? 32 : 16);
  dim3 grd((unsigned)((R + b - 1) / b), (unsigned)((m + b - 1) / b), (unsigned)s);
  if (v == 0) k_mode_simt<T, 4, 4><<<grd, 256, 0, st>>>(X, K, Y, m, R, scale);
  else if (v == 1) k_mode_simt<T, 2, 2><<<grd, 256, 0, st>>>(X, K, Y, m, R, scale);
  else k_mode_simt<T, 1, 1><<<grd, 256, 0, st>>>(X, K, Y, m, R, scale);
}

// Tile autotuner of the SIMT mode product: the first product of a given
// (element size, m, R, s) on a device times the three tile shapes (64, 32,
// 16 square; one warm-up and three timed launches each, CUDA events on the
// caller's stream) and remembers the fastest.  While the stream is being
// captured into a graph no timing is possible and a CTA-count heuristic picks.
struct TuneKey {
  int dev, es, m, s;
  long long R;
  bool operator<(const TuneKey& o) const {
    if (dev != o.dev) return dev < o.dev;
    if (es != o.es) return es < o.es;
    if (m != o.m) return m < o.m;
    if (s != o.s) return s < o.s;
    return R < o.R;
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;
thread_local bool g_no_tune = false;   // set by callers that must not create events

template <class T>
int pick_variant(const T* X, const T* K, T* Y, int m, long long R, int s, T scale, int sms,
                 cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  const TuneKey key{dev, (int)sizeof(T), m, s, R};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  auto ctas = [&](int b) { return ((R + b - 1) / b) * (long long)((m + b - 1) / b) * s; };
  const int heur = ctas(64) >= 2LL * sms ? 0 : (ctas(32) >= 2LL * sms ? 1 : 2);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (g_no_tune || cudaStreamIsCapturing(st, &cap) != cudaSuccess ||
      cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return heur;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    cudaGetLastError();
    if (a) cudaEventDestroy(a);
    return heur;
  }
  int best = heur;
  float best_ms = 1e30f;
  for (int v = 0; v < 3; ++v) {
    mode_simt_variant<T>(v, X, K, Y, m, R, s, scale, st);
    cudaEventRecord(a, st);
    for (int rep = 0; rep < 3; ++rep) mode_simt_variant<T>(v, X, K, Y, m, R, s, scale, st);
    cudaEventRecord(b, st);
    float ms = 0.f;
    if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess &&
        ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  count_launches(12);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  return best;
}

template <class T>
void mode_simt(dski_handle h, const T* X, const T* K, T* Y, int m, long long R, int s, T scale,
               int sms, cudaStream_t st) {
  const int v = pick_variant<T>(X, K, Y, m, R, s, scale, sms, st);
  StageScope sc(h, ST_KRON, st);
  mode_simt_variant<T>(v, X, K, Y, m, R, s, scale, st);
}

}  // namespace

void set_no_tune(bool on) { g_no_tune = on; }

// the FP32 d = 2 scatter takes the per-cell passes for cubic stencils
static bool cells_path(dski_handle h, bool prec64) { return h->d == 2 && !prec64 && h->sw == 4; }

bool df_scatter_path(dski_handle h, bool prec64) {
  return prec64 && h->prec == DSKI_FP64_TC && !h->kron_exact && h->d == 2 && h->sw == 4 &&
         h->Wdf.ptr != nullptr;
}

// lanes per cell of the double-float per-cell pass: about eight points per
// lane, as the FP32 pass
static int df_group(dski_handle h) {
  const double per = (double)h->n / std::max(1, h->mc[0] * h->mc[1]);
  return per <= 16.0 ? 2 : per <= 32.0 ? 4 : per <= 64.0 ? 8 : per <= 128.0 ? 16 : 32;
}

int scatter_update_blocks(dski_handle h) { return (h->n + 255) / 256; }

size_t scatter_ws_bytes(dski_handle h, int s, bool prec64) {
  if (cells_path(h, prec64)) return (size_t)s * 16 * h->mc[0] * h->mc[1] * 4;
  if (df_scatter_path(h, prec64))   // cell planes, then the points' double-float values
    return (size_t)s * (16 * (size_t)h->mc[0] * h->mc[1] + 3 * (size_t)h->n) * sizeof(float2);
  if (!(prec64 && h->d >= 2 && s <= 4)) return 0;
  const size_t S = (size_t)h->sw;
  return (size_t)s * h->n * (h->d == 2 ? 2 * S : 2 * S * S) * 8;
}

namespace {
// d = 2: the per-cell pass with the group size that fits the mean points per
// cell, then the per-node pass
template <class T, int CB>
void scatter_cells_d2(dski_handle h, T* v, T* S, T* grid, int s, T sv, T sg, const double* z,
                      const double* beta, cudaStream_t st) {
  // group size: about eight points per lane.  The pass is bound by
  // instruction issue (ncu at n = 1e7: issue slots 60% busy, DRAM 25%), and
  // the butterfly over the group costs 2 x 16 CB instructions per level and
  // lane, so fewer lanes per cell leave more issue slots to the points
  const int ncell = h->mc[0] * h->mc[1];
  const double per = (double)h->n / std::max(1, ncell);
  if (per <= 16.0) launch_scatter_cells<T, CB, 2>(h, v, S, s, sv, sg, z, beta, st);
  else if (per <= 32.0) launch_scatter_cells<T, CB, 4>(h, v, S, s, sv, sg, z, beta, st);
  else if (per <= 64.0) launch_scatter_cells<T, CB, 8>(h, v, S, s, sv, sg, z, beta, st);
  else if (per <= 128.0) launch_scatter_cells<T, CB, 16>(h, v, S, s, sv, sg, z, beta, st);
  else launch_scatter_cells<T, CB, 32>(h, v, S, s, sv, sg, z, beta, st);
  const dim3 gn((unsigned)((h->M + 255) / 256), (unsigned)((s + CB - 1) / CB));
  k_scatter_nodes<T, CB><<<gn, 256, 0, st>>>(make_geo(h), S, grid, s, h->M, ncell);
}
}  // namespace

int scatter_internal(dski_handle h, const void* vin, void* g, int s, bool prec64) {
  return scatter_internal_ws(h, vin, g, s, prec64, nullptr);
}

int scatter_internal_ws(dski_handle h, const void* vin, void* g, int s, bool prec64, void* ws) {
  return scatter_scaled(h, vin, g, s, prec64, ws, 1.0, 1.0);
}

int scatter_scaled(dski_handle h, const void* vin, void* g, int s, bool prec64, void* ws,
                   double sv, double sg, const CgUpdate* up) {
  return scatter_fused(h, vin, g, s, prec64, ws, sv, sg, nullptr, nullptr, up);
}

int scatter_fused(dski_handle h, const void* vin, void* g, int s, bool prec64, void* ws,
                  double sv, double sg, const double* z, const double* beta, const CgUpdate* up) {
  const CgUpdate upd = up ? *up : CgUpdate{};
  const MvmGeo geo = make_geo(h);
  cudaStream_t st = h->stream;
  // FP32 vectors, d = 2: the per-cell two-pass scatter.  FP64 keeps the
  // point-parallel prep + node pass below: on GB300 one warp-wide FP64
  // instruction holds an SM sub-partition for ~64 cycles (ncu: FP64 pipe 83%
  // active), and with ~1.5 points per cell the per-cell groups issue ~7 FP64
  // warp instructions per point against ~1.4 there.
  if (up && !(prec64 && h->d >= 2 && s <= 4))
    return set_error(DSKI_ERR_ARG, "fused CG update needs FP64, d >= 2 and s <= 4");
  if (cells_path(h, prec64)) {
    if (z || sv != 1.0 || sg != 1.0)
      return set_error(DSKI_ERR_ARG, "scaled / fused scatter needs FP64 vectors");
    void* S = ws;
    if (!S) {
      if (h->scat_ab.ensure(scatter_ws_bytes(h, s, prec64)))
        return set_error(DSKI_ERR_ALLOC, "scatter workspace allocation failed");
      S = h->scat_ab.ptr;
    }
    StageScope sc(h, ST_SCATTER, st, 2);
    if (s == 1)
      scatter_cells_d2<float, 1>(h, (float*)vin, (float*)S, (float*)g, s, 1.f, 1.f, nullptr,
                                 nullptr, st);
    else   // two columns per pass: 16 x 4 accumulators capped occupancy at 2 blocks per SM
      scatter_cells_d2<float, 2>(h, (float*)vin, (float*)S, (float*)g, s, 1.f, 1.f, nullptr,
                                 nullptr, st);
    DSKI_LAUNCHED();
    return DSKI_OK;
  }
  if (df_scatter_path(h, prec64)) {
    if (up && s > 4) return set_error(DSKI_ERR_ARG, "fused CG update needs s <= 4");
    float2* S = static_cast<float2*>(ws);
    if (!S) {
      if (h->scat_ab.ensure(scatter_ws_bytes(h, s, prec64)))
        return set_error(DSKI_ERR_ALLOC, "scatter workspace allocation failed");
      S = h->scat_ab.as<float2>();
    }
    const int ncell = h->mc[0] * h->mc[1];
    float2* Vdf = S + (size_t)s * 16 * ncell;   // s x n x 3 pairs after the cell planes
    const int G = df_group(h);
    const float2* W = h->Wdf.as<float2>();
    const int* cs = h->cell_start.as<int>();
    StageScope sc(h, ST_SCATTER, st, 3);
    auto pair = [](double x) {
      const float hi = (float)x;
      return make_float2(hi, (float)(x - (double)hi));
    };
    k_scatter_split_df<<<dim3((unsigned)((h->n + 255) / 256), (unsigned)s), 256, 0, st>>>(
        (double*)vin, Vdf, h->n, h->N, sv != 1.0 || sg != 1.0, pair(sv), pair(sg), z, beta, upd);
    const dim3 gc((unsigned)(((long long)ncell * G + 255) / 256), (unsigned)s);
    switch (G) {
      case 2: k_scatter_cells_df<2><<<gc, 256, 0, st>>>(cs, W, Vdf, h->n, S, ncell); break;
      case 4: k_scatter_cells_df<4><<<gc, 256, 0, st>>>(cs, W, Vdf, h->n, S, ncell); break;
      case 8: k_scatter_cells_df<8><<<gc, 256, 0, st>>>(cs, W, Vdf, h->n, S, ncell); break;
      case 16: k_scatter_cells_df<16><<<gc, 256, 0, st>>>(cs, W, Vdf, h->n, S, ncell); break;
      default: k_scatter_cells_df<32><<<gc, 256, 0, st>>>(cs, W, Vdf, h->n, S, ncell); break;
    }
    const dim3 gn((unsigned)((h->M + 255) / 256), (unsigned)s);
    k_scatter_nodes_df<<<gn, 256, 0, st>>>(geo, S, (double*)g, h->M, ncell);
    DSKI_LAUNCHED();
    return DSKI_OK;
  }
  if (prec64 && h->d >= 2 && s <= 4) {
    double* ab = static_cast<double*>(ws);
    if (!ab) {
      if (h->scat_ab.ensure(scatter_ws_bytes(h, s, prec64)))
        return set_error(DSKI_ERR_ALLOC, "scatter workspace allocation failed");
      ab = h->scat_ab.as<double>();
    }
    const double* wt = h->W64.as<double>();
    const dim3 gp((unsigned)((h->n + 255) / 256));
    StageScope sc(h, ST_SCATTER, st, 2);
    with_stencil(h, [&](auto Sc) {
      constexpr int S = decltype(Sc)::value;
      const dim3 gs((unsigned)((h->M * scatter_split(2, S) + 255) / 256), 1);
      if (h->d == 2) {
        k_scatter_prep<2, S><<<gp, 256, 0, st>>>(wt, (double*)vin, s, h->n, h->N, sv, sg, z,
                                                 beta, ab, upd);
        if (s == 1)
          k_scatter_ab<2, 1, S><<<gs, 256, 0, st>>>(geo, h->cell_start.as<int>(),
                                                    h->cell.as<int>(), wt, ab, (double*)g, s,
                                                    h->n, h->M);
        else
          k_scatter_ab<2, 4, S><<<gs, 256, 0, st>>>(geo, h->cell_start.as<int>(),
                                                    h->cell.as<int>(), wt, ab, (double*)g, s,
                                                    h->n, h->M);
      } else {
        k_scatter_prep<3, S><<<gp, 256, 0, st>>>(wt, (double*)vin, s, h->n, h->N, sv, sg, z,
                                                 beta, ab, upd);
        if (s == 1)
          k_scatter_ab<3, 1, S><<<gs, 256, 0, st>>>(geo, h->cell_start.as<int>(),
                                                    h->cell.as<int>(), wt, ab, (double*)g, s,
                                                    h->n, h->M);
        else
          k_scatter_ab<3, 4, S><<<gs, 256, 0, st>>>(geo, h->cell_start.as<int>(),
                                                    h->cell.as<int>(), wt, ab, (double*)g, s,
                                                    h->n, h->M);
      }
    });
    DSKI_LAUNCHED();
    return DSKI_OK;
  }
  if (sv != 1.0 || sg != 1.0 || z)
    return set_error(DSKI_ERR_ARG, "scaled / fused scatter needs FP64, d >= 2 and s <= 4");
  if (prec64) {
    const double* fr = h->W64.as<double>();
    switch (h->d) {
      case 1: scatter_dispatch<double, 1>(h, geo, fr, (const double*)vin, (double*)g, s, st); break;
      case 2: scatter_dispatch<double, 2>(h, geo, fr, (const double*)vin, (double*)g, s, st); break;
      default: scatter_dispatch<double, 3>(h, geo, fr, (const double*)vin, (double*)g, s, st); break;
    }
  } else {
    const float* fr = h->W32.as<float>();
    switch (h->d) {
      case 1: scatter_dispatch<float, 1>(h, geo, fr, (const float*)vin, (float*)g, s, st); break;
      case 2: scatter_dispatch<float, 2>(h, geo, fr, (const float*)vin, (float*)g, s, st); break;
      default: scatter_dispatch<float, 3>(h, geo, fr, (const float*)vin, (float*)g, s, st); break;
    }
  }
  DSKI_LAUNCHED();
  return DSKI_OK;
}

// d mode products g -> result (ping-pong between g and tmp).  Factor k is
// K_k, except k == dfactor which uses dK (same precision as the path).
int kron_internal(dski_handle h, void* g, void* tmp, int s, bool prec64, int dfactor,
                  const void* dK, void** result, void* tc_ws) {
  cudaStream_t st = h->stream;
  void* cur = g;
  void* nxt = tmp;
  for (int t = 0; t < h->d; ++t) {
    const int k = h->d - 1 - t;
    const long long R = h->M / h->m[k];
    const bool last = t == h->d - 1;
    const double scale = last ? h->sf * h->sf : 1.0;
    // FP64_TC: the tensor-core product from m_k = 64 on; below, its fixed
    // per-CTA latency (~10 us) exceeds the FP64 product (~8 us at m_k = 24)
    if (prec64 && h->kuu_fft && dfactor < 0 && !h->kron_exact) {
      // Toeplitz factor by circulant embedding and FFT (all FP64); the PCG's
      // true residuals take the dense factors (kron_exact), so its restarts
      // refine x against the dense operator
      DSKI_TRY(mode_fft(h, k, (const double*)cur, (double*)nxt, R, s, scale));
    } else if (prec64 && h->prec == DSKI_FP64_TC && dfactor < 0 && !h->kron_exact &&
               h->m[k] >= kOzMinM) {
      DSKI_TRY(mode_tc_oz(h, (const double*)cur, h->Kdig[k].as<uint16_t>(), h->Kexp[k].as<int>(),
                          (double*)nxt, h->m[k], R, s, scale));
    } else if (prec64) {
      const double* K = k == dfactor ? (const double*)dK : h->K64[k].as<double>();
      mode_simt<double>(h, (const double*)cur, K, (double*)nxt, h->m[k], R, s, scale, h->sm_count,
                        st);
    } else if (dfactor < 0) {
      // mixed modes: tensor cores, TF32 or 3xTF32
      DSKI_TRY(mode_tc_tf32(h, (const float*)cur, h->Khi[k].as<float>(), h->Klo[k].as<float>(),
                            (float*)nxt, h->m[k], R, s, (float)scale,
                            h->prec == DSKI_MIXED_3XTF32, static_cast<float*>(tc_ws)));
    } else {
      const float* K = k == dfactor ? (const float*)dK : h->K32[k].as<float>();
      mode_simt<float>(h, (const float*)cur, K, (float*)nxt, h->m[k], R, s, (float)scale,
                       h->sm_count, st);
    }
    DSKI_LAUNCHED();
    std::swap(cur, nxt);
  }
  *result = cur;
  return DSKI_OK;
}

int mvm_internal(dski_handle h, const void* vin, void* vout, int s, bool prec64) {
  const size_t es = prec64 ? 8 : 4;
  const size_t gbytes = (size_t)h->M * s * es;
  if (h->gridA.ensure(gbytes) || h->gridB.ensure(gbytes))
    return set_error(DSKI_ERR_ALLOC, "grid workspace allocation failed (%zu bytes)", gbytes);
  DSKI_TRY(scatter_internal(h, vin, h->gridA.ptr, s, prec64));
  void* res = nullptr;
  DSKI_TRY(kron_internal(h, h->gridA.ptr, h->gridB.ptr, s, prec64, -1, nullptr, &res));
  const MvmGeo geo = make_geo(h);
  cudaStream_t st = h->stream;
  if (prec64) {
    const double* fr = h->W64.as<double>();
    switch (h->d) {
      case 1: gather_dispatch<double, 1>(h, geo, fr, (const double*)res, (const double*)vin, (double*)vout, s, st); break;
      case 2: gather_dispatch<double, 2>(h, geo, fr, (const double*)res, (const double*)vin, (double*)vout, s, st); break;
      default: gather_dispatch<double, 3>(h, geo, fr, (const double*)res, (const double*)vin, (double*)vout, s, st); break;
    }
  } else {
    const float* fr = h->W32.as<float>();
    switch (h->d) {
      case 1: gather_dispatch<float, 1>(h, geo, fr, (const float*)res, (const float*)vin, (float*)vout, s, st); break;
      case 2: gather_dispatch<float, 2>(h, geo, fr, (const float*)res, (const float*)vin, (float*)vout, s, st); break;
      default: gather_dispatch<float, 3>(h, geo, fr, (const float*)res, (const float*)vin, (float*)vout, s, st); break;
    }
  }
  DSKI_LAUNCHED();
  return DSKI_OK;
}

int gather_scaled(dski_handle h, const double* grid, const double* vin, double* vout, int s,
                  double av, double ag, double nv, double ng, int stage, double* dpart,
                  const CgFinish* fin, bool grid_scratch) {
  if (fin && fin->kind >= 0 && !dpart)
    return set_error(DSKI_ERR_ARG, "a folded CG finisher needs the gather's partial sums");
  const MvmGeo geo = make_geo(h);
  GatherScale gs;
  gs.av = av;
  gs.ag = ag;
  gs.nv = nv;
  gs.ng = ng;
  gs.stage = stage;
  gs.dpart = dpart;
  if (fin) gs.fin = *fin;
  gs.grid_scratch = grid_scratch;
  const double* fr = h->W64.as<double>();
  switch (h->d) {
    case 1: gather_dispatch<double, 1>(h, geo, fr, grid, vin, vout, s, h->stream, &gs); break;
    case 2: gather_dispatch<double, 2>(h, geo, fr, grid, vin, vout, s, h->stream, &gs); break;
    default: gather_dispatch<double, 3>(h, geo, fr, grid, vin, vout, s, h->stream, &gs); break;
  }
  DSKI_LAUNCHED();
  return DSKI_OK;
}

int gather_internal(dski_handle h, const void* grid, const void* vin, void* vout, int s,
                    bool prec64) {
  const MvmGeo geo = make_geo(h);
  cudaStream_t st = h->stream;
  if (prec64) {
    const double* fr = h->W64.as<double>();
    switch (h->d) {
      case 1: gather_dispatch<double, 1>(h, geo, fr, (const double*)grid, (const double*)vin, (double*)vout, s, st); break;
      case 2: gather_dispatch<double, 2>(h, geo, fr, (const double*)grid, (const double*)vin, (double*)vout, s, st); break;
      default: gather_dispatch<double, 3>(h, geo, fr, (const double*)grid, (const double*)vin, (double*)vout, s, st); break;
    }
  } else {
    const float* fr = h->W32.as<float>();
    switch (h->d) {
      case 1: gather_dispatch<float, 1>(h, geo, fr, (const float*)grid, (const float*)vin, (float*)vout, s, st); break;
      case 2: gather_dispatch<float, 2>(h, geo, fr, (const float*)grid, (const float*)vin, (float*)vout, s, st); break;
      default: gather_dispatch<float, 3>(h, geo, fr, (const float*)grid, (const float*)vin, (float*)vout, s, st); break;
    }
  }
  DSKI_LAUNCHED();
  return DSKI_OK;
}

bool pcg_fusable(dski_handle h, int s) { return f64_vectors(h) && h->d >= 2 && s <= 4; }

int mvm_pcg_fused(dski_handle h, double* P, const double* Z, const double* beta, double* Q,
                  int s, double* dpart, const CgFinish* fin) {
  const size_t gbytes = (size_t)h->M * s * 8;
  if (h->gridA.ensure(gbytes) || h->gridB.ensure(gbytes))
    return set_error(DSKI_ERR_ALLOC, "grid workspace allocation failed (%zu bytes)", gbytes);
  DSKI_TRY(scatter_fused(h, P, h->gridA.ptr, s, true, nullptr, 1.0, 1.0, Z, beta, nullptr));
  void* res = nullptr;
  DSKI_TRY(kron_internal(h, h->gridA.ptr, h->gridB.ptr, s, true, -1, nullptr, &res));
  if (!dpart) return gather_internal(h, res, P, Q, s, true);
  // the gather also leaves per-block partial sums of p^T q
  // (the product grid is this call's scratch)
  return gather_scaled(h, (const double*)res, P, Q, s, 1.0, 1.0, h->nv, h->ng, ST_GATHER, dpart,
                       fin, true);
}

int permute_in(dski_handle h, const void* v_user, void* v_int, int s, bool f64, cudaStream_t st) {
  const unsigned nb = (unsigned)((h->n + 255) / 256);
  StageScope sc(h, ST_PERMUTE, st);
  if (f64)
    k_perm_in<double><<<nb, 256, 0, st>>>(h->perm.as<int>(), (const double*)v_user,
                                          (double*)v_int, h->n, h->d, h->N, s);
  else
    k_perm_in<float><<<nb, 256, 0, st>>>(h->perm.as<int>(), (const float*)v_user, (float*)v_int,
                                         h->n, h->d, h->N, s);
  DSKI_LAUNCHED();
  return DSKI_OK;
}

int permute_out(dski_handle h, const void* v_int, void* v_user, int s, bool f64,
                cudaStream_t st) {
  const unsigned nb = (unsigned)((h->n + 255) / 256);
  StageScope sc(h, ST_PERMUTE, st);
  if (f64)
    k_perm_out<double><<<nb, 256, 0, st>>>(h->perm.as<int>(), (const double*)v_int,
                                           (double*)v_user, h->n, h->d, h->N, s);
  else
    k_perm_out<float><<<nb, 256, 0, st>>>(h->perm.as<int>(), (const float*)v_int,
                                          (float*)v_user, h->n, h->d, h->N, s);
  DSKI_LAUNCHED();
  return DSKI_OK;
}

}  // namespace dski
