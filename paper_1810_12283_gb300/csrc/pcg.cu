// Batched preconditioned conjugate gradients (Sec. 2 "conjugate gradients",
// Sec. 3.3 preconditioning), stochastic Lanczos quadrature for log|K~|
// (Sec. 2) and the gradient of the log marginal likelihood (Eq. 1).
//
// One PCG runs s columns at once on the internal layout.  Per iteration:
//   q = K~ p                         (D-SKI MVM: scatter, mode products, gather)
//   alpha = r^T z / p^T q            (fused column dot + scalar update)
//   x += alpha p,  r -= alpha q      (fused, with ||r||^2)
//   z = M^-1 r                       (QR-form apply: C = Q1^T D^-1/2 r, then
//                                     z = D^-1/2 (D^-1/2 r - Q1 C), fused r^T z)
//   beta = r'^T z' / r^T z,  p = z + beta p
// Scalars (alpha, beta, r^T z, norms) stay on the device in FP64; the host
// reads one "columns still active" count per chunk of iterations.  When the
// recursive residual of every column meets the tolerance, the true residual
// b - K~ x is recomputed with the FP64 operator and the columns that miss the
// tolerance restart from it (p = M^-1 r).  Continuing with the old search
// direction instead (residual replacement) stalled near the attainable
// accuracy on the 800-point sine workload, while restarting converged.  In
// the mixed modes the MVM of the inner
// iteration runs in FP32 / (3x)TF32 on a float copy of p while x, r, z and
// every scalar stay FP64; the inner solve then targets a reduction of 1e-4
// of the residual it restarted from, and the FP64 true residual refines x.
// In FP64_TC the inner MVM takes the tensor-core mode products and the true
// residual the FP64-unit ones.
//
// The first `depth` alpha_j, beta_j of each column are recorded: CG on
// K~ x = z with preconditioner M is the Lanczos process on
// M^-1/2 K~ M^-1/2, whose tridiagonal T has
//   T[j][j]   = 1/alpha_j + beta_{j-1}/alpha_{j-1},
//   T[j][j+1] = sqrt(beta_j)/alpha_j
// (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed., Sec. 6.7.3).
#include <algorithm>
#include <cmath>
#include <vector>

#include "solve_internal.cuh"

namespace dski {
namespace {

constexpr int CG_THREADS = 256;
constexpr int CG_UNROLL = 4;   // elements per thread and step in the streaming kernels

__device__ __forceinline__ bool cg_last(unsigned* ticket) {
  return last_block(ticket, gridDim.x * gridDim.y);
}

// r = b - q, y = dis .* r; ||b||^2 (first call) and ||r||^2; (re)activates
// the columns whose residual misses the target.
__global__ void __launch_bounds__(CG_THREADS) k_cg_init(
    const double* __restrict__ b, const double* __restrict__ q, double* __restrict__ r,
    double* __restrict__ y, const double* __restrict__ dis, long long N, int first, double tol2,
    double eta2, ColState cs, double* part, unsigned* ticket) {
  __shared__ double sh[32];
  const int c = blockIdx.y;
  double sb = 0.0, sr = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long o = (long long)c * N + i;
    const double bi = b[o];
    const double ri = bi - q[o];
    r[o] = ri;
    if (y) y[o] = dis[i] * ri;
    sb = fma(bi, bi, sb);
    sr = fma(ri, ri, sr);
  }
  sb = block_sum(sb, sh);
  __syncthreads();
  sr = block_sum(sr, sh);
  if (threadIdx.x == 0) {
    part[2 * ((long long)c * gridDim.x + blockIdx.x)] = sb;
    part[2 * ((long long)c * gridDim.x + blockIdx.x) + 1] = sr;
  }
  if (cg_last(ticket)) {
    __shared__ double totb[CG_MAXS], totr[CG_MAXS];
    sum_columns(part, gridDim.x, cs.s, 2, 0, totb, sh);
    sum_columns(part, gridDim.x, cs.s, 2, 1, totr, sh);
    int nact = 0;
    for (int cc = threadIdx.x; cc < cs.s; cc += blockDim.x) {
      const double tb = totb[cc], tr = totr[cc];
      if (first) cs.bn2[cc] = tb;
      cs.rn2[cc] = tr;
      const double goal = fmax(tol2 * cs.bn2[cc], eta2 * tr);
      cs.target[cc] = goal;
      const int act = (!cs.bd[cc] && tr > tol2 * cs.bn2[cc] && isfinite(tr)) ? 1 : 0;
      cs.active[cc] = act;
      nact += act;
    }
    nact = (int)block_sum((double)nact, sh);
    if (threadIdx.x == 0) *cs.nactive = nact;
  }
}

// z = dis .* (y - Q1 C) (preconditioned) or z = r (plain); r^T z.
// init: p = z (and its float copy), r^T z becomes rz and rz0.
// else: beta = (r^T z)_new / rz for active columns, recorded.
// SPLIT: Q1 = Qh + Ql in FP32 halves, the product taken in double-float.
// ZIN: z given (computed by the grid-form apply); only the dots/updates run.
template <bool SPLIT>
__global__ void __launch_bounds__(CG_THREADS) k_cg_z(
    const double* __restrict__ r, const double* __restrict__ y, const double* __restrict__ Q1,
    const float* __restrict__ Qh, const float* __restrict__ Ql, const double* __restrict__ zin,
    int rank, const double* __restrict__ C, const double* __restrict__ dis,
    double* __restrict__ z, double* __restrict__ p, float* __restrict__ p32, long long N,
    int init, ColState cs, double* part, unsigned* ticket) {
  extern __shared__ double Cs[];   // rank values of column c (SPLIT: 2 rank floats)
  __shared__ double sh[32];
  const int c = blockIdx.y;
  float* Cf = reinterpret_cast<float*>(Cs);
  for (int t = threadIdx.x; t < rank; t += blockDim.x) {
    if (SPLIT) split_d(C[(long long)t * cs.s + c], Cf[t], Cf[rank + t]);
    else Cs[t] = C[(long long)t * cs.s + c];
  }
  __syncthreads();
  double acc = 0.0;
#pragma unroll 4
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long o = (long long)c * N + i;
    double zi;
    if (zin) {
      zi = zin[o];
    } else if (y) {
      double v = y[o];
      // Q1 columns in groups of 8: the group's loads are issued together so
      // that each thread keeps 8 (16) independent loads in flight
      if (SPLIT && rank) {
        float s_h = 0.f, s_l = 0.f;
        for (int t0 = 0; t0 < rank; t0 += 8) {
          float qh[8], ql[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const bool in = t0 + k < rank;
            qh[k] = in ? Qh[(long long)(t0 + k) * N + i] : 0.f;
            ql[k] = in ? Ql[(long long)(t0 + k) * N + i] : 0.f;
          }
#pragma unroll
          for (int k = 0; k < 8; ++k)
            if (t0 + k < rank) df_fma(qh[k], ql[k], Cf[t0 + k], Cf[rank + t0 + k], s_h, s_l);
        }
        v = (v - (double)s_h) - (double)s_l;
      } else if (Q1) {
        for (int t0 = 0; t0 < rank; t0 += 8) {
          double q[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) q[k] = t0 + k < rank ? Q1[(long long)(t0 + k) * N + i] : 0.0;
#pragma unroll
          for (int k = 0; k < 8; ++k)
            if (t0 + k < rank) v = fma(-q[k], Cs[t0 + k], v);
        }
      }
      zi = dis[i] * v;
    } else {
      zi = r[o];
    }
    acc = fma(r[o], zi, acc);
    // z is kept also at a (re)start: the fused MVM forms p = z + beta p from it
    if (!zin) z[o] = zi;
    if (init) {
      p[o] = zi;
      if (p32) p32[o] = (float)zi;
    }
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[(long long)c * gridDim.x + blockIdx.x] = acc;
  if (cg_last(ticket)) {
    __shared__ double tot[CG_MAXS];
    sum_columns(part, gridDim.x, cs.s, 1, 0, tot, sh);
    beta_finish(tot, cs, init);
  }
}

// C[t][c] from per-group blocks: group g = c / 4 holds rank x q_g row-major.
__global__ void k_regroup(const double* __restrict__ Cg, int rank, int s, double* __restrict__ C) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rank * s) return;
  const int t = idx / s, c = idx % s;
  const int g = c / 4, cc = c % 4;
  const int q = min(4, s - 4 * g);
  C[idx] = Cg[(long long)4 * g * rank + (long long)t * q + cc];
}

__global__ void __launch_bounds__(CG_THREADS) k_cg_p(const double* __restrict__ z,
                                                     double* __restrict__ p,
                                                     float* __restrict__ p32, long long N,
                                                     ColState cs) {
  const int c = blockIdx.y;
  if (!cs.active[c]) return;
  const double be = cs.beta[c];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long o = (long long)c * N + i;
    const double v = fma(be, p[o], z[o]);
    p[o] = v;
    if (p32) p32[o] = (float)v;
  }
}

// p^T q and alpha = r^T z / p^T q (zero for finished columns).
template <class TQ>
__global__ void __launch_bounds__(CG_THREADS) k_cg_alpha(const double* __restrict__ p,
                                                         const TQ* __restrict__ q, long long N,
                                                         ColState cs, double* part,
                                                         unsigned* ticket) {
  __shared__ double sh[32];
  const int c = blockIdx.y;
  double acc = 0.0;
  if (cs.active[c]) {
    const long long st = (long long)gridDim.x * blockDim.x;
    const double* pc = p + (long long)c * N;
    const TQ* qc = q + (long long)c * N;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    // CG_UNROLL independent elements per thread and step: all loads in flight
    for (; i + (CG_UNROLL - 1) * st < N; i += CG_UNROLL * st) {
      double pv[CG_UNROLL], qv[CG_UNROLL];
#pragma unroll
      for (int u = 0; u < CG_UNROLL; ++u) {
        pv[u] = pc[i + u * st];
        qv[u] = (double)qc[i + u * st];
      }
#pragma unroll
      for (int u = 0; u < CG_UNROLL; ++u) acc = fma(pv[u], qv[u], acc);
    }
    for (; i < N; i += st) acc = fma(pc[i], (double)qc[i], acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[(long long)c * gridDim.x + blockIdx.x] = acc;
  if (cg_last(ticket)) {
    __shared__ double tot[CG_MAXS];
    sum_columns(part, gridDim.x, cs.s, 1, 0, tot, sh);
    alpha_finish(tot, cs);
  }
}

// x += alpha p; r -= alpha q; y = dis .* r; ||r||^2; convergence.
template <class TQ>
__global__ void __launch_bounds__(CG_THREADS) k_cg_update(
    double* __restrict__ x, double* __restrict__ r, double* __restrict__ y,
    const double* __restrict__ p, const TQ* __restrict__ q, const double* __restrict__ dis,
    long long N, ColState cs, double* part, unsigned* ticket) {
  __shared__ double sh[32];
  const int c = blockIdx.y;
  const double al = cs.alpha[c];
  double acc = 0.0;
  if (cs.active[c]) {
    const long long st = (long long)gridDim.x * blockDim.x;
    const long long off = (long long)c * N;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (CG_UNROLL - 1) * st < N; i += CG_UNROLL * st) {
      double xv[CG_UNROLL], pv[CG_UNROLL], qv[CG_UNROLL], rv[CG_UNROLL], dv[CG_UNROLL];
#pragma unroll
      for (int u = 0; u < CG_UNROLL; ++u) {
        const long long o = off + i + u * st;
        xv[u] = x[o];
        pv[u] = p[o];
        qv[u] = (double)q[o];
        rv[u] = r[o];
        dv[u] = y ? dis[i + u * st] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < CG_UNROLL; ++u) {
        const long long o = off + i + u * st;
        x[o] = fma(al, pv[u], xv[u]);
        const double ri = fma(-al, qv[u], rv[u]);
        r[o] = ri;
        if (y) y[o] = dv[u] * ri;
        acc = fma(ri, ri, acc);
      }
    }
    for (; i < N; i += st) {
      const long long o = off + i;
      x[o] = fma(al, p[o], x[o]);
      const double ri = fma(-al, (double)q[o], r[o]);
      r[o] = ri;
      if (y) y[o] = dis[i] * ri;
      acc = fma(ri, ri, acc);
    }
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[(long long)c * gridDim.x + blockIdx.x] = acc;
  if (cg_last(ticket)) {
    __shared__ double tot[CG_MAXS];
    sum_columns(part, gridDim.x, cs.s, 1, 0, tot, sh);
    update_finish(tot, cs, sh);
  }
}

}  // namespace

// ----------------------------------------------------------------- engine --


int cg_run(dski_handle h, CgRun& run) {
  const long long N = h->N;
  const int s = run.s;
  if (s < 1 || s > CG_MAXS) return set_error(DSKI_ERR_ARG, "cg_run: %d columns (max %d)", s, CG_MAXS);
  const bool mixed = !f64_vectors(h);
  const int rank = run.pc ? run.pc->rank : 0;
  cudaStream_t st = h->stream;
  const size_t Ns = (size_t)N * s;
  double* R = wbuf(h->s_vec[0], Ns);
  double* Z = wbuf(h->s_vec[1], Ns);
  double* P = wbuf(h->s_vec[2], Ns);
  double* Q = wbuf(h->s_vec[3], Ns);
  double* Y = run.pc ? wbuf(h->s_vec[4], Ns) : nullptr;
  double* C = rank ? wbuf(h->s_vec[5], (size_t)rank * s) : nullptr;
  // split-preconditioner results per group of <= 4 columns (c0 rank x q blocks)
  double* Cg = rank ? wbuf(h->s_vec[10], (size_t)rank * (s + 4)) : nullptr;
  float* P32 = mixed ? (float*)wbuf(h->s_vec[6], (Ns + 1) / 2) : nullptr;
  float* Q32 = mixed ? (float*)wbuf(h->s_vec[7], (Ns + 1) / 2) : nullptr;
  const int depth = run.depth;
  const size_t nstate = 8 * (size_t)s + 2 * (size_t)depth * s + 8;
  double* stbuf = wbuf(h->s_state, nstate + 6 * (size_t)s + 8);
  // one row per thread where the grid allows (memory-level parallelism),
  // at most 16 blocks per SM over all columns
  const int nbx = (int)std::min<long long>((N + CG_THREADS - 1) / CG_THREADS,
                                           std::max(1, 16 * h->sm_count / std::max(1, s)));
  // the streaming kernels (dots, updates): ~2 blocks per SM over all columns,
  // CG_UNROLL elements per thread and step -- few blocks keep the
  // last-block reduction (one ticket atomic per block, a sum over the
  // blocks' partials) short
  const int nbv = (int)std::min<long long>(
      std::max<long long>(1, (N + (long long)CG_THREADS * CG_UNROLL - 1) / (CG_THREADS * CG_UNROLL)),
      std::max(1, 2 * h->sm_count / std::max(1, s)));
  double* part = wbuf(h->s_part, (size_t)nbx * s * 2 + 16);
  unsigned* tk = tickets(h, 1);
  if (!R || !Z || !P || !Q || (run.pc && !Y) || (rank && !C) || (mixed && (!P32 || !Q32)) ||
      !stbuf || !part || !tk)
    return set_error(DSKI_ERR_ALLOC, "dski_pcg_solve: workspace allocation failed");
  if (run.pc && !Y) return DSKI_ERR_ALLOC;
  ColState cs{};
  cs.s = s;
  cs.depth = depth;
  cs.bn2 = stbuf;
  cs.rn2 = cs.bn2 + s;
  cs.rz = cs.rn2 + s;
  cs.rz0 = cs.rz + s;
  cs.alpha = cs.rz0 + s;
  cs.beta = cs.alpha + s;
  cs.target = cs.beta + s;
  cs.ahist = depth ? cs.target + s : nullptr;
  cs.bhist = depth ? cs.target + s + (size_t)depth * s : nullptr;
  int* ib = (int*)(cs.target + s + 2 * (size_t)depth * s + 1);
  cs.active = ib;
  cs.iters = ib + s;
  cs.bd = ib + 2 * s;
  cs.nactive = ib + 3 * s;
  if (cudaMemsetAsync(stbuf, 0, (nstate + 6 * (size_t)s + 8) * sizeof(double), st) != cudaSuccess)
    return set_error(DSKI_ERR_CUDA, "dski_pcg_solve: memset failed");
  const double tol2 = run.rtol * run.rtol;
  // inner reduction target (1e-4)^2 where the iterations run a perturbed
  // operator (mixed modes; FFT products, whose normwise rounding stalls the
  // recurrence on ill-conditioned systems): each pass then ends at a 1e-4
  // reduction and the restart from the dense true residual refines x.  Not
  // while Lanczos coefficients are recorded: the record covers the first
  // pass, which must then run the full depth.
  const double eta2 = (depth == 0 && (mixed || h->kuu_fft)) ? 1e-8 : 0.0;
  cs.soft = eta2 > 0.0 ? 1 : 0;
  const double* dis = run.pc ? run.pc->dis.as<double>() : nullptr;
  const dim3 grd(nbx, s);
  const dim3 grv(std::min(nbv, nbx), s);
  const size_t zsmem = (size_t)std::max(rank, 1) * sizeof(double);

  const bool split = run.pc && run.pc->split;
  const bool gridf = run.pc && run.pc->grid_form;
  const bool fused = !mixed && pcg_fusable(h, s);
  auto precond_z = [&](int init) -> int {
    if (gridf) {
      DSKI_TRY(grid_precond_apply(h, run.pc, R, Z, s));
      StageScope sc(h, ST_PCGVEC, st);
      k_cg_z<false><<<grv, CG_THREADS, zsmem, st>>>(R, nullptr, nullptr, nullptr, nullptr, Z, 0,
                                                   nullptr, nullptr, Z, P, P32, N, init, cs, part,
                                                   tk);
      DSKI_LAUNCHED();
      return DSKI_OK;
    }
    if (rank && split) {
      for (int c0 = 0; c0 < s; c0 += 4)
        DSKI_TRY(df_gemv_t(h, run.pc->Qh.as<float>(), run.pc->Ql.as<float>(), rank,
                           Y + (size_t)c0 * N, std::min(4, s - c0), nullptr, Cg + (size_t)c0 * rank));
      // gather the per-group results into C[t][c] (t-major, s columns)
      StageScope sc(h, ST_PRECOND, st);
      k_regroup<<<(rank * s + 255) / 256, 256, 0, st>>>(Cg, rank, s, C);
      DSKI_LAUNCHED();
    } else if (rank) {
      DSKI_TRY(ts_tn(h, run.pc->Q1.as<double>(), rank, Y, s, nullptr, C));
    }
    StageScope sc(h, ST_PRECOND, st);
    if (split)
      k_cg_z<true><<<grd, CG_THREADS, zsmem, st>>>(R, Y, nullptr, run.pc->Qh.as<float>(),
                                                  run.pc->Ql.as<float>(), nullptr, rank, C, dis, Z,
                                                  P, P32, N, init, cs, part, tk);
    else
      k_cg_z<false><<<grd, CG_THREADS, zsmem, st>>>(R, Y, rank ? run.pc->Q1.as<double>() : nullptr,
                                                   nullptr, nullptr, nullptr, rank, C, dis, Z, P,
                                                   P32, N, init, cs, part, tk);
    DSKI_LAUNCHED();
    return DSKI_OK;
  };
  auto true_residual = [&](int first) -> int {
    // FP64_TC and FFT products: the true residual takes the dense FP64-unit
    // mode products, so the restarts refine x against that operator
    h->kron_exact = true;
    const int mrc = mvm_internal(h, run.X, Q, s, true);
    h->kron_exact = false;
    DSKI_TRY(mrc);
    StageScope sc(h, ST_PCGVEC, st);
    k_cg_init<<<grv, CG_THREADS, 0, st>>>(run.B, Q, R, Y, dis, N, first, tol2, eta2, cs, part,
                                          tk);
    DSKI_LAUNCHED();
    return DSKI_OK;
  };
  auto read_nactive = [&](int* out) -> int {
    if (cudaMemcpyAsync(out, cs.nactive, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return set_error(DSKI_ERR_CUDA, "dski_pcg_solve: %s", cudaGetErrorString(cudaGetLastError()));
    return check_device_error(h);   // synchronises
  };
  // FP64 grid-form path: the three CG vector passes fold into the kernels
  // around them (p^T q into the MVM's gather, x += alpha p, r -= alpha q
  // and ||r||^2 into the preconditioner's scatter pass, r^T z into its
  // gather); one-block kernels finish the sums
  const bool fusedg = fused && gridf && s <= 4;
  // partial sums per column: the gathers write ceil(n / 256), the fused
  // scatter of the preconditioner scatter_update_blocks
  const int nbp = std::max((h->n + 255) / 256, scatter_update_blocks(h));
  double* dpA = fusedg ? wbuf(h->s_dpart, (size_t)3 * nbp * 4 + 16) : nullptr;
  if (fusedg && !dpA) return set_error(DSKI_ERR_ALLOC, "dski_pcg_solve: workspace allocation failed");
  double* dpU = fusedg ? dpA + (size_t)nbp * 4 : nullptr;
  double* dpZ = fusedg ? dpU + (size_t)nbp * 4 : nullptr;
  auto iteration = [&]() -> int {
    if (fusedg) {
      // alpha from p^T q in the last block of the MVM's gather
      CgFinish fa;
      fa.kind = 0;
      fa.cs = cs;
      fa.ticket = tk;
      DSKI_TRY(mvm_pcg_fused(h, P, Z, cs.beta, Q, s, dpA, &fa));
      CgUpdate up;
      up.x = run.X;
      up.p = P;
      up.q = Q;
      up.alpha = cs.alpha;
      up.active = cs.active;
      up.dpart = dpU;
      // the update's bookkeeping (||r||^2 from the scatter pass) and beta
      // (r^T z) in the last block of the preconditioner's gather
      CgFinish fb;
      fb.kind = 1;
      fb.cs = cs;
      fb.ticket = tk;
      fb.part2 = dpU;
      fb.nb2 = scatter_update_blocks(h);
      DSKI_TRY(grid_precond_apply(h, run.pc, R, Z, s, &up, dpZ, &fb));
      return DSKI_OK;
    }
    if (mixed) {
      DSKI_TRY(mvm_internal(h, P32, Q32, s, false));
      StageScope sc(h, ST_PCGVEC, st, 2);
      k_cg_alpha<float><<<grv, CG_THREADS, 0, st>>>(P, Q32, N, cs, part, tk);
      k_cg_update<float><<<grv, CG_THREADS, 0, st>>>(run.X, R, Y, P, Q32, dis, N, cs, part, tk);
    } else {
      // fused: the previous iteration's p = z + beta p happens in the MVM's
      // first pass (after an (re)start beta = 0 and p = z already)
      if (fused) DSKI_TRY(mvm_pcg_fused(h, P, Z, cs.beta, Q, s));
      else DSKI_TRY(mvm_internal(h, P, Q, s, true));
      StageScope sc(h, ST_PCGVEC, st, 2);
      k_cg_alpha<double><<<grv, CG_THREADS, 0, st>>>(P, Q, N, cs, part, tk);
      k_cg_update<double><<<grv, CG_THREADS, 0, st>>>(run.X, R, Y, P, Q, dis, N, cs, part, tk);
    }
    DSKI_LAUNCHED();
    DSKI_TRY(precond_z(0));
    if (!fused) {
      StageScope sc(h, ST_PCGVEC, st);
      k_cg_p<<<grd, CG_THREADS, 0, st>>>(Z, P, P32, N, cs);
      DSKI_LAUNCHED();
    }
    return DSKI_OK;
  };

  // A CUDA graph of one 16-iteration chunk, captured once the first chunk
  // has run (its launches allocate the workspaces and run the tile tuner)
  // and replayed for every later full chunk: the chunk's ~250 launches then
  // cost one.  Off while the stage timers record (their events) and while
  // Lanczos coefficients are recorded (the depth travels in the kernels'
  // arguments), and on a stream that cannot be captured.
  cudaGraphExec_t gexec = nullptr;
  long long glaunches = 0;
  bool gtried = false;
  int chunks_run = 0;
  struct GraphGuard {
    cudaGraphExec_t* g;
    ~GraphGuard() {
      if (*g) cudaGraphExecDestroy(*g);
    }
  } gguard{&gexec};
  auto run_chunk = [&](int chunk) -> int {
    const bool can = chunk == 16 && depth == 0 && chunks_run >= 1 && !profiling_on(h) &&
                     st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
    if (can && !gexec && !gtried) {
      gtried = true;
      const long long l0 = launches_so_far();
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        int rc = DSKI_OK;
        for (int k = 0; k < chunk && rc == DSKI_OK; ++k) rc = iteration();
        const cudaError_t ce = cudaStreamEndCapture(st, &g);
        const long long captured = launches_so_far() - l0;
        count_launches((int)-captured);   // recorded into the graph, not run
        if (rc == DSKI_OK && ce == cudaSuccess && g &&
            cudaGraphInstantiate(&gexec, g, 0) == cudaSuccess)
          glaunches = captured;
        else
          gexec = nullptr;
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        clear_error();
      } else {
        cudaGetLastError();
      }
    }
    ++chunks_run;
    if (gexec && chunk == 16) {   // the graph holds exactly one full chunk
      if (cudaGraphLaunch(gexec, st) != cudaSuccess)
        return set_error(DSKI_ERR_CUDA, "dski_pcg_solve: graph launch: %s",
                         cudaGetErrorString(cudaGetLastError()));
      count_launches((int)glaunches);
      return DSKI_OK;
    }
    for (int k = 0; k < chunk; ++k) DSKI_TRY(iteration());
    return DSKI_OK;
  };

  int its = 0, restarts = 0, nact = 0;
  const int max_restarts = mixed ? 200 : 64;
  // Passes on a perturbed operator (cs.soft): refinement from the FP64 true
  // residual converges only while the operator's error stays below the
  // system's smallest eigenvalue.  The x of the smallest true residual is
  // kept, and the solve stops once three passes in a row have not improved
  // on it; x is then restored to that iterate.
  double* Xbest = cs.soft ? wbuf(h->s_vec[12], Ns) : nullptr;
  if (cs.soft && !Xbest) return set_error(DSKI_ERR_ALLOC, "dski_pcg_solve: workspace allocation failed");
  std::vector<double> best_rn2(s, HUGE_VAL), cur_rn2(s), bn2(s);
  std::vector<int> stale(s, 0);
  bool diverged = false;
  auto track_best = [&](bool first) -> int {   // after a true residual (stream synchronised)
    if (!cs.soft) return DSKI_OK;
    if ((first && cudaMemcpy(bn2.data(), cs.bn2, s * 8, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        cudaMemcpy(cur_rn2.data(), cs.rn2, s * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return set_error(DSKI_ERR_CUDA, "dski_pcg_solve: %s", cudaGetErrorString(cudaGetLastError()));
    bool stop = true;
    for (int c = 0; c < s; ++c) {
      if (cur_rn2[c] < best_rn2[c]) {
        best_rn2[c] = cur_rn2[c];
        stale[c] = 0;
        if (cudaMemcpyAsync(Xbest + (size_t)c * N, run.X + (size_t)c * N, (size_t)N * 8,
                            cudaMemcpyDeviceToDevice, st) != cudaSuccess)
          return set_error(DSKI_ERR_CUDA, "dski_pcg_solve: copy failed");
      } else {
        ++stale[c];
      }
      const bool done = cur_rn2[c] <= tol2 * bn2[c];
      if (!done && stale[c] < 3) stop = false;
    }
    if (stop && !first) {
      // restore the best iterate of every column that has moved away from it
      for (int c = 0; c < s; ++c)
        if (cur_rn2[c] > best_rn2[c] &&
            cudaMemcpyAsync(run.X + (size_t)c * N, Xbest + (size_t)c * N, (size_t)N * 8,
                            cudaMemcpyDeviceToDevice, st) != cudaSuccess)
          return set_error(DSKI_ERR_CUDA, "dski_pcg_solve: copy failed");
      diverged = true;
    }
    return DSKI_OK;
  };
  DSKI_TRY(true_residual(1));
  DSKI_TRY(read_nactive(&nact));
  DSKI_TRY(track_best(true));
  while (nact > 0) {
    DSKI_TRY(precond_z(1));   // p = M^-1 r
    while (its < run.maxit) {
      const int chunk = std::min(16, run.maxit - its);
      DSKI_TRY(run_chunk(chunk));
      its += chunk;
      DSKI_TRY(read_nactive(&nact));
      if (nact == 0) break;
    }
    DSKI_TRY(true_residual(0));
    DSKI_TRY(read_nactive(&nact));
    DSKI_TRY(track_best(false));
    if (diverged) {
      // the restored iterates' true residuals, for the results below
      DSKI_TRY(true_residual(0));
      DSKI_TRY(read_nactive(&nact));
      break;
    }
    if (nact == 0 || its >= run.maxit || restarts >= max_restarts) break;
    ++restarts;
    cs.depth = 0;   // the Lanczos record covers the first pass only
  }
  // results
  std::vector<double> hb(s), hr(s);
  std::vector<int> hi(s), hbd(s);
  run.rz0.resize(s);
  if (cudaMemcpyAsync(hb.data(), cs.bn2, s * 8, cudaMemcpyDeviceToHost, st) ||
      cudaMemcpyAsync(hr.data(), cs.rn2, s * 8, cudaMemcpyDeviceToHost, st) ||
      cudaMemcpyAsync(run.rz0.data(), cs.rz0, s * 8, cudaMemcpyDeviceToHost, st) ||
      cudaMemcpyAsync(hi.data(), cs.iters, s * 4, cudaMemcpyDeviceToHost, st) ||
      cudaMemcpyAsync(hbd.data(), cs.bd, s * 4, cudaMemcpyDeviceToHost, st))
    return set_error(DSKI_ERR_CUDA, "dski_pcg_solve: result copy failed");
  cs.ahist = depth ? cs.target + s : nullptr;
  cs.bhist = depth ? cs.target + s + (size_t)depth * s : nullptr;
  if (depth) {
    run.ahist.resize((size_t)depth * s);
    run.bhist.resize((size_t)depth * s);
    if (cudaMemcpyAsync(run.ahist.data(), cs.ahist, (size_t)depth * s * 8, cudaMemcpyDeviceToHost,
                        st) ||
        cudaMemcpyAsync(run.bhist.data(), cs.bhist, (size_t)depth * s * 8, cudaMemcpyDeviceToHost,
                        st))
      return set_error(DSKI_ERR_CUDA, "dski_pcg_solve: history copy failed");
  }
  if (cudaStreamSynchronize(st) != cudaSuccess)
    return set_error(DSKI_ERR_CUDA, "dski_pcg_solve: %s", cudaGetErrorString(cudaGetLastError()));
  run.iters = hi;
  run.relres.resize(s);
  bool conv = true;
  for (int c = 0; c < s; ++c) {
    run.relres[c] = hb[c] > 0 ? std::sqrt(hr[c] / hb[c]) : 0.0;
    if (!(run.relres[c] <= run.rtol)) conv = false;
    if (hbd[c]) run.breakdown = true;
  }
  if (run.breakdown)
    return set_error(DSKI_ERR_BREAKDOWN, "dski_pcg_solve: p^T K~ p <= 0 or non-finite value");
  if (!conv)
    return set_error(DSKI_ERR_NOT_CONVERGED,
                     "dski_pcg_solve: tolerance %.3g not met after %d iterations", run.rtol, its);
  return DSKI_OK;
}

}  // namespace dski

using namespace dski;

extern "C" int dski_pcg_solve(dski_handle h, pivchol_handle pc, const double* b_dev, double* x_dev,
                              int s, double rtol, int maxit, int* iters_host, double* relres_host) {
  clear_error();
  if (!h || !b_dev || !x_dev) return set_error(DSKI_ERR_ARG, "dski_pcg_solve: NULL argument");
  if (s < 1 || s > 256) return set_error(DSKI_ERR_ARG, "dski_pcg_solve: s must be in 1..256");
  if (!(rtol > 0.0) || maxit < 1) return set_error(DSKI_ERR_ARG, "dski_pcg_solve: need rtol > 0, maxit >= 1");
  if (pc && pc->h != h) return set_error(DSKI_ERR_ARG, "dski_pcg_solve: preconditioner of another handle");
  // run on the handle's private stream (capturable), ordered after the
  // caller's stream by an event and before its later work by another
  cudaStream_t user = h->stream;
  if (!h->pstream) {
    if (cudaStreamCreateWithFlags(&h->pstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->pev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->pev_out, cudaEventDisableTiming) != cudaSuccess)
      return set_error(DSKI_ERR_CUDA, "dski_pcg_solve: stream creation failed: %s",
                       cudaGetErrorString(cudaGetLastError()));
  }
  if (cudaEventRecord(h->pev_in, user) != cudaSuccess ||
      cudaStreamWaitEvent(h->pstream, h->pev_in, 0) != cudaSuccess)
    return set_error(DSKI_ERR_CUDA, "dski_pcg_solve: %s", cudaGetErrorString(cudaGetLastError()));
  h->stream = h->pstream;
  struct StreamBack {
    dski_handle h;
    cudaStream_t user;
    ~StreamBack() {
      cudaEventRecord(h->pev_out, h->pstream);
      cudaStreamWaitEvent(user, h->pev_out, 0);
      h->stream = user;
    }
  } back{h, user};
  const size_t Ns = (size_t)h->N * s;
  double* Bi = wbuf(h->s_vec[8], Ns);
  double* Xi = wbuf(h->s_vec[9], Ns);
  if (!Bi || !Xi) return DSKI_ERR_ALLOC;
  DSKI_TRY(permute_in(h, b_dev, Bi, s, true, h->stream));
  DSKI_TRY(permute_in(h, x_dev, Xi, s, true, h->stream));
  CgRun run;
  run.s = s;
  run.rtol = rtol;
  run.maxit = maxit;
  run.pc = pc;
  run.B = Bi;
  run.X = Xi;
  const int rc = cg_run(h, run);
  if (rc == DSKI_OK || rc == DSKI_ERR_NOT_CONVERGED || rc == DSKI_ERR_BREAKDOWN) {
    const int rc2 = permute_out(h, Xi, x_dev, s, true, h->stream);
    if (rc2 != DSKI_OK) return rc2;
    for (int c = 0; c < s && !run.iters.empty(); ++c) {
      if (iters_host) iters_host[c] = run.iters[c];
      if (relres_host) relres_host[c] = run.relres[c];
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess)
      return set_error(DSKI_ERR_CUDA, "dski_pcg_solve: %s", cudaGetErrorString(cudaGetLastError()));
  }
  return rc;
}
