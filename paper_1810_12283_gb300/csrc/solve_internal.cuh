// Internal declarations of the solvers (Sec. 2, Sec. 3.3, Eq. 1).
//
// All solver vectors live in the handle's internal layout (points sorted by
// grid cell, rows point-interleaved: row e = j (d + 1) + c) as FP64 N x s
// column-major arrays.  Dot products and norms are permutation invariant, so
// only the C-ABI boundary permutes.
//
// Reductions are deterministic: each block writes a partial sum, and the
// last block to finish (an atomic ticket after a memory fence) adds the
// partials in block order.
#pragma once

#include <vector>

#include "dski_internal.cuh"

// Preconditioner of Sec. 3.3 in the handle's internal layout:
//   M = D + L L^T,  Lt = D^-1/2 L,  [Lt; I] = [Q1; Q2] R  (CholeskyQR2, FP64),
//   M^-1 b = D^-1/2 (y - Q1 Q1^T y),  y = D^-1/2 b.
struct pivchol_ {
  dski_handle h = nullptr;
  int N = 0;
  int rank = 0;           // columns of L / Q1 actually built
  double nv = 0, ng = 0;  // noise diagonal at build time
  double logdetM = 0;     // log|M| = sum log D + 2 sum log diag(R)
  dski::DevBuf L;         // N x rank FP64, col-major
  dski::DevBuf Q1;        // N x rank FP64, col-major (FP64 mode)
  // other modes: Q1 = Qh + Ql as two FP32 arrays (N x rank each), applied
  // with error-free FP32 products and double-float sums (~2^-44 relative)
  bool split = false;
  dski::DevBuf Qh, Ql;
  // grid form (d = 2, M < N, FP64 vectors): M^-1 r = D^-1 (r - B H S H^T B^T D^-1 r)
  // with H's columns rank-1 Kronecker products (factors Hf: r x m0 then r x m1,
  // H1T = the second block transposed) and S = T T^T (r x r)
  bool grid_form = false;
  dski::DevBuf Hf, H1T, Sg, gwork;
  // FP64_TC: the grid form's two products on the tensor cores -- digit planes
  // of H1 (r x m1) and of H1^T (m1 x rp, rp = r rounded up to 8), their row
  // exponents (r + m1 ints) and H0^T padded to m0 x rp (FP64)
  bool oz = false;
  int rp = 0;
  dski::DevBuf ozH1, ozH1T, ozE, H0Tp;
  dski::DevBuf dis;       // D^-1/2 per internal row
  dski::DevBuf ds;        // D^1/2 per internal row
  std::vector<int> piv;   // internal row of pivot k
};

namespace dski {

constexpr int RED_THREADS = 256;

// ---- device reduction helpers (header-only, used by several .cu files) ----
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; the result is valid in thread 0.  `sh` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    t = lane < nw ? sh[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// True in every thread of the last block (of nblocks) to reach this point.
// Must be called by all threads of every block, after the block's partial
// results are written.  The last block resets the ticket for the next use.
__device__ __forceinline__ bool last_block(unsigned* ticket, unsigned nblocks) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(ticket, 1u);
    is_last = (t == nblocks - 1);
    if (is_last) *ticket = 0u;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// ---- double-float helpers: FP64-class accuracy on the FP32 units ----
// (Dekker / Knuth error-free transformations: TwoSum and the FMA-based
// exact product error.)  GB300 runs FP32 ~60x faster than FP64.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// (sh, sl) += (qh + ql) (yh + yl), dropping ql yl (below 2^-48 relative)
__device__ __forceinline__ void df_fma(float qh, float ql, float yh, float yl, float& sh,
                                       float& sl) {
  const float p = qh * yh;
  const float e = fmaf(qh, yh, -p);
  const float t = fmaf(qh, yl, fmaf(ql, yh, e));
  float s, err;
  two_sum(sh, p, s, err);
  sh = s;
  sl += err + t;
}
// (sh, sl) += (bh, bl)
__device__ __forceinline__ void df_add(float& sh, float& sl, float bh, float bl) {
  float s, err;
  two_sum(sh, bh, s, err);
  sh = s;
  sl += err + bl;
}
__device__ __forceinline__ void split_d(double x, float& h, float& l) {
  h = (float)x;
  l = (float)(x - (double)h);
}

// ---- host-side building blocks (pcg.cu) ----
// Column dots: out[q] = sum_i a[q L + i] b[q L + i] for q < s (FP64,
// deterministic); L = len, or N when len <= 0.
int col_dots(dski_handle h, const double* a, const double* b, int s, double* out_dev,
             long long len = 0);
// Tall-skinny products over N rows, col-major operands:
//   C (p x q) = A^T B   (A: N x p, B: N x q), optional row scaling w (B rows times w)
int ts_tn(dski_handle h, const double* A, int p, const double* B, int q, const double* w,
          double* C_dev);
//   Y (N x q) = rowscale .* (alpha xscale .* X + beta A C)
//   (A: N x p col-major, C: p x q row-major; X, xscale, rowscale may be NULL)
int ts_nn(dski_handle h, const double* X, double alpha, const double* xscale, double beta,
          const double* A, int p, const double* C, int q, double* Y, const double* rowscale);
unsigned* tickets(dski_handle h, int count);   // zeroed last-block tickets
//   C (p x q) = Q^T (w .* B) with Q = Qh + Ql split FP32 (q <= 4), FP64 result
int df_gemv_t(dski_handle h, const float* Qh, const float* Ql, int p, const double* B, int q,
              const double* w, double* C_dev);
// build pc->Qh / pc->Ql from pc->Q1 and mark the preconditioner split
int split_q1(dski_handle h, pivchol_handle pc);
// grid form of the preconditioner (precond_grid.cu): build after CholeskyQR2
// (no-op where it does not apply), and apply to s internal-layout columns
int grid_precond_build(dski_handle h, pivchol_handle pc, const int* piv_dev, const double* R1i,
                       const double* R2i);
// with up, the CG update of R runs in the scatter's point pass first (R is
// updated in place); with dpart_rz, the final gather leaves per-block partial
// sums of R^T Z (s <= 4 for either)
// with fin, the final gather's last block also runs that CG finisher
int grid_precond_apply(dski_handle h, pivchol_handle pc, const double* R, double* Z, int s,
                       const CgUpdate* up = nullptr, double* dpart_rz = nullptr,
                       const CgFinish* fin = nullptr);
// Noise diagonal of the internal layout: D[e] = nv (value rows) or ng.
int noise_diag(dski_handle h, double nv, double ng, double* D_dev);
// M^-1 for s columns: Z = D^-1/2 (Y - Q1 Q1^T Y), Y = D^-1/2 R.
int precond_apply(dski_handle h, pivchol_handle pc, const double* R, double* Z, int s);

// One batched PCG run on the internal layout (pcg.cu).
// ---- per-column PCG state and the scalar steps every finisher shares ----
// (device-resident FP64 scalars; the CG kernels and the gathers that fold a
// finisher into their last block both use them)
struct ColState {
  double *bn2, *rn2, *rz, *rz0, *alpha, *beta, *target;
  int *active, *iters, *bd, *nactive;
  double *ahist, *bhist;
  int depth;
  int s;
  // the inner passes run a perturbed operator (mixed modes, FFT products):
  // a non-positive p^T q there ends the pass instead of breaking down, and
  // the restart from the FP64 true residual refines x against the exact
  // operator
  int soft;
};

constexpr int CG_MAXS = 264;   // >= 1 + the largest probe count (256)

// In the last block: tot[c] = sum over bx of part[(c nb + bx) stride + off]
// for every column c < s.  The block's threads split the partials and a
// fixed tree combines them (deterministic).  tot is shared, length >= s.
__device__ inline void sum_columns(const double* part, int nb, int s, int stride, int off,
                            double* tot, double* sh) {
  for (int c = 0; c < s; ++c) {
    double v = 0.0;
    for (int bx = threadIdx.x; bx < nb; bx += blockDim.x)
      v += part[((long long)c * nb + bx) * stride + off];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) tot[c] = v;
  }
  __syncthreads();
}

// From the column sums tot[c] = r^T z: at (re)start rz (and rz0 once), else
// beta = (r^T z)_new / rz for active columns (recorded), 0 for the others.
__device__ inline void beta_finish(const double* tot, ColState& cs, int init) {
  for (int cc = threadIdx.x; cc < cs.s; cc += blockDim.x) {
    const double t = tot[cc];
    if (init) {
      cs.rz[cc] = t;
      cs.beta[cc] = 0.0;
      if (cs.rz0[cc] == 0.0) cs.rz0[cc] = t;
    } else if (cs.active[cc]) {
      const double be = t / cs.rz[cc];
      cs.beta[cc] = be;
      cs.rz[cc] = t;
      const int k = cs.iters[cc] - 1;
      if (cs.bhist && k >= 0 && k < cs.depth) cs.bhist[(long long)k * cs.s + cc] = be;
    } else {
      cs.beta[cc] = 0.0;
    }
  }
}

// From tot[c] = p^T q: alpha = r^T z / p^T q for active columns (recorded),
// breakdown (non-positive or non-finite) deactivates a column.
__device__ inline void alpha_finish(const double* tot, ColState& cs) {
  for (int cc = threadIdx.x; cc < cs.s; cc += blockDim.x) {
    double al = 0.0;
    if (cs.active[cc]) {
      const double t = tot[cc];
      if (!(t > 0.0) || !isfinite(t) || !isfinite(cs.rz[cc])) {
        if (!cs.soft || !isfinite(cs.rz[cc])) cs.bd[cc] = 1;
        cs.active[cc] = 0;
      } else {
        al = cs.rz[cc] / t;
        const int k = cs.iters[cc];
        if (cs.ahist && k < cs.depth) cs.ahist[(long long)k * cs.s + cc] = al;
      }
    }
    cs.alpha[cc] = al;
  }
}

// From tot[c] = ||r||^2 after the update: record it, count the iteration,
// deactivate the columns that met their target; the active count.
__device__ inline void update_finish(const double* tot, ColState& cs, double* sh) {
  int nact = 0;
  for (int cc = threadIdx.x; cc < cs.s; cc += blockDim.x) {
    if (cs.active[cc]) {
      const double t = tot[cc];
      cs.rn2[cc] = t;
      cs.iters[cc] += 1;
      if (!(t > cs.target[cc])) cs.active[cc] = 0;
    }
    nact += cs.active[cc];
  }
  nact = (int)block_sum((double)nact, sh);
  if (threadIdx.x == 0) *cs.nactive = nact;
}


// A CG finisher folded into the last block of a gather whose per-block
// partial sums it completes (see k_gather): kind 0 sums the gather's
// p^T q partials and sets alpha; kind 1 sums part2 (||r||^2 after the
// update), does the update's bookkeeping, then sums the gather's r^T z
// partials and sets beta.  kind < 0: none.
struct CgFinish {
  int kind = -1;
  ColState cs{};
  unsigned* ticket = nullptr;
  const double* part2 = nullptr;
  int nb2 = 0;   // partial sums per column in part2 (0: as many as the gather's blocks)
};

struct CgRun {
  int s = 1;
  double rtol = 1e-8;
  int maxit = 1000;
  int depth = 0;
  pivchol_handle pc = nullptr;
  const double* B = nullptr;   // internal layout N x s
  double* X = nullptr;         // internal layout N x s (initial guess in, solution out)
  // host results
  std::vector<int> iters;
  std::vector<double> relres, rz0, ahist, bhist;
  bool breakdown = false;
};
int cg_run(dski_handle h, CgRun& run);

// Ensure `count` doubles in b; returns the pointer or NULL (error set).
double* wbuf(DevBuf& b, size_t count);

}  // namespace dski
