// Stochastic Lanczos quadrature for log|K~| (Sec. 2) and the gradient of the
// log marginal likelihood (Eq. 1) with respect to
// theta = (log l_1..log l_d, log s_f, log sigma_n).
//
// Probes.  With the preconditioner M = D + L L^T of Sec. 3.3, probe j is
//   z_j = D^1/2 w1 + L w2,  w = [w1; w2] Rademacher of length N + r,
// so E[z z^T] = M.  For any such z,
//   E[ z^T M^-1/2 log(M^-1/2 K~ M^-1/2) M^-1/2 z ] = tr log(M^-1/2 K~ M^-1/2)
//                                                 = log|K~| - log|M|,
// and PCG on K~ x = z with preconditioner M is the Lanczos process on
// M^-1/2 K~ M^-1/2 started from M^-1/2 z (norm^2 = z^T M^-1 z).  Gauss
// quadrature gives the quadratic form as
//   (z^T M^-1 z) sum_i tau_i^2 log(lambda_i)
// with (lambda_i, tau_i) the eigenvalues and first eigenvector components of
// the Lanczos tridiagonal (Golub and Welsch, Math. Comp. 1969).  The
// Rademacher entries come from the counter-based SplitMix64 generator
// (Steele, Lea and Flood, OOPSLA 2014): entry e (caller block order, then the
// r extra rows) of probe j is the sign of output number j (N + r) + e + 1.
//
// Gradient.  dL/dtheta_i = 1/2 a^T dK~_i a - 1/2 tr(K~^-1 dK~_i), a = K~^-1 y,
// the trace estimated as mean_j (K~^-1 z_j)^T dK~_i (M^-1 z_j) (unbiased
// because E[z z^T] = M).  B does not depend on theta, so every bilinear form
// u^T dK~_i v with i < d + 1 is a grid form (B^T u)^T dK_UU,i (B^T v), with
//   dK_UU / dlog l_k = s_f^2 K_1 (x) .. (x) (K_k .* (u_a - u_b)^2 / l_k^2) (x) .. (x) K_d,
//   dK_UU / dlog s_f = 2 K_UU,
// and dK~ / dlog sigma_n = 2 D (both noise levels scale with sigma_n^2).
#include <algorithm>
#include <cmath>
#include <vector>

#include "solve_internal.cuh"

namespace dski {
namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double rademacher(unsigned long long seed, unsigned long long k) {
  const unsigned long long v = mix64(seed + k * 0x9E3779B97F4A7C15ULL);
  return (v >> 63) ? -1.0 : 1.0;
}

// Z[:, j] = D^1/2 w1 + L w2 on the internal layout (grid: rows x probes).
__global__ void __launch_bounds__(256) k_probes(const int* __restrict__ perm, int n, int d,
                                                long long N, const double* __restrict__ ds,
                                                const double* __restrict__ L, int rank,
                                                unsigned long long seed, double* __restrict__ Z) {
  __shared__ double w2[128];
  const int j = blockIdx.y;
  const unsigned long long base = (unsigned long long)j * (unsigned long long)(N + rank);
  for (int t = threadIdx.x; t < rank; t += blockDim.x)
    w2[t] = rademacher(seed, base + (unsigned long long)N + t + 1);
  __syncthreads();
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N;
       e += (long long)gridDim.x * blockDim.x) {
    const long long pt = e / (d + 1);
    const int c = (int)(e % (d + 1));
    const long long u = (long long)c * n + perm[pt];
    double v = ds[e] * rademacher(seed, base + (unsigned long long)u + 1);
    for (int t = 0; t < rank; ++t) v = fma(L[(long long)t * N + e], w2[t], v);
    Z[(long long)j * N + e] = v;
  }
}

// Gauss quadrature of each probe's Lanczos tridiagonal: one thread per probe.
// Eigen-decomposition by the implicit QL method with Wilkinson shifts
// (Golub and Van Loan, Matrix Computations, Sec. 8.3), accumulating only the
// first row of the eigenvector matrix.  gam[j] = rz0_j sum_i tau_i^2 log lambda_i.
__global__ void k_quadrature(const double* __restrict__ ah, const double* __restrict__ bh,
                             const int* __restrict__ kk, const double* __restrict__ rz0,
                             int s, int col0, int P, int depth, double* __restrict__ gam,
                             int* __restrict__ bad) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  const int c = col0 + j;
  const int k = min(kk[c], depth);
  double dg[128], of[128], z[128];
  for (int i = 0; i < k; ++i) {
    const double a = ah[(long long)i * s + c];
    dg[i] = 1.0 / a + (i > 0 ? bh[(long long)(i - 1) * s + c] / ah[(long long)(i - 1) * s + c] : 0.0);
    of[i] = (i + 1 < k) ? sqrt(bh[(long long)i * s + c]) / a : 0.0;
    z[i] = (i == 0) ? 1.0 : 0.0;
  }
  // implicit QL on (dg, of): of[i] couples i and i+1
  int fail = 0;
  for (int l = 0; l < k; ++l) {
    int iter = 0;
    while (true) {
      int m = l;
      for (; m < k - 1; ++m) {
        const double dd = fabs(dg[m]) + fabs(dg[m + 1]);
        if (fabs(of[m]) <= 1e-15 * dd) break;
      }
      if (m == l) break;
      if (++iter > 60) { fail = 1; break; }
      double g = (dg[l + 1] - dg[l]) / (2.0 * of[l]);
      double r = hypot(g, 1.0);
      g = dg[m] - dg[l] + of[l] / (g + copysign(r, g));
      double sn = 1.0, cs = 1.0, p = 0.0;
      int i = m - 1;
      bool deflated = false;
      for (; i >= l; --i) {
        double f = sn * of[i];
        const double b = cs * of[i];
        r = hypot(f, g);
        of[i + 1] = r;
        if (r == 0.0) {
          dg[i + 1] -= p;
          of[m] = 0.0;
          deflated = true;
          break;
        }
        sn = f / r;
        cs = g / r;
        g = dg[i + 1] - p;
        r = (dg[i] - g) * sn + 2.0 * cs * b;
        p = sn * r;
        dg[i + 1] = g + p;
        g = cs * r - b;
        // rotate the first-row components of columns i and i+1
        f = z[i + 1];
        z[i + 1] = sn * z[i] + cs * f;
        z[i] = cs * z[i] - sn * f;
      }
      if (deflated) continue;
      dg[l] -= p;
      of[l] = g;
      of[m] = 0.0;
    }
    if (fail) break;
  }
  double acc = 0.0;
  for (int i = 0; i < k; ++i) {
    if (!(dg[i] > 0.0)) fail = 1;
    acc += z[i] * z[i] * log(fmax(dg[i], 1e-300));
  }
  gam[j] = rz0[c] * acc;
  if (fail) atomicExch(bad, 1);
}

}  // namespace

struct SlqOut {
  double logdet = 0, stderr_ = 0, mean = 0;
  std::vector<double> gam;
};

// Probes, one batched PCG of `cols` = extra + P columns (the first `extra`
// columns of B are given), quadrature of the probe columns.
static int probe_solve(dski_handle h, pivchol_handle pc, int P, int depth, uint64_t seed,
                       double rtol, int maxit, CgRun& run, double* Bi, double* Xi, int extra,
                       SlqOut& out) {
  const long long N = h->N;
  const int s = extra + P;
  cudaStream_t st = h->stream;
  {
    StageScope sc(h, ST_LANCZOS, st);
    const int nbx = (int)std::min<long long>((N + 255) / 256, 4LL * h->sm_count);
    k_probes<<<dim3(nbx, P), 256, 0, st>>>(h->perm.as<int>(), h->n, h->d, N, pc->ds.as<double>(),
                                            pc->L.as<double>(), pc->rank,
                                            (unsigned long long)seed, Bi + (size_t)extra * N);
  }
  DSKI_LAUNCHED();
  if (cudaMemsetAsync(Xi, 0, (size_t)N * s * 8, st) != cudaSuccess)
    return set_error(DSKI_ERR_CUDA, "slq: memset failed");
  run.s = s;
  run.rtol = rtol;
  run.maxit = maxit;
  run.depth = depth;
  run.pc = pc;
  run.B = Bi;
  run.X = Xi;
  int rc = cg_run(h, run);
  if (rc == DSKI_ERR_BREAKDOWN || (rc != DSKI_OK && rc != DSKI_ERR_NOT_CONVERGED)) return rc;
  const int crc = rc;
  // quadrature on the device
  DevBuf tmp;
  const size_t hs = (size_t)depth * s;
  if (tmp.ensure((2 * hs + s + P + 4) * 8 + (size_t)s * 4 + 16))
    return set_error(DSKI_ERR_ALLOC, "slq: allocation failed");
  double* ah = tmp.as<double>();
  double* bh = ah + hs;
  double* rz0 = bh + hs;
  double* gam = rz0 + s;
  int* kk = (int*)(gam + P + 2);
  int* bad = kk + s;
  std::vector<int> k_used(s);
  for (int c = 0; c < s; ++c) k_used[c] = std::min(run.iters[c], depth);
  rc = DSKI_OK;
  if (cudaMemcpyAsync(ah, run.ahist.data(), hs * 8, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(bh, run.bhist.data(), hs * 8, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(rz0, run.rz0.data(), s * 8, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(kk, k_used.data(), s * 4, cudaMemcpyHostToDevice, st) ||
      cudaMemsetAsync(bad, 0, 4, st))
    rc = set_error(DSKI_ERR_CUDA, "slq: copy failed");
  if (rc == DSKI_OK) {
    {
      StageScope sc(h, ST_LANCZOS, st);
      k_quadrature<<<(P + 63) / 64, 64, 0, st>>>(ah, bh, kk, rz0, s, extra, P, depth, gam, bad);
    }
    out.gam.resize(P);
    int hbad = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(out.gam.data(), gam, P * 8, cudaMemcpyDeviceToHost, st) ||
        cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, st) ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = set_error(DSKI_ERR_CUDA, "slq: quadrature failed: %s",
                     cudaGetErrorString(cudaGetLastError()));
    else if (hbad)
      rc = set_error(DSKI_ERR_BREAKDOWN, "slq: Lanczos tridiagonal not positive definite");
  }
  tmp.release();
  if (rc != DSKI_OK) return rc;
  double mean = 0.0;
  for (double g : out.gam) mean += g;
  mean /= P;
  double var = 0.0;
  for (double g : out.gam) var += (g - mean) * (g - mean);
  var = P > 1 ? var / (P - 1) : 0.0;
  out.mean = mean;
  out.logdet = pc->logdetM + mean;
  out.stderr_ = std::sqrt(var / P);
  return crc;
}

}  // namespace dski

using namespace dski;

extern "C" int dski_logdet_slq(dski_handle h, pivchol_handle pc, int probes, int depth,
                               uint64_t seed, double* logdet_host, double* stderr_host) {
  clear_error();
  if (!h || !pc) return set_error(DSKI_ERR_ARG, "dski_logdet_slq: NULL handle or preconditioner");
  if (pc->h != h) return set_error(DSKI_ERR_ARG, "dski_logdet_slq: preconditioner of another handle");
  if (probes < 2 || probes > 256) return set_error(DSKI_ERR_ARG, "dski_logdet_slq: probes in 2..256");
  if (depth < 1 || depth > 128) return set_error(DSKI_ERR_ARG, "dski_logdet_slq: depth in 1..128");
  const size_t Ns = (size_t)h->N * probes;
  DevBuf Bb, Xb;
  if (Bb.ensure(Ns * 8) || Xb.ensure(Ns * 8))
    return set_error(DSKI_ERR_ALLOC, "dski_logdet_slq: allocation failed");
  CgRun run;
  SlqOut out;
  // depth iterations per probe; a column stops earlier only at round-off level
  int rc = probe_solve(h, pc, probes, depth, seed, 1e-15, depth, run, Bb.as<double>(),
                       Xb.as<double>(), 0, out);
  if (rc == DSKI_ERR_NOT_CONVERGED) rc = DSKI_OK;   // truncated Lanczos is the method
  clear_error();
  Bb.release();
  Xb.release();
  if (rc != DSKI_OK) return rc;
  if (logdet_host) *logdet_host = out.logdet;
  if (stderr_host) *stderr_host = out.stderr_;
  return DSKI_OK;
}

extern "C" int dski_mll_grad(dski_handle h, pivchol_handle pc, const double* y_dev, int probes,
                             uint64_t seed, double* mll_host, double* grad_host) {
  return dski_mll_grad_tol(h, pc, y_dev, probes, seed, 1e-8, 100000, mll_host, grad_host);
}

extern "C" int dski_mll_grad_tol(dski_handle h, pivchol_handle pc, const double* y_dev,
                                 int probes, uint64_t seed, double rtol, int maxit,
                                 double* mll_host, double* grad_host) {
  clear_error();
  if (!h || !pc || !y_dev) return set_error(DSKI_ERR_ARG, "dski_mll_grad: NULL argument");
  if (pc->h != h) return set_error(DSKI_ERR_ARG, "dski_mll_grad: preconditioner of another handle");
  if (probes < 2 || probes > 256) return set_error(DSKI_ERR_ARG, "dski_mll_grad: probes in 2..256");
  if (!(rtol > 0.0) || !(rtol < 1.0) || maxit < 1)
    return set_error(DSKI_ERR_ARG, "dski_mll_grad: rtol in (0, 1) and maxit >= 1");
  const long long N = h->N;
  const long long M = h->M;
  const int d = h->d;
  const int s = 1 + probes;
  const int depth = 30;
  cudaStream_t st = h->stream;
  DevBuf Bb, Xb, Vb, Ga, Gb, Tb, Wb, dots;
  if (Bb.ensure((size_t)N * s * 8) || Xb.ensure((size_t)N * s * 8) ||
      Vb.ensure((size_t)N * s * 8) || Ga.ensure((size_t)M * s * 8) ||
      Gb.ensure((size_t)M * s * 8) || Tb.ensure((size_t)M * s * 8) ||
      Wb.ensure((size_t)N * s * 8) || dots.ensure((size_t)(d + 3) * s * 8))
    return set_error(DSKI_ERR_ALLOC, "dski_mll_grad: allocation failed");
  double* Bi = Bb.as<double>();
  double* Xi = Xb.as<double>();
  DSKI_TRY(permute_in(h, y_dev, Bi, 1, true, st));
  CgRun run;
  SlqOut out;
  int rc = probe_solve(h, pc, probes, depth, seed, rtol, maxit, run, Bi, Xi, 1, out);
  if (rc != DSKI_OK) return rc;
  // V = [alpha, M^-1 z_1 .. M^-1 z_P]
  double* V = Vb.as<double>();
  if (cudaMemcpyAsync(V, Xi, (size_t)N * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return set_error(DSKI_ERR_CUDA, "dski_mll_grad: copy failed");
  DSKI_TRY(precond_apply(h, pc, Bi + N, V + N, probes));
  // grids: Ga = B^T [alpha, u_j], Gb = B^T [alpha, v_j]
  DSKI_TRY(scatter_internal(h, Xi, Ga.ptr, s, true));
  DSKI_TRY(scatter_internal(h, V, Gb.ptr, s, true));
  double* D = dots.as<double>();   // (d + 3) x s: rows per theta + y^T alpha
  if (h->gridA.ensure((size_t)M * s * 8) || h->gridB.ensure((size_t)M * s * 8))
    return set_error(DSKI_ERR_ALLOC, "dski_mll_grad: grid workspace");
  for (int k = 0; k <= d; ++k) {
    // H = dK_UU,k Gb  (k < d: lengthscale k; k == d: K_UU itself)
    if (cudaMemcpyAsync(h->gridA.ptr, Gb.ptr, (size_t)M * s * 8, cudaMemcpyDeviceToDevice, st))
      return set_error(DSKI_ERR_CUDA, "dski_mll_grad: copy failed");
    void* res = nullptr;
    DSKI_TRY(kron_internal(h, h->gridA.ptr, Tb.ptr, s, true, k < d ? k : -1,
                           k < d ? h->dK64[k].ptr : nullptr, &res));
    DSKI_TRY(col_dots(h, Ga.as<double>(), (const double*)res, s, D + (size_t)k * s, M));
  }
  // noise: W = D .* V;  u^T D v
  DSKI_TRY(ts_nn(h, V, 1.0, pc->ds.as<double>(), 0.0, nullptr, 0, nullptr, s, Wb.as<double>(),
                 pc->ds.as<double>()));
  DSKI_TRY(col_dots(h, Xi, Wb.as<double>(), s, D + (size_t)(d + 1) * s));
  DSKI_TRY(col_dots(h, Bi, Xi, 1, D + (size_t)(d + 2) * s));
  std::vector<double> hd((size_t)(d + 3) * s);
  if (cudaMemcpyAsync(hd.data(), D, hd.size() * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return set_error(DSKI_ERR_CUDA, "dski_mll_grad: %s", cudaGetErrorString(cudaGetLastError()));
  const double scale[3] = {1.0, 2.0, 2.0};   // dK factors: lengthscales, s_f (2 K), sigma_n (2 D)
  for (int i = 0; i < d + 2; ++i) {
    const double* row = hd.data() + (size_t)i * s;
    const double sc = i < d ? scale[0] : (i == d ? scale[1] : scale[2]);
    double tr = 0.0;
    for (int j = 1; j < s; ++j) tr += row[j];
    tr /= probes;
    if (grad_host) grad_host[i] = 0.5 * sc * row[0] - 0.5 * sc * tr;
  }
  const double yta = hd[(size_t)(d + 2) * s];
  if (mll_host) *mll_host = -0.5 * (yta + out.logdet + (double)N * std::log(2.0 * M_PI));
  return DSKI_OK;
}
