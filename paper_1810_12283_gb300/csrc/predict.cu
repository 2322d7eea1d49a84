// Prediction with the D-SKI GP (Sec. 5: the mean and the fast variance
// estimate that Bayesian optimisation needs at many test points).
//
//   mean and gradient:  mu* = [W*; dW*] K_UU [W; dW]^T alpha,   alpha = K~^-1 y
//     (the test rows of the D-SKI cross-covariance, Sec. 3.1): one scatter of
//     alpha, the d mode products, then a gather at the test points;
//   variance estimate:  v_hat(x) = s_f^2 - k_x^T M^-1 k_x,  k_x = [W; dW] K_UU w*(x)^T
//     (Sec. 5's first approach: K~^-1 replaced by the pivoted-Cholesky
//     preconditioner solve): per batch of test points, their value weights
//     as grid columns, the mode products, a gather at the training points,
//     the preconditioner apply and one column dot each.
// Every step runs in FP64 whatever the handle's mode.
#include <algorithm>

#include "solve_internal.cuh"
#include "interp.cuh"

namespace dski {
namespace {

struct PredGeo {
  int d;
  int m[DSKI_MAXD];
  long long stride[DSKI_MAXD];   // grid strides (C order)
  double lo[DSKI_MAXD], h[DSKI_MAXD];
};

// Stencil of a test point: first node (c - S/2 + 1) per dimension, weights
// and derivative weights (already divided by h), as for the training points.
template <int D, int S>
__device__ __forceinline__ bool pred_stencil(const double* x, const PredGeo& g, int first[D],
                                             double w[D][S], double dw[D][S]) {
  constexpr int lead = S / 2 - 1;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double t = (x[k] - g.lo[k]) / g.h[k];
    const double c = floor(t);
    if (!(c >= (double)lead && c <= (double)(g.m[k] - S + lead))) {   // NaN fails too
      ok = false;
      first[k] = 0;
      for (int o = 0; o < S; ++o) w[k][o] = dw[k][o] = 0.0;
      continue;
    }
    first[k] = (int)c - lead;
    double ww[S], dd[S];
    stencil_weights<S, double>(t - c, ww, dd);
    const double ih = 1.0 / g.h[k];
#pragma unroll
    for (int o = 0; o < S; ++o) {
      w[k][o] = ww[o];
      dw[k][o] = dd[o] * ih;
    }
  }
  return ok;
}

// out (block order) = [W*; dW*] h at n* test points: one thread per point.
template <int D, int S>
__global__ void k_pred_gather(const double* __restrict__ Xs, int ns, PredGeo g,
                              const double* __restrict__ hgrid, int with_grad,
                              double* __restrict__ out, int* __restrict__ bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ns) return;
  int first[D];
  double w[D][S], dw[D][S];
  if (!pred_stencil<D, S>(Xs + (long long)i * D, g, first, w, dw)) atomicAdd(bad, 1);
  double val = 0.0, grad[D];
#pragma unroll
  for (int p = 0; p < D; ++p) grad[p] = 0.0;
  constexpr int NS = D == 1 ? S : (D == 2 ? S * S : S * S * S);
  for (int t = 0; t < NS; ++t) {
    int o[D];
    int r = t;
#pragma unroll
    for (int k = D - 1; k >= 0; --k) {
      o[k] = r % S;
      r /= S;
    }
    long long idx = 0;
    double wp = 1.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      idx += (long long)(first[k] + o[k]) * g.stride[k];
      wp *= w[k][o[k]];
    }
    const double hv = hgrid[idx];
    val = fma(wp, hv, val);
    if (with_grad) {
#pragma unroll
      for (int p = 0; p < D; ++p) {
        double gp = 1.0;
#pragma unroll
        for (int k = 0; k < D; ++k) gp *= k == p ? dw[k][o[k]] : w[k][o[k]];
        grad[p] = fma(gp, hv, grad[p]);
      }
    }
  }
  out[i] = val;
  if (with_grad)
#pragma unroll
    for (int p = 0; p < D; ++p) out[(long long)(p + 1) * ns + i] = grad[p];
}

// Column c of G (M x s, zeroed) = value weights of test point i0 + c.
template <int D, int S>
__global__ void k_pred_scatter(const double* __restrict__ Xs, int i0, int s, PredGeo g,
                               long long M, double* __restrict__ G, int* __restrict__ bad) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= s) return;
  int first[D];
  double w[D][S], dw[D][S];
  if (!pred_stencil<D, S>(Xs + (long long)(i0 + c) * D, g, first, w, dw)) atomicAdd(bad, 1);
  constexpr int NS = D == 1 ? S : (D == 2 ? S * S : S * S * S);
  for (int t = 0; t < NS; ++t) {
    int o[D];
    int r = t;
#pragma unroll
    for (int k = D - 1; k >= 0; --k) {
      o[k] = r % S;
      r /= S;
    }
    long long idx = 0;
    double wp = 1.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      idx += (long long)(first[k] + o[k]) * g.stride[k];
      wp *= w[k][o[k]];
    }
    G[(long long)c * M + idx] = wp;
  }
}

// var[c] = s_f^2 - dots[c]
__global__ void k_pred_var(const double* __restrict__ dots, int s, double sf2,
                           double* __restrict__ var) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < s) var[c] = sf2 - dots[c];
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Rademacher probe entry (test point i, probe j): the sign of output number
// j n* + i + 1 of the SplitMix64 stream seeded with `seed` (Steele, Lea and
// Flood, OOPSLA 2014; the top bit 0 gives +1).
__device__ __forceinline__ double test_probe(unsigned long long seed, long long ns, int j, int i) {
  const unsigned long long k = (unsigned long long)j * (unsigned long long)ns + (unsigned long long)i + 1ULL;
  return (mix64(seed + k * 0x9E3779B97F4A7C15ULL) >> 63) ? -1.0 : 1.0;
}

// G[j][:] (M x P, zeroed) = sum_i z_ij w*_i: thread (test point, probe),
// FP64 atomics where test points share grid nodes.
template <int D, int S>
__global__ void k_pred_scatter_z(const double* __restrict__ Xs, int ns, int P,
                                 unsigned long long seed, PredGeo g, long long M,
                                 double* __restrict__ G, int* __restrict__ bad) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)ns * P) return;
  const int i = (int)(t % ns), j = (int)(t / ns);
  int first[D];
  double w[D][S], dw[D][S];
  if (!pred_stencil<D, S>(Xs + (long long)i * D, g, first, w, dw)) {
    if (j == 0) atomicAdd(bad, 1);
    return;
  }
  const double z = test_probe(seed, ns, j, i);
  constexpr int NS = D == 1 ? S : (D == 2 ? S * S : S * S * S);
  for (int s4 = 0; s4 < NS; ++s4) {
    int o[D];
    int r = s4;
#pragma unroll
    for (int k = D - 1; k >= 0; --k) {
      o[k] = r % S;
      r /= S;
    }
    long long idx = 0;
    double wp = z;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      idx += (long long)(first[k] + o[k]) * g.stride[k];
      wp *= w[k][o[k]];
    }
    atomicAdd(&G[(long long)j * M + idx], wp);
  }
}

// var[i] -= (1/P) sum_j z_ij (w*_i . H[j]): one thread per test point.
template <int D, int S>
__global__ void k_pred_cv(const double* __restrict__ Xs, int ns, int P, unsigned long long seed,
                          PredGeo g, long long M, const double* __restrict__ H,
                          double* __restrict__ var) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ns) return;
  int first[D];
  double w[D][S], dw[D][S];
  if (!pred_stencil<D, S>(Xs + (long long)i * D, g, first, w, dw)) return;
  constexpr int NS = D == 1 ? S : (D == 2 ? S * S : S * S * S);
  double acc = 0.0;
  for (int j = 0; j < P; ++j) {
    const double* hj = H + (long long)j * M;
    double dot = 0.0;
    for (int s4 = 0; s4 < NS; ++s4) {
      int o[D];
      int r = s4;
#pragma unroll
      for (int k = D - 1; k >= 0; --k) {
        o[k] = r % S;
        r /= S;
      }
      long long idx = 0;
      double wp = 1.0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        idx += (long long)(first[k] + o[k]) * g.stride[k];
        wp *= w[k][o[k]];
      }
      dot = fma(wp, hj[idx], dot);
    }
    acc = fma(test_probe(seed, ns, j, i), dot, acc);
  }
  var[i] -= acc / P;
}

__global__ void k_axpy_neg(const double* __restrict__ a, const double* __restrict__ b,
                           long long n, double* __restrict__ c) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) c[t] = a[t] - b[t];
}

PredGeo pred_geo(dski_handle h) {
  PredGeo g{};
  g.d = h->d;
  long long st = 1;
  for (int k = h->d - 1; k >= 0; --k) {
    g.m[k] = h->m[k];
    g.stride[k] = st;
    st *= h->m[k];
    g.lo[k] = h->lo[k];
    g.h[k] = h->h[k];
  }
  return g;
}

}  // namespace
}  // namespace dski

using namespace dski;

extern "C" int dski_predict(dski_handle h, pivchol_handle pc, const double* alpha_dev,
                            const double* Xs_dev, int n_star, int with_grad, double* mean_dev,
                            double* var_dev) {
  clear_error();
  if (!h || !Xs_dev || n_star < 1) return set_error(DSKI_ERR_ARG, "dski_predict: NULL handle / points or n_star < 1");
  if (mean_dev && !alpha_dev) return set_error(DSKI_ERR_ARG, "dski_predict: the mean needs alpha");
  if (var_dev && !pc) return set_error(DSKI_ERR_ARG, "dski_predict: the variance needs a preconditioner");
  if (pc && pc->h != h) return set_error(DSKI_ERR_ARG, "dski_predict: preconditioner of another handle");
  if (!mean_dev && !var_dev) return DSKI_OK;
  cudaStream_t st = h->stream;
  const int d = h->d;
  const long long N = h->N, M = h->M;
  const PredGeo g = pred_geo(h);
  DevBuf bad;
  if (bad.ensure(16) || cudaMemsetAsync(bad.ptr, 0, 16, st) != cudaSuccess)
    return set_error(DSKI_ERR_ALLOC, "dski_predict: allocation failed");
  int* badp = bad.as<int>();
  if (mean_dev) {
    DevBuf A, G1, G2;
    if (A.ensure((size_t)N * 8) || G1.ensure((size_t)M * 8) || G2.ensure((size_t)M * 8))
      return set_error(DSKI_ERR_ALLOC, "dski_predict: allocation failed");
    DSKI_TRY(permute_in(h, alpha_dev, A.ptr, 1, true, st));
    DSKI_TRY(scatter_internal(h, A.ptr, G1.ptr, 1, true));
    void* res = nullptr;
    DSKI_TRY(kron_internal(h, G1.ptr, G2.ptr, 1, true, -1, nullptr, &res));
    {
      StageScope sc(h, ST_GATHER, st);
      const unsigned nb = (unsigned)((n_star + 127) / 128);
      with_stencil(h, [&](auto Sc) {
        constexpr int S = decltype(Sc)::value;
        switch (d) {
          case 1: k_pred_gather<1, S><<<nb, 128, 0, st>>>(Xs_dev, n_star, g, (const double*)res, with_grad, mean_dev, badp); break;
          case 2: k_pred_gather<2, S><<<nb, 128, 0, st>>>(Xs_dev, n_star, g, (const double*)res, with_grad, mean_dev, badp); break;
          default: k_pred_gather<3, S><<<nb, 128, 0, st>>>(Xs_dev, n_star, g, (const double*)res, with_grad, mean_dev, badp); break;
        }
      });
    }
    DSKI_LAUNCHED();
    if (cudaStreamSynchronize(st) != cudaSuccess)
      return set_error(DSKI_ERR_CUDA, "dski_predict: %s", cudaGetErrorString(cudaGetLastError()));
  }
  if (var_dev) {
    const int SB = (int)std::min<long long>(64, n_star);
    DevBuf G1, G2, K, Z, dots;
    if (G1.ensure((size_t)M * SB * 8) || G2.ensure((size_t)M * SB * 8) ||
        K.ensure((size_t)N * SB * 8) || Z.ensure((size_t)N * SB * 8) || dots.ensure((size_t)SB * 8))
      return set_error(DSKI_ERR_ALLOC, "dski_predict: allocation failed");
    for (int i0 = 0; i0 < n_star; i0 += SB) {
      const int s = std::min(SB, n_star - i0);
      if (cudaMemsetAsync(G1.ptr, 0, (size_t)M * s * 8, st) != cudaSuccess ||
          cudaMemsetAsync(K.ptr, 0, (size_t)N * s * 8, st) != cudaSuccess)
        return set_error(DSKI_ERR_CUDA, "dski_predict: memset failed");
      {
        StageScope sc(h, ST_SCATTER, st);
        with_stencil(h, [&](auto Sc) {
          constexpr int S = decltype(Sc)::value;
          switch (d) {
            case 1: k_pred_scatter<1, S><<<1, 64, 0, st>>>(Xs_dev, i0, s, g, M, G1.as<double>(), badp); break;
            case 2: k_pred_scatter<2, S><<<1, 64, 0, st>>>(Xs_dev, i0, s, g, M, G1.as<double>(), badp); break;
            default: k_pred_scatter<3, S><<<1, 64, 0, st>>>(Xs_dev, i0, s, g, M, G1.as<double>(), badp); break;
          }
        });
      }
      DSKI_LAUNCHED();
      void* res = nullptr;
      DSKI_TRY(kron_internal(h, G1.ptr, G2.ptr, s, true, -1, nullptr, &res));
      // k_x = [W; dW] (K_UU w*): the gather with no noise term (K holds zeros)
      DSKI_TRY(gather_scaled(h, (const double*)res, K.as<double>(), K.as<double>(), s, 1.0, 1.0,
                             0.0, 0.0, ST_GATHER));
      DSKI_TRY(precond_apply(h, pc, K.as<double>(), Z.as<double>(), s));
      DSKI_TRY(col_dots(h, K.as<double>(), Z.as<double>(), s, dots.as<double>()));
      {
        StageScope sc(h, ST_PCGVEC, st);
        k_pred_var<<<1, 64, 0, st>>>(dots.as<double>(), s, h->sf * h->sf, var_dev + i0);
      }
      DSKI_LAUNCHED();
    }
    if (cudaStreamSynchronize(st) != cudaSuccess)
      return set_error(DSKI_ERR_CUDA, "dski_predict: %s", cudaGetErrorString(cudaGetLastError()));
  }
  int hb = 0;
  if (cudaMemcpy(&hb, badp, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return set_error(DSKI_ERR_CUDA, "dski_predict: %s", cudaGetErrorString(cudaGetLastError()));
  if (hb) return set_error(DSKI_ERR_OUT_OF_GRID, "dski_predict: %d test point(s) lack a full interpolation stencil", hb);
  return check_device_error(h);
}

extern "C" int dski_predict_var_cv(dski_handle h, pivchol_handle pc, const double* Xs_dev,
                                   int n_star, int probes, uint64_t seed, double rtol, int maxit,
                                   double* var_dev) {
  clear_error();
  if (!h || !pc || !Xs_dev || !var_dev || n_star < 1)
    return set_error(DSKI_ERR_ARG, "dski_predict_var_cv: NULL argument or n_star < 1");
  if (pc->h != h) return set_error(DSKI_ERR_ARG, "dski_predict_var_cv: preconditioner of another handle");
  if (probes < 1 || probes > 256) return set_error(DSKI_ERR_ARG, "dski_predict_var_cv: probes in 1..256");
  if (!(rtol > 0.0) || maxit < 1) return set_error(DSKI_ERR_ARG, "dski_predict_var_cv: need rtol > 0, maxit >= 1");
  // v_hat first (the control variate)
  DSKI_TRY(dski_predict(h, pc, nullptr, Xs_dev, n_star, 0, nullptr, var_dev));
  cudaStream_t st = h->stream;
  const int d = h->d, P = probes;
  const long long N = h->N, M = h->M;
  const PredGeo g = pred_geo(h);
  DevBuf bad, G1, G2, U, A, Bm;
  if (bad.ensure(16) || G1.ensure((size_t)M * P * 8) || G2.ensure((size_t)M * P * 8) ||
      U.ensure((size_t)N * P * 8) || A.ensure((size_t)N * P * 8) || Bm.ensure((size_t)N * P * 8))
    return set_error(DSKI_ERR_ALLOC, "dski_predict_var_cv: allocation failed");
  if (cudaMemsetAsync(bad.ptr, 0, 16, st) != cudaSuccess ||
      cudaMemsetAsync(G1.ptr, 0, (size_t)M * P * 8, st) != cudaSuccess ||
      cudaMemsetAsync(U.ptr, 0, (size_t)N * P * 8, st) != cudaSuccess ||
      cudaMemsetAsync(A.ptr, 0, (size_t)N * P * 8, st) != cudaSuccess)
    return set_error(DSKI_ERR_CUDA, "dski_predict_var_cv: memset failed");
  int* badp = bad.as<int>();
  // U = K_X* Z: the probes' test weights on the grid, K_UU, gather at the training points
  {
    StageScope sc(h, ST_SCATTER, st);
    const long long th = (long long)n_star * P;
    const unsigned nb = (unsigned)((th + 255) / 256);
    with_stencil(h, [&](auto Sc) {
      constexpr int S = decltype(Sc)::value;
      switch (d) {
        case 1: k_pred_scatter_z<1, S><<<nb, 256, 0, st>>>(Xs_dev, n_star, P, seed, g, M, G1.as<double>(), badp); break;
        case 2: k_pred_scatter_z<2, S><<<nb, 256, 0, st>>>(Xs_dev, n_star, P, seed, g, M, G1.as<double>(), badp); break;
        default: k_pred_scatter_z<3, S><<<nb, 256, 0, st>>>(Xs_dev, n_star, P, seed, g, M, G1.as<double>(), badp); break;
      }
    });
  }
  DSKI_LAUNCHED();
  void* res = nullptr;
  DSKI_TRY(kron_internal(h, G1.ptr, G2.ptr, P, true, -1, nullptr, &res));
  DSKI_TRY(gather_scaled(h, (const double*)res, U.as<double>(), U.as<double>(), P, 1.0, 1.0, 0.0,
                         0.0, ST_GATHER));
  // A = K~^-1 U (PCG), Bm = M^-1 U, U <- A - Bm
  CgRun run;
  run.s = P;
  run.rtol = rtol;
  run.maxit = maxit;
  run.pc = pc;
  run.B = U.as<double>();
  run.X = A.as<double>();
  int rc = cg_run(h, run);
  if (rc != DSKI_OK && rc != DSKI_ERR_NOT_CONVERGED) return rc;
  const int crc = rc;
  DSKI_TRY(precond_apply(h, pc, U.as<double>(), Bm.as<double>(), P));
  {
    StageScope sc(h, ST_PCGVEC, st);
    const long long tot = N * P;
    k_axpy_neg<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(A.as<double>(), Bm.as<double>(), tot,
                                                           U.as<double>());
  }
  DSKI_LAUNCHED();
  // K_*X (A - Bm): scatter at the training points, K_UU, then per test point
  // the probe-weighted mean of its value interpolation
  DSKI_TRY(scatter_internal(h, U.ptr, G1.ptr, P, true));
  DSKI_TRY(kron_internal(h, G1.ptr, G2.ptr, P, true, -1, nullptr, &res));
  {
    StageScope sc(h, ST_GATHER, st);
    const unsigned nb = (unsigned)((n_star + 127) / 128);
    with_stencil(h, [&](auto Sc) {
      constexpr int S = decltype(Sc)::value;
      switch (d) {
        case 1: k_pred_cv<1, S><<<nb, 128, 0, st>>>(Xs_dev, n_star, P, seed, g, M, (const double*)res, var_dev); break;
        case 2: k_pred_cv<2, S><<<nb, 128, 0, st>>>(Xs_dev, n_star, P, seed, g, M, (const double*)res, var_dev); break;
        default: k_pred_cv<3, S><<<nb, 128, 0, st>>>(Xs_dev, n_star, P, seed, g, M, (const double*)res, var_dev); break;
      }
    });
  }
  DSKI_LAUNCHED();
  int hb = 0;
  if (cudaMemcpyAsync(&hb, badp, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return set_error(DSKI_ERR_CUDA, "dski_predict_var_cv: %s", cudaGetErrorString(cudaGetLastError()));
  if (hb) return set_error(DSKI_ERR_OUT_OF_GRID, "dski_predict_var_cv: %d test point(s) lack a full stencil", hb);
  rc = check_device_error(h);
  if (rc != DSKI_OK) return rc;
  if (crc == DSKI_ERR_NOT_CONVERGED)
    return set_error(DSKI_ERR_NOT_CONVERGED, "dski_predict_var_cv: probe solves missed rtol %.3g", rtol);
  return DSKI_OK;
}
