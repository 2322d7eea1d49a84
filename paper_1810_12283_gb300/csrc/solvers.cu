// Solver entry points (Sec. 2, Sec. 3.3, Eq. 1).
#include "dski_internal.cuh"

using namespace dski;

struct pivchol_ {
  int dummy;
};

extern "C" int pivchol_build(dski_handle h, int rank, pivchol_handle* out, int* rank_achieved) {
  (void)h; (void)rank; (void)out; (void)rank_achieved;
  return set_error(DSKI_ERR_ARG, "pivchol_build: not available in this build");
}

extern "C" void pivchol_destroy(pivchol_handle pc) { (void)pc; }

extern "C" int dski_pcg_solve(dski_handle h, pivchol_handle pc, const double* b_dev, double* x_dev,
                              int s, double rtol, int maxit, int* iters_host, double* relres_host) {
  (void)h; (void)pc; (void)b_dev; (void)x_dev; (void)s; (void)rtol; (void)maxit;
  (void)iters_host; (void)relres_host;
  return set_error(DSKI_ERR_ARG, "dski_pcg_solve: not available in this build");
}

extern "C" int dski_logdet_slq(dski_handle h, pivchol_handle pc, int probes, int depth,
                               uint64_t seed, double* logdet_host, double* stderr_host) {
  (void)h; (void)pc; (void)probes; (void)depth; (void)seed; (void)logdet_host; (void)stderr_host;
  return set_error(DSKI_ERR_ARG, "dski_logdet_slq: not available in this build");
}

extern "C" int dski_mll_grad(dski_handle h, pivchol_handle pc, const double* y_dev, int probes,
                             uint64_t seed, double* mll_host, double* grad_host) {
  (void)h; (void)pc; (void)y_dev; (void)probes; (void)seed; (void)mll_host; (void)grad_host;
  return set_error(DSKI_ERR_ARG, "dski_mll_grad: not available in this build");
}
