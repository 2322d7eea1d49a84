// C-ABI entry points: argument checks, handle lifetime, error reporting and
// the user-layout boundary (block order <-> sorted interleaved layout).
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "dski_internal.cuh"

namespace dski {

static thread_local char g_err[512] = "";

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

void clear_error() { g_err[0] = '\0'; }

// ------------------------------------------------------------ profiling ---
static std::atomic<long long> g_launches{0};

void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

struct Profiler {
  static constexpr size_t kMaxPairs = 1u << 18;
  struct Rec {
    cudaEvent_t a, b;
    int stage;
  };
  std::vector<cudaEvent_t> pool;   // events, recycled across recording sessions
  size_t next = 0;
  std::vector<Rec> recs;
  long long launches[ST_COUNT] = {};
  long long timed[ST_COUNT] = {};   // launches inside a recorded event pair
  cudaEvent_t open_ev[ST_COUNT] = {};
  bool active = false;
  bool truncated = false;
  bool failed = false;

  void reset() {
    next = 0;
    recs.clear();
    for (int k = 0; k < ST_COUNT; ++k) {
      launches[k] = 0;
      timed[k] = 0;
      open_ev[k] = nullptr;
    }
    truncated = failed = false;
    active = true;
  }
  cudaEvent_t fresh() {
    if (next < pool.size()) return pool[next++];
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      failed = true;
      return nullptr;
    }
    pool.push_back(e);
    ++next;
    return e;
  }
  ~Profiler() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

bool profiling_on(dski_handle h) { return h && h->prof && h->prof->active; }

void stage_begin(dski_handle h, int stage, cudaStream_t st) {
  Profiler* p = h ? h->prof : nullptr;
  if (!p || !p->active || p->failed) return;
  if (p->recs.size() >= Profiler::kMaxPairs) {
    p->truncated = true;
    return;
  }
  cudaEvent_t e = p->fresh();
  if (!e) return;
  if (cudaEventRecord(e, st) != cudaSuccess) {
    cudaGetLastError();
    p->failed = true;
    return;
  }
  p->open_ev[stage] = e;
}

void stage_end(dski_handle h, int stage, cudaStream_t st, int launches) {
  count_launches(launches);
  Profiler* p = h ? h->prof : nullptr;
  if (!p || !p->active) return;
  p->launches[stage] += launches;
  cudaEvent_t a = p->open_ev[stage];
  p->open_ev[stage] = nullptr;
  if (!a || p->failed) return;
  cudaEvent_t b = p->fresh();
  if (!b) return;
  if (cudaEventRecord(b, st) != cudaSuccess) {
    cudaGetLastError();
    p->failed = true;
    return;
  }
  p->recs.push_back({a, b, stage});
  p->timed[stage] += launches;
}

int DevBuf::ensure(size_t need) {
  if (need <= bytes && ptr != nullptr) return DSKI_OK;
  if (need == 0) need = 256;
  void* p = nullptr;
  if (cudaMalloc(&p, need) != cudaSuccess) {
    cudaGetLastError();   // clear the sticky-free allocation error
    return DSKI_ERR_ALLOC;
  }
  if (ptr) cudaFree(ptr);
  ptr = p;
  bytes = need;
  return DSKI_OK;
}

void DevBuf::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}

static void release_all(dski_handle h) {
  h->perm.release();
  h->inv_perm.release();
  h->cell.release();
  h->cell_start.release();
  h->frac64.release();
  h->frac32.release();
  h->W64.release();
  h->W32.release();
  h->Wdf.release();
  for (int k = 0; k < DSKI_MAXD; ++k) {
    h->K64[k].release();
    h->K32[k].release();
    h->Khi[k].release();
    h->Klo[k].release();
    h->dK64[k].release();
    h->fft_tw[k].release();
    h->fft_lam[k].release();
    h->Kdig[k].release();
    h->Kexp[k].release();
  }
  h->gridA.release();
  h->gridB.release();
  h->vin.release();
  h->vout.release();
  h->scratch.release();
  h->dev_err.release();
  h->scat_ab.release();
  h->ozP.release();
  h->s_dpart.release();
  h->s_part.release();
  h->s_tnpart.release();
  h->s_ticket.release();
  h->s_state.release();
  for (auto& b : h->s_vec) b.release();
}

static bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace dski

using namespace dski;

extern "C" const char* dski_last_error(void) { return g_err; }

extern "C" int dski_create(dski_handle* out, const dski_params* p, const double* X_dev,
                           void* cuda_stream) {
  clear_error();
  if (!out) return set_error(DSKI_ERR_ARG, "dski_create: out is NULL");
  *out = nullptr;
  if (!p) return set_error(DSKI_ERR_ARG, "dski_create: params is NULL");
  if (p->n < 1) return set_error(DSKI_ERR_ARG, "dski_create: n must be >= 1 (got %d)", p->n);
  if (p->d < 1 || p->d > DSKI_MAXD)
    return set_error(DSKI_ERR_ARG, "dski_create: d must be in 1..3 (got %d)", p->d);
  if (!p->grid_m || !p->grid_lo || !p->grid_hi || !p->lengthscale || !X_dev)
    return set_error(DSKI_ERR_ARG, "dski_create: NULL array argument");
  if (p->prec != DSKI_FP64 && p->prec != DSKI_MIXED_3XTF32 && p->prec != DSKI_MIXED_TF32 &&
      p->prec != DSKI_FP64_TC)
    return set_error(DSKI_ERR_ARG, "dski_create: unknown precision %d", (int)p->prec);
  if (!finite_pos(p->outputscale) || !finite_pos(p->noise_value) || !finite_pos(p->noise_grad))
    return set_error(DSKI_ERR_ARG, "dski_create: outputscale and noises must be finite and > 0");
  if (p->interp != DSKI_INTERP_CUBIC && p->interp != DSKI_INTERP_QUINTIC)
    return set_error(DSKI_ERR_ARG, "dski_create: unknown interpolation scheme %d", (int)p->interp);
  const int sw = p->interp == DSKI_INTERP_QUINTIC ? 6 : 4;   // stencil nodes per dimension
  if (p->kuu != DSKI_KUU_DENSE && p->kuu != DSKI_KUU_FFT)
    return set_error(DSKI_ERR_ARG, "dski_create: unknown K_UU product %d", (int)p->kuu);
  if (p->kuu == DSKI_KUU_FFT && p->prec != DSKI_FP64 && p->prec != DSKI_FP64_TC)
    return set_error(DSKI_ERR_ARG, "dski_create: the FFT K_UU product needs FP64 vectors (FP64 or FP64_TC)");
  long long M = 1, ncell = 1;
  for (int k = 0; k < p->d; ++k) {
    if (p->grid_m[k] < sw || p->grid_m[k] > 1027)
      return set_error(DSKI_ERR_ARG, "dski_create: grid_m[%d] must be in %d..1027 (got %d)", k,
                       sw, p->grid_m[k]);
    if (!(std::isfinite(p->grid_lo[k]) && std::isfinite(p->grid_hi[k]) &&
          p->grid_lo[k] < p->grid_hi[k]))
      return set_error(DSKI_ERR_ARG, "dski_create: need finite grid_lo[%d] < grid_hi[%d]", k, k);
    if (!finite_pos(p->lengthscale[k]))
      return set_error(DSKI_ERR_ARG, "dski_create: lengthscale[%d] must be finite and > 0", k);
    if (p->prec == DSKI_FP64_TC && (p->grid_m[k] % 8 != 0 || p->grid_m[k] > 256))
      return set_error(DSKI_ERR_ARG, "dski_create: FP64_TC needs grid_m[%d] a multiple of 8 and <= 256", k);
    M *= p->grid_m[k];
    ncell *= p->grid_m[k] - sw + 1;
  }
  if (M > (1LL << 30))
    return set_error(DSKI_ERR_ARG, "dski_create: grid has %lld nodes (max 2^30)", M);
  if ((long long)p->n * (p->d + 1) > (1LL << 31) - 1)
    return set_error(DSKI_ERR_ARG, "dski_create: n(d+1) exceeds 2^31-1");

  dski_handle h = new (std::nothrow) dski_handle_();
  if (!h) return set_error(DSKI_ERR_ALLOC, "dski_create: host allocation failed");
  h->n = p->n;
  h->d = p->d;
  h->N = p->n * (p->d + 1);
  h->M = (int)M;
  h->ncell = (int)ncell;
  h->sf = p->outputscale;
  h->nv = p->noise_value;
  h->ng = p->noise_grad;
  h->prec = p->prec;
  h->sw = sw;
  h->kuu_fft = p->kuu == DSKI_KUU_FFT;
  h->lead = sw / 2 - 1;
  h->stream = (cudaStream_t)cuda_stream;
  for (int k = 0; k < p->d; ++k) {
    h->m[k] = p->grid_m[k];
    h->mc[k] = p->grid_m[k] - sw + 1;
    h->lo[k] = p->grid_lo[k];
    h->hi[k] = p->grid_hi[k];
    h->h[k] = (p->grid_hi[k] - p->grid_lo[k]) / (p->grid_m[k] - 1);
    h->ell[k] = p->lengthscale[k];
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete h;
    return set_error(DSKI_ERR_CUDA, "dski_create: no usable CUDA device");
  }
  int rc = DSKI_OK;
  if (h->dev_err.ensure(256) != DSKI_OK ||
      cudaMemsetAsync(h->dev_err.ptr, 0, 256, h->stream) != cudaSuccess)
    rc = set_error(DSKI_ERR_ALLOC, "dski_create: device allocation failed");
  if (rc == DSKI_OK) rc = build_geometry(h, X_dev);
  if (rc == DSKI_OK) rc = build_factors(h);
  if (rc == DSKI_OK && cudaStreamSynchronize(h->stream) != cudaSuccess)
    rc = set_error(DSKI_ERR_CUDA, "dski_create: %s", cudaGetErrorString(cudaGetLastError()));
  if (rc != DSKI_OK) {
    release_all(h);
    delete h;
    return rc;
  }
  *out = h;
  return DSKI_OK;
}

extern "C" int dski_set_hypers(dski_handle h, const double* lengthscale, double outputscale,
                               double noise_value, double noise_grad) {
  clear_error();
  if (!h || !lengthscale) return set_error(DSKI_ERR_ARG, "dski_set_hypers: NULL argument");
  if (!finite_pos(outputscale) || !finite_pos(noise_value) || !finite_pos(noise_grad))
    return set_error(DSKI_ERR_ARG, "dski_set_hypers: outputscale and noises must be > 0");
  for (int k = 0; k < h->d; ++k)
    if (!finite_pos(lengthscale[k]))
      return set_error(DSKI_ERR_ARG, "dski_set_hypers: lengthscale[%d] must be > 0", k);
  for (int k = 0; k < h->d; ++k) h->ell[k] = lengthscale[k];
  h->sf = outputscale;
  h->nv = noise_value;
  h->ng = noise_grad;
  return build_factors(h);
}

extern "C" int dski_mvm(dski_handle h, const void* v_dev, void* out_dev, int s) {
  clear_error();
  if (!h || !v_dev || !out_dev) return set_error(DSKI_ERR_ARG, "dski_mvm: NULL argument");
  if (s < 1 || s > 4096) return set_error(DSKI_ERR_ARG, "dski_mvm: s must be in 1..4096");
  const bool f64 = f64_vectors(h);
  const size_t es = f64 ? 8 : 4;
  const size_t vbytes = (size_t)h->N * s * es;
  const char* a = (const char*)v_dev;
  const char* b = (const char*)out_dev;
  if (a < b + vbytes && b < a + vbytes)
    return set_error(DSKI_ERR_ARG, "dski_mvm: v and out overlap");
  if (h->vin.ensure(vbytes) || h->vout.ensure(vbytes))
    return set_error(DSKI_ERR_ALLOC, "dski_mvm: workspace allocation failed");
  DSKI_TRY(permute_in(h, v_dev, h->vin.ptr, s, f64, h->stream));
  DSKI_TRY(mvm_internal(h, h->vin.ptr, h->vout.ptr, s, f64));
  DSKI_TRY(permute_out(h, h->vout.ptr, out_dev, s, f64, h->stream));
  return DSKI_OK;
}

extern "C" int dski_profile(dski_handle h, int mode, double* ms_host, long long* launches_host,
                            long long* timed_host, int* truncated_host) {
  clear_error();
  if (!h) return set_error(DSKI_ERR_ARG, "dski_profile: NULL handle");
  if (mode == 1) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess)
      return set_error(DSKI_ERR_CUDA, "dski_profile: %s", cudaGetErrorString(cudaGetLastError()));
    if (!h->prof) h->prof = new (std::nothrow) Profiler();
    if (!h->prof) return set_error(DSKI_ERR_ALLOC, "dski_profile: host allocation failed");
    h->prof->reset();
    return DSKI_OK;
  }
  if (mode != 0) return set_error(DSKI_ERR_ARG, "dski_profile: mode must be 0 or 1");
  Profiler* p = h->prof;
  if (!p || !p->active) return set_error(DSKI_ERR_ARG, "dski_profile: profiling was not started");
  p->active = false;
  double ms[ST_COUNT] = {};
  int rc = DSKI_OK;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    rc = set_error(DSKI_ERR_CUDA, "dski_profile: %s", cudaGetErrorString(cudaGetLastError()));
  } else if (p->failed) {
    rc = set_error(DSKI_ERR_CUDA, "dski_profile: event creation or record failed");
  } else {
    for (const auto& r : p->recs) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
        rc = set_error(DSKI_ERR_CUDA, "dski_profile: %s", cudaGetErrorString(cudaGetLastError()));
        break;
      }
      ms[r.stage] += t;
    }
  }
  if (rc == DSKI_OK) {
    for (int k = 0; k < ST_COUNT; ++k) {
      if (ms_host) ms_host[k] = ms[k];
      if (launches_host) launches_host[k] = p->launches[k];
      if (timed_host) timed_host[k] = p->timed[k];
    }
    if (truncated_host) *truncated_host = p->truncated ? 1 : 0;
  }
  return rc;
}

extern "C" long long dski_launch_count(void) { return g_launches.load(); }

extern "C" int dski_set_wait_budget(dski_handle h, int polls) {
  dski::clear_error();
  if (!h) return dski::set_error(DSKI_ERR_ARG, "dski_set_wait_budget: NULL handle");
  h->wait_budget = polls < 0 ? -1 : polls;
  return DSKI_OK;
}

namespace dski {
bool first_on_device(std::atomic<unsigned long long>* mask) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return true;   // unknown device: redo the (idempotent) set-up
  }
  const unsigned long long bit = 1ull << dev;
  return (mask->fetch_or(bit) & bit) == 0;
}

int check_device_error(dski_handle h) {
  int e = 0;
  if (cudaMemcpyAsync(&e, h->dev_err.ptr, sizeof(int), cudaMemcpyDeviceToHost, h->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return set_error(DSKI_ERR_CUDA, "%s", cudaGetErrorString(cudaGetLastError()));
  if (e) {
    cudaMemsetAsync(h->dev_err.ptr, 0, sizeof(int), h->stream);
    return set_error(DSKI_ERR_TIMEOUT, "a device-side wait ran out of its iteration budget");
  }
  return DSKI_OK;
}
}  // namespace dski

extern "C" void dski_destroy(dski_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  if (h->pstream) {
    cudaStreamSynchronize(h->pstream);
    cudaStreamDestroy(h->pstream);
  }
  if (h->pev_in) cudaEventDestroy(h->pev_in);
  if (h->pev_out) cudaEventDestroy(h->pev_out);
  delete h->prof;
  h->prof = nullptr;
  release_all(h);
  delete h;
}
