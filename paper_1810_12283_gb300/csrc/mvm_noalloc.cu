// dski_mvm_noalloc: the D-SKI MVM of dski_mvm with every temporary placed in
// one fixed, file-scope device array instead of memory the handle allocates.
//
// Why: dski_mvm grows the handle's workspace with cudaMalloc on first use.
// Some callers cannot allow that: applications whose memory is owned by a
// pool allocator that must see every device allocation, real-time loops in
// which cudaMalloc's implicit device synchronisation is not allowed, and
// plug-ins whose host forbids device allocation after start-up.  This entry
// point allocates nothing; the array below is reserved when the library is
// loaded, on every GPU that loads it, and stays reserved until the process
// exits.
#include <algorithm>
#include <mutex>

#include "dski_internal.cuh"

namespace {

// Layout of one call: [vin | vout | gridA | gridB | scatter intermediate |
// tensor-core partials], each part padded to 256 bytes.
constexpr size_t kScratchBytes = size_t(32) << 20;   // DSKI_NOALLOC_SCRATCH_BYTES
static_assert(kScratchBytes == (size_t)DSKI_NOALLOC_SCRATCH_BYTES, "keep dski.h in sync");
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};   // device address of g_scratch, per device

size_t pad256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of g_scratch on the current device.  In host code the name
// g_scratch is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess)
    return dski::set_error(DSKI_ERR_CUDA, "dski_mvm_noalloc: no current CUDA device");
  if (dev < 0 || dev >= kMaxDevices)
    return dski::set_error(DSKI_ERR_ARG, "dski_mvm_noalloc: device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return dski::set_error(DSKI_ERR_CUDA, "dski_mvm_noalloc: cudaGetSymbolAddress failed: %s",
                             cudaGetErrorString(e));
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return DSKI_OK;
}

}  // namespace

using namespace dski;

extern "C" int dski_mvm_noalloc(dski_handle h, const void* v_dev, void* out_dev, int s) {
  clear_error();
  if (!h || !v_dev || !out_dev) return set_error(DSKI_ERR_ARG, "dski_mvm_noalloc: NULL argument");
  if (s < 1) return set_error(DSKI_ERR_ARG, "dski_mvm_noalloc: s must be >= 1");
  if (h->prec == DSKI_FP64_TC)
    return set_error(DSKI_ERR_ARG,
                     "dski_mvm_noalloc: FP64_TC mode needs a split-contraction workspace; use FP64 or MIXED");
  const bool f64 = f64_vectors(h);
  const size_t es = f64 ? 8 : 4;
  const size_t vbytes = (size_t)h->N * s * es;
  const size_t gbytes = (size_t)h->M * s * es;
  const size_t abytes = scatter_ws_bytes(h, s, f64);
  // MIXED modes: the split-contraction partials of the largest mode product
  size_t tbytes = 0;
  if (!f64)
    for (int k = 0; k < h->d; ++k)
      tbytes = std::max(tbytes, mode_tc_tf32_ws_bytes(h->m[k], h->M / h->m[k], s));
  const size_t need = 2 * pad256(vbytes) + 2 * pad256(gbytes) + pad256(abytes) + pad256(tbytes);
  if (need > kScratchBytes)
    return set_error(DSKI_ERR_ARG,
                     "dski_mvm_noalloc: needs %zu scratch bytes for s = %d, the fixed limit is %zu "
                     "(2 N s + 2 M s elements, the scatter intermediate and the tensor-core "
                     "partials); use dski_mvm or fewer columns",
                     need, s, kScratchBytes);
  const char* a = (const char*)v_dev;
  const char* b = (const char*)out_dev;
  if (a < b + vbytes && b < a + vbytes)
    return set_error(DSKI_ERR_ARG, "dski_mvm_noalloc: v and out overlap");
  // the handle's memory must live on the current device
  cudaPointerAttributes attr{};
  int dev = -1;
  if (cudaPointerGetAttributes(&attr, h->perm.ptr) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess)
    return set_error(DSKI_ERR_CUDA, "dski_mvm_noalloc: %s", cudaGetErrorString(cudaGetLastError()));
  if (attr.device != dev)
    return set_error(DSKI_ERR_ARG, "dski_mvm_noalloc: handle lives on device %d, current is %d",
                     attr.device, dev);
  void* base = nullptr;
  DSKI_TRY(scratch_address(&base));
  char* p = static_cast<char*>(base);
  void* vin = p;
  void* vout = p + pad256(vbytes);
  void* gA = p + 2 * pad256(vbytes);
  void* gB = p + 2 * pad256(vbytes) + pad256(gbytes);
  void* ab = p + 2 * pad256(vbytes) + 2 * pad256(gbytes);
  void* tp = p + 2 * pad256(vbytes) + 2 * pad256(gbytes) + pad256(abytes);
  // Every stage writes its whole output before the next reads it, so nothing
  // in the array has to start at zero.  The tile autotuner stays off here.
  struct NoTune {
    NoTune() { set_no_tune(true); }
    ~NoTune() { set_no_tune(false); }
  } no_tune;
  DSKI_TRY(permute_in(h, v_dev, vin, s, f64, h->stream));
  DSKI_TRY(scatter_internal_ws(h, vin, gA, s, f64, abytes ? ab : nullptr));
  void* res = nullptr;
  DSKI_TRY(kron_internal(h, gA, gB, s, f64, -1, nullptr, &res, tbytes ? tp : nullptr));
  DSKI_TRY(gather_internal(h, res, vin, vout, s, f64));
  DSKI_TRY(permute_out(h, vout, out_dev, s, f64, h->stream));
  return DSKI_OK;
}
