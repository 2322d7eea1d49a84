// Internal declarations of the D-SKI library (not part of the C ABI).
//
// Internal data layout (all device memory owned by the handle):
//   * points are kept sorted by grid cell (stable, by original index within a
//     cell); sorted position j <-> original point perm[j];
//   * an internal vector row is e = j (d + 1) + c, c = 0 for the value and
//     c = 1..d for d/dx_c ("point-interleaved"), s columns column-major
//     (column q at q N).  Dot products are permutation invariant, so the
//     solvers run entirely in this layout; only the C-ABI boundary permutes;
//   * a grid vector is the C-order grid (last dimension fastest), s columns
//     column-major (column q at q M).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <atomic>
#include <type_traits>

#include "../../include/dski.h"

#define DSKI_MAXD 3

namespace dski {

// ---------------------------------------------------------------- errors ---
int set_error(int code, const char* fmt, ...);
void clear_error();

#define DSKI_TRY(expr)                      \
  do {                                      \
    int rc__ = (expr);                      \
    if (rc__ != DSKI_OK) return rc__;       \
  } while (0)

#define DSKI_CUDA(call)                                                        \
  do {                                                                         \
    cudaError_t e__ = (call);                                                  \
    if (e__ != cudaSuccess)                                                    \
      return ::dski::set_error(DSKI_ERR_CUDA, "%s failed: %s (%s:%d)", #call,  \
                               cudaGetErrorString(e__), __FILE__, __LINE__);   \
  } while (0)

#define DSKI_LAUNCHED() DSKI_CUDA(cudaGetLastError())

// ------------------------------------------------------- stage profiling ---
// Per-stage CUDA-event timers (off unless dski_profile switched them on) and
// a process-wide count of the kernels this library launched.
enum Stage { ST_PERMUTE = 0, ST_SCATTER, ST_KRON, ST_GATHER, ST_PRECOND, ST_PCGVEC,
             ST_PIVCHOL, ST_LANCZOS, ST_COUNT };
static_assert(ST_COUNT == DSKI_NSTAGES, "stage table out of sync with dski.h");

struct Profiler;   // defined in capi.cu
void count_launches(int k);   // adds to the process-wide launch counter
long long launches_so_far();  // the process-wide launch counter
bool profiling_on(dski_handle h);   // stage timers recording
void stage_begin(dski_handle h, int stage, cudaStream_t st);
void stage_end(dski_handle h, int stage, cudaStream_t st, int launches);

// Brackets the launches of one stage: stage_begin on construction,
// stage_end (which also counts `launches` kernels) on destruction.
struct StageScope {
  dski_handle h;
  int stage;
  cudaStream_t st;
  int launches;
  StageScope(dski_handle h_, int stage_, cudaStream_t st_, int launches_ = 1)
      : h(h_), stage(stage_), st(st_), launches(launches_) {
    stage_begin(h, stage, st);
  }
  ~StageScope() { stage_end(h, stage, st, launches); }
};

// --------------------------------------------------------- device buffer ---
// A grow-only device allocation owned by a handle.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  int ensure(size_t need);   // grows (never shrinks); DSKI_OK or ALLOC
  void release();
  template <class T> T* as() const { return static_cast<T*>(ptr); }
};

}  // namespace dski

struct dski_handle_ {
  int n = 0, d = 0, N = 0;
  int m[DSKI_MAXD] = {1, 1, 1};     // grid nodes per dimension
  int mc[DSKI_MAXD] = {1, 1, 1};    // cells per dimension (m_k - sw + 1)
  // interpolation stencil: sw nodes per dimension (4 cubic, 6 quintic); a
  // point in cell floor(t) uses the nodes floor(t) - lead .. floor(t) - lead + sw - 1
  int sw = 4, lead = 1;
  double lo[DSKI_MAXD] = {0, 0, 0}, hi[DSKI_MAXD] = {0, 0, 0}, h[DSKI_MAXD] = {1, 1, 1};
  double ell[DSKI_MAXD] = {1, 1, 1};
  double sf = 1.0, nv = 0.0, ng = 0.0;
  int prec = DSKI_FP64;
  // FP64_TC and FFT products: run the mode products as dense factors on the
  // FP64 units instead (the PCG's true residuals)
  bool kron_exact = false;
  cudaStream_t stream = nullptr;
  // private non-blocking stream for the captured PCG chunks (the legacy
  // default stream cannot be captured), ordered against `stream` by events
  cudaStream_t pstream = nullptr;
  cudaEvent_t pev_in = nullptr, pev_out = nullptr;
  int M = 0;        // grid size prod m_k
  int ncell = 0;    // prod mc_k
  int sm_count = 0;

  // geometry (sorted order); W64/W32: per point and dimension the sw
  // stencil weights then the sw derivative weights (already divided by h_k)
  dski::DevBuf perm, inv_perm, cell, cell_start, frac64, frac32, W64, W32;
  // FP64_TC, d = 2, cubic stencil: the W64 table as double-float pairs
  // (float2 {hi, lo}, hi = fl32(w), lo = fl32(w - hi)) for the scatter's
  // stencil products on the FP32 units
  dski::DevBuf Wdf;
  // Kronecker factors K_k (m_k x m_k, row-major, symmetric): FP64, FP32 and
  // the TF32 hi/lo split of the FP64 value (hi = rna_tf32(K), lo = rna_tf32(K - hi)).
  dski::DevBuf K64[DSKI_MAXD], K32[DSKI_MAXD], Khi[DSKI_MAXD], Klo[DSKI_MAXD];
  // dK_k / dlog l_k = K_k .* ((a - b) h_k)^2 / l_k^2 (FP64), for the gradient of Eq. 1
  dski::DevBuf dK64[DSKI_MAXD];
  // FP64_TC mode: eight BF16 digit planes of K_k (8 x m x m) and row exponents
  dski::DevBuf Kdig[DSKI_MAXD], Kexp[DSKI_MAXD];
  // Toeplitz/FFT products of K_UU (kuu_fft): per factor the twiddles
  // exp(-2 pi i j / L) (L/2 complex) and the circulant's spectrum / L (L
  // values, bit-reversed order)
  bool kuu_fft = false;
  dski::DevBuf fft_tw[DSKI_MAXD], fft_lam[DSKI_MAXD];
  // FP64_TC: split-K partial sums of the mode products (workspace)
  dski::DevBuf ozP;
  // PCG: per-block partial sums of the dots fused into other kernels
  dski::DevBuf s_dpart;
  // FP64 scatter: per-point sum-factorised coefficients (workspace)
  dski::DevBuf scat_ab;
  // workspace
  dski::DevBuf gridA, gridB, vin, vout, scratch;
  // solver workspace: reduction partials, last-block tickets (zeroed at
  // allocation), per-column scalar state and solver vectors
  dski::DevBuf s_part, s_tnpart, s_ticket, s_state, s_vec[13];
  // device error word (int): set by kernels whose bounded waits ran out
  dski::DevBuf dev_err;
  // polls of the first mbarrier wait of the tensor-core mode products
  // (dski_set_wait_budget; -1: the default budget)
  int wait_budget = -1;
  // stage timers (NULL unless profiling is on)
  dski::Profiler* prof = nullptr;
};

namespace dski {

// Geometry / factors (geom.cu)
int build_geometry(dski_handle h, const double* X_dev);
int build_factors(dski_handle h);

// MVM pieces (mvm.cu).  `prec64` selects the FP64 operator (double vectors)
// or the FP32 operator (float vectors, (3x)TF32 mode products per h->prec).
int mvm_internal(dski_handle h, const void* vin, void* vout, int s, bool prec64);
int permute_in(dski_handle h, const void* v_user, void* v_int, int s, bool f64, cudaStream_t st);
int permute_out(dski_handle h, const void* v_int, void* v_user, int s, bool f64, cudaStream_t st);
// grid-only pieces used by the adjoint: g = B^T v, and the Kronecker product
// with one factor optionally replaced by dK_k/dlog l_k (which = k) or none (which = -1).
int scatter_internal(dski_handle h, const void* vin, void* g, int s, bool prec64);
// as scatter_internal with the sum-factorised coefficients in caller memory
// `ws` (scatter_ws_bytes bytes; NULL = the handle's workspace)
int scatter_internal_ws(dski_handle h, const void* vin, void* g, int s, bool prec64, void* ws);
size_t scatter_ws_bytes(dski_handle h, int s, bool prec64);
// FP64_TC (d = 2, cubic, outside the true residuals): the scatter forms its
// stencil products in double-float arithmetic on the FP32 units (~2^-48
// relative) per cell, then adds the cells per node
bool df_scatter_path(dski_handle h, bool prec64);
// number of per-block partial sums of ||r||^2 (per column) that a scatter
// fused with a CG update (CgUpdate) writes
int scatter_update_blocks(dski_handle h);
// A CG update fused into the scatter's point pass (FP64, d >= 2, s <= 4):
// for every active column q, x += alpha_q p and r -= alpha_q q on the scattered
// vector r (written back) before it is scattered, and per-block partial sums
// of ||r||^2 to dpart[q nblocks + block] (nblocks = ceil(n / 256)).
struct CgUpdate {
  double* x = nullptr;   // NULL: no update
  const double* p = nullptr;
  const double* q = nullptr;
  const double* alpha = nullptr;
  const int* active = nullptr;
  double* dpart = nullptr;
};
// FP64 scatter of (sv v^0, sg v^1..d) (FP64, d >= 2, s <= 4 when scaled)
int scatter_scaled(dski_handle h, const void* vin, void* g, int s, bool prec64, void* ws,
                   double sv, double sg, const CgUpdate* up = nullptr);
// as scatter_scaled; with z != NULL first v <- z + beta_q v (written back)
int scatter_fused(dski_handle h, const void* vin, void* g, int s, bool prec64, void* ws,
                  double sv, double sg, const double* z, const double* beta,
                  const CgUpdate* up = nullptr);
// PCG: P <- Z + beta P fused into the FP64 MVM Q = K~ P (when pcg_fusable);
// with dpart, the gather leaves per-block partial sums of p^T q there
bool pcg_fusable(dski_handle h, int s);
struct CgFinish;   // a CG finisher folded into a gather (solve_internal.cuh)
int mvm_pcg_fused(dski_handle h, double* P, const double* Z, const double* beta, double* Q,
                  int s, double* dpart = nullptr, const CgFinish* fin = nullptr);
// FP64 gather: vout^0 = av (B grid)^0 + nv vin^0, vout^p = ag (B grid)^p + ng vin^p;
// with dpart, per-block partial sums of vin^T vout per column
// (dpart[q nblocks + block], nblocks = ceil(n / 256))
// grid_scratch: the grid is the caller's scratch, which FP64_TC (d = 2,
// cubic) may overwrite with its double-float split for the FP32-unit gather
int gather_scaled(dski_handle h, const double* grid, const double* vin, double* vout, int s,
                  double av, double ag, double nv, double ng, int stage, double* dpart = nullptr,
                  const CgFinish* fin = nullptr, bool grid_scratch = false);
// tc_ws: caller memory for the MIXED modes' tensor-core partials (the
// largest mode_tc_tf32_ws_bytes over the modes); NULL = the handle's workspace
int kron_internal(dski_handle h, void* g, void* tmp, int s, bool prec64, int dfactor,
                  const void* dK, void** result, void* tc_ws = nullptr);

// while on, the mode-product tile autotuner uses its heuristic (no timing, no
// events) on this thread -- for callers that must not create resources
void set_no_tune(bool on);

// gather stage alone: vout = B grid + noise .* vin (internal layout)
int gather_internal(dski_handle h, const void* grid, const void* vin, void* vout, int s,
                    bool prec64);

// Toeplitz mode products by FFT (kron_fft.cu): the per-factor multipliers
// (after the factors), and Y = scale K_k X with the contracted mode first
int fft_circulant_size(int m);
int fft_prepare(dski_handle h);
int mode_fft(dski_handle h, int k, const double* X, double* Y, long long R, int s, double scale);

// tensor-core mode product (kron_tc.cu): TF32 (three = false) or 3xTF32.
// ws: caller memory for the split contraction's FP32 partials
// (mode_tc_tf32_ws_bytes bytes); NULL = the handle's workspace, grown on demand
int mode_tc_tf32(dski_handle h, const float* X, const float* Khi, const float* Klo, float* Y,
                 int m, long long R, int s, float scale, bool three, float* ws = nullptr);
// bytes of split-contraction partials one mode_tc_tf32 call needs (0: none)
size_t mode_tc_tf32_ws_bytes(int m, long long R, int s);
// FP64_TC mode products (kron_tc.cu): digits and row exponents of a factor,
// and one mode product;
// a factor's digit planes take kOzDigits x m x m BF16 values
constexpr int kOzDigits = 8;
// smallest mode size whose FP64_TC products take the tensor cores
constexpr int kOzMinM = 64;
int oz_slice_factor(dski_handle h, const double* K, int m, uint16_t* Ad, int* fA);
int mode_tc_oz(dski_handle h, const double* X, const uint16_t* Ad, const int* fA, double* Y,
               int m, long long R, int s, double scale);
// General FP64-accurate product on the tensor cores:
//   Y_q[j][r] = scale sum_i A[j][i] xs_q[i] X_q[r][i]   (ytrans: Y_q[r][j])
// A: Mrows x mp as digit planes Ad (oz_slice) with row exponents fA; X_q:
// R rows of stride ldx (FP64, zero beyond the contraction), X_q = X + q xq;
// xs optional (xs_q = xs + q xsq, zero at i >= xsn); mp % 8 == 0, mp <= 256.
struct OzGemm {
  const uint16_t* Ad = nullptr;
  const int* fA = nullptr;
  int Mrows = 0, mp = 0;
  const double* X = nullptr;
  long long ldx = 0, xq = 0, R = 0;
  const double* xs = nullptr;
  long long xsq = 0;
  int xsn = 0;
  double* Y = nullptr;
  bool ytrans = false;
  double scale = 1.0;
  int s = 1;
  dski::DevBuf* workspace = nullptr;   // default: the handle's
};
int oz_gemm(dski_handle h, const OzGemm& g, int stage);
// digits of A (rows x cols, row stride lda) into Ad (row stride mp, zero padded)
int oz_slice(dski_handle h, const double* A, int rows, int cols, int lda, int mp, uint16_t* Ad,
             int* fA, int stage);
// vectors of this handle are double (FP64, FP64_TC) or float (MIXED modes)
inline bool f64_vectors(dski_handle h) { return h->prec == DSKI_FP64 || h->prec == DSKI_FP64_TC; }
// fn(std::integral_constant<int, S>{}) with S the handle's stencil width
template <class F>
auto with_stencil(dski_handle h, F&& fn) {
  if (h->sw == 6) return fn(std::integral_constant<int, 6>{});
  return fn(std::integral_constant<int, 4>{});
}
// true the first time it is called for the current device with this mask
// (one bit per device ordinal < 64): per-device, once-only set-up such as
// cudaFuncSetAttribute, which acts on the current device only
bool first_on_device(std::atomic<unsigned long long>* mask);
// read and clear the device error word: DSKI_OK, or DSKI_ERR_TIMEOUT if a
// kernel's bounded wait ran out since the last check (synchronises)
int check_device_error(dski_handle h);

// internal vector length
inline size_t nrows(dski_handle h) { return (size_t)h->N; }

}  // namespace dski
