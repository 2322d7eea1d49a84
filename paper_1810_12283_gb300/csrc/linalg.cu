// Tall-skinny FP64 linear algebra on the internal layout, used by the
// preconditioner build and apply of Sec. 3.3 and by the solvers:
//   ts_tn   C = A^T (w .* B)         (N x p)^T (N x q) -> p x q, split over rows
//   ts_nn   Y = r .* (alpha x .* X + beta A C)  (N x p)(p x q) -> N x q, row-parallel
//   col_dots, noise_diag, precond_apply.
// All reductions are deterministic (fixed-order partial sums).
#include <algorithm>

#include "solve_internal.cuh"

namespace dski {

double* wbuf(DevBuf& b, size_t count) {
  if (b.ensure(count * sizeof(double)) != DSKI_OK) {
    set_error(DSKI_ERR_ALLOC, "solver workspace allocation failed (%zu doubles)", count);
    return nullptr;
  }
  return b.as<double>();
}

namespace {

constexpr int TN_TP = 32;     // output tile rows (columns of A)
constexpr int TN_TQ = 8;      // output tile cols (columns of B)
constexpr int TN_SUB = 64;    // rows staged per sub-chunk

// partial[chunk][tp][tq] of A^T (w .* B) over one chunk of rows.
__global__ void __launch_bounds__(256) k_ts_tn(const double* __restrict__ A, int p,
                                               const double* __restrict__ B, int q,
                                               const double* __restrict__ w, long long N,
                                               int TN_CHUNK, double* __restrict__ part) {
  __shared__ double As[TN_SUB][TN_TP + 1];
  __shared__ double Bs[TN_SUB][TN_TQ + 1];
  const int t0 = blockIdx.y * TN_TP, u0 = blockIdx.z * TN_TQ;
  const long long r0 = (long long)blockIdx.x * TN_CHUNK;
  const long long r1 = min(N, r0 + TN_CHUNK);
  const int ti = threadIdx.x / TN_TQ, ui = threadIdx.x % TN_TQ;   // 32 x 8
  double acc = 0.0;
  for (long long rs = r0; rs < r1; rs += TN_SUB) {
    for (int idx = threadIdx.x; idx < TN_SUB * TN_TP; idx += 256) {
      const int rr = idx % TN_SUB, tt = idx / TN_SUB;
      const long long row = rs + rr;
      As[rr][tt] = (row < r1 && t0 + tt < p) ? A[(long long)(t0 + tt) * N + row] : 0.0;
    }
    for (int idx = threadIdx.x; idx < TN_SUB * TN_TQ; idx += 256) {
      const int rr = idx % TN_SUB, uu = idx / TN_SUB;
      const long long row = rs + rr;
      double v = 0.0;
      if (row < r1 && u0 + uu < q) {
        v = B[(long long)(u0 + uu) * N + row];
        if (w) v *= w[row];
      }
      Bs[rr][uu] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < TN_SUB; ++rr) acc = fma(As[rr][ti], Bs[rr][ui], acc);
    __syncthreads();
  }
  const int t = t0 + ti, u = u0 + ui;
  if (t < p && u < q) part[((long long)blockIdx.x * p + t) * q + u] = acc;
}

// C = A^T (w .* B) for few columns q <= QMAX (the PCG's Q1^T y): each block
// owns GV_ROWS rows, each thread GV_RPT of them with its B values held in
// registers; A's columns are streamed once, 8 at a time, and the 8 x q
// per-thread sums are reduced over the block in a fixed order.
constexpr int GV_RPT = 4;
constexpr int GV_ROWS = 256 * GV_RPT;
constexpr int GV_TG = 8;
template <int QMAX>
__global__ void __launch_bounds__(256) k_gemv_t(const double* __restrict__ A, int p,
                                                const double* __restrict__ B, int q,
                                                const double* __restrict__ w, long long N,
                                                double* __restrict__ part) {
  __shared__ double red[8][GV_TG * QMAX];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long base = (long long)blockIdx.x * GV_ROWS;
  double bv[GV_RPT][QMAX];
#pragma unroll
  for (int k = 0; k < GV_RPT; ++k) {
    const long long row = base + k * 256 + threadIdx.x;
#pragma unroll
    for (int u = 0; u < QMAX; ++u) {
      double v = 0.0;
      if (row < N && u < q) {
        v = B[(long long)u * N + row];
        if (w) v *= w[row];
      }
      bv[k][u] = v;
    }
  }
  for (int t0 = 0; t0 < p; t0 += GV_TG) {
    double acc[GV_TG][QMAX];
#pragma unroll
    for (int tt = 0; tt < GV_TG; ++tt)
#pragma unroll
      for (int u = 0; u < QMAX; ++u) acc[tt][u] = 0.0;
#pragma unroll
    for (int k = 0; k < GV_RPT; ++k) {
      const long long row = base + k * 256 + threadIdx.x;
      if (row < N) {
#pragma unroll
        for (int tt = 0; tt < GV_TG; ++tt) {
          const double a = (t0 + tt < p) ? A[(long long)(t0 + tt) * N + row] : 0.0;
#pragma unroll
          for (int u = 0; u < QMAX; ++u) acc[tt][u] = fma(a, bv[k][u], acc[tt][u]);
        }
      }
    }
#pragma unroll
    for (int tt = 0; tt < GV_TG; ++tt)
#pragma unroll
      for (int u = 0; u < QMAX; ++u) {
        const double v = warp_sum(acc[tt][u]);
        if (lane == 0) red[warp][tt * QMAX + u] = v;
      }
    __syncthreads();
    if (threadIdx.x < GV_TG * QMAX) {
      const int tt = threadIdx.x / QMAX, u = threadIdx.x % QMAX;
      double v = 0.0;
#pragma unroll
      for (int wv = 0; wv < 8; ++wv) v += red[wv][threadIdx.x];
      if (t0 + tt < p && u < q) part[((long long)blockIdx.x * p + t0 + tt) * q + u] = v;
    }
    __syncthreads();
  }
}

// As k_gemv_t with A = Qh + Ql held as two FP32 arrays and every product and
// sum taken in double-float arithmetic on the FP32 units; one FP64 value per
// block and output at the end.
template <int QMAX>
__global__ void __launch_bounds__(256) k_df_gemv_t(const float* __restrict__ Qh,
                                                   const float* __restrict__ Ql, int p,
                                                   const double* __restrict__ B, int q,
                                                   const double* __restrict__ w, long long N,
                                                   double* __restrict__ part) {
  __shared__ float red[2][8][GV_TG * QMAX];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long base = (long long)blockIdx.x * GV_ROWS;
  float bh[GV_RPT][QMAX], bl[GV_RPT][QMAX];
#pragma unroll
  for (int k = 0; k < GV_RPT; ++k) {
    const long long row = base + k * 256 + threadIdx.x;
#pragma unroll
    for (int u = 0; u < QMAX; ++u) {
      double v = 0.0;
      if (row < N && u < q) {
        v = B[(long long)u * N + row];
        if (w) v *= w[row];
      }
      split_d(v, bh[k][u], bl[k][u]);
    }
  }
  for (int t0 = 0; t0 < p; t0 += GV_TG) {
    float sh[GV_TG][QMAX], sl[GV_TG][QMAX];
#pragma unroll
    for (int tt = 0; tt < GV_TG; ++tt)
#pragma unroll
      for (int u = 0; u < QMAX; ++u) sh[tt][u] = sl[tt][u] = 0.f;
#pragma unroll
    for (int k = 0; k < GV_RPT; ++k) {
      const long long row = base + k * 256 + threadIdx.x;
      if (row < N) {
#pragma unroll
        for (int tt = 0; tt < GV_TG; ++tt) {
          const bool in = t0 + tt < p;
          const float qh = in ? Qh[(long long)(t0 + tt) * N + row] : 0.f;
          const float ql = in ? Ql[(long long)(t0 + tt) * N + row] : 0.f;
#pragma unroll
          for (int u = 0; u < QMAX; ++u) df_fma(qh, ql, bh[k][u], bl[k][u], sh[tt][u], sl[tt][u]);
        }
      }
    }
    // warp tree in double-float, fixed order
#pragma unroll
    for (int tt = 0; tt < GV_TG; ++tt)
#pragma unroll
      for (int u = 0; u < QMAX; ++u) {
        float a = sh[tt][u], b = sl[tt][u];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float oa = __shfl_xor_sync(0xffffffffu, a, o);
          const float ob = __shfl_xor_sync(0xffffffffu, b, o);
          df_add(a, b, oa, ob);
        }
        if (lane == 0) {
          red[0][warp][tt * QMAX + u] = a;
          red[1][warp][tt * QMAX + u] = b;
        }
      }
    __syncthreads();
    if (threadIdx.x < GV_TG * QMAX) {
      const int tt = threadIdx.x / QMAX, u = threadIdx.x % QMAX;
      float a = 0.f, b = 0.f;
#pragma unroll
      for (int wv = 0; wv < 8; ++wv) df_add(a, b, red[0][wv][threadIdx.x], red[1][wv][threadIdx.x]);
      if (t0 + tt < p && u < q)
        part[((long long)blockIdx.x * p + t0 + tt) * q + u] = (double)a + (double)b;
    }
    __syncthreads();
  }
}

__global__ void k_qsplit(const double* __restrict__ Q, long long count, float* __restrict__ Qh,
                         float* __restrict__ Ql) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    float h, l;
    split_d(Q[i], h, l);
    Qh[i] = h;
    Ql[i] = l;
  }
}

// C = A^T (w .* b) for ONE column (the solve's Q1^T y) in FP64: a block owns
// GT_ROWS rows with w .* b staged in shared memory; warp w owns the outputs
// t = w, w + 8, ...; for each, its lanes sweep the rows (coalesced, 8 loads in
// flight) and a single warp reduction ends the output -- so the FP64
// reduction work is ~1/16 of the FP64 FMAs (on GB300 FP64 adds are as slow
// as FMAs).
constexpr int GT_ROWS = 2048;
__global__ void __launch_bounds__(256) k_gemv_t1(const double* __restrict__ A, int p,
                                                 const double* __restrict__ b,
                                                 const double* __restrict__ w, long long N,
                                                 double* __restrict__ part) {
  __shared__ double ys[GT_ROWS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long r0 = (long long)blockIdx.x * GT_ROWS;
  const int nr = (int)min((long long)GT_ROWS, N - r0);
  for (int i = threadIdx.x; i < GT_ROWS; i += 256) {
    double v = 0.0;
    if (i < nr) {
      v = b[r0 + i];
      if (w) v *= w[r0 + i];
    }
    ys[i] = v;
  }
  __syncthreads();
  for (int t = warp; t < p; t += 8) {
    const double* at = A + (long long)t * N + r0;
    double acc = 0.0;
    for (int i0 = 0; i0 < nr; i0 += 32 * 8) {
      double a[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int i = i0 + k * 32 + lane;
        a[k] = i < nr ? at[i] : 0.0;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) acc = fma(a[k], ys[i0 + k * 32 + lane], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) part[(long long)blockIdx.x * p + t] = acc;
  }
}

// One warp per output: lane l adds chunks l, l + 32, ... then a fixed tree.
__global__ void k_sum_chunks(const double* __restrict__ part, int nchunk, int pq,
                             double* __restrict__ out) {
  const int idx = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (idx >= pq) return;
  double s = 0.0;
  for (int c = lane; c < nchunk; c += 32) s += part[(long long)c * pq + idx];
  s = warp_sum(s);
  if (lane == 0) out[idx] = s;
}

// Y[:, u] = rowscale .* (alpha xscale .* X[:, u] + beta sum_t A[:, t] C[t, u])
template <int QB>
__global__ void __launch_bounds__(256) k_ts_nn(const double* __restrict__ X, double alpha,
                                               const double* __restrict__ xscale, double beta,
                                               const double* __restrict__ A, int p,
                                               const double* __restrict__ C, int q,
                                               double* __restrict__ Y,
                                               const double* __restrict__ rowscale,
                                               long long N) {
  extern __shared__ double Cs[];   // p x q
  for (int i = threadIdx.x; i < p * q; i += blockDim.x) Cs[i] = beta * C[i];
  __syncthreads();
  const int u0 = blockIdx.y * QB;
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < N;
       row += (long long)gridDim.x * blockDim.x) {
    double acc[QB];
    const double xs = xscale ? alpha * xscale[row] : alpha;
#pragma unroll
    for (int u = 0; u < QB; ++u)
      acc[u] = (X && u0 + u < q) ? xs * X[(long long)(u0 + u) * N + row] : 0.0;
    for (int t = 0; t < p; ++t) {
      const double a = A[(long long)t * N + row];
#pragma unroll
      for (int u = 0; u < QB; ++u)
        if (u0 + u < q) acc[u] = fma(a, Cs[t * q + u0 + u], acc[u]);
    }
    const double sc = rowscale ? rowscale[row] : 1.0;
#pragma unroll
    for (int u = 0; u < QB; ++u)
      if (u0 + u < q) Y[(long long)(u0 + u) * N + row] = sc * acc[u];
  }
}

__global__ void k_col_dots(const double* __restrict__ a, const double* __restrict__ b,
                           long long N, int s, double* __restrict__ part,
                           unsigned* __restrict__ ticket, double* __restrict__ out) {
  __shared__ double sh[32];
  const int q = blockIdx.y;
  double v = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    v = fma(a[(long long)q * N + i], b[(long long)q * N + i], v);
  v = block_sum(v, sh);
  if (threadIdx.x == 0) part[(long long)q * gridDim.x + blockIdx.x] = v;
  if (last_block(ticket, gridDim.x * gridDim.y)) {
    for (int c = threadIdx.x; c < s; c += blockDim.x) {
      double t = 0.0;
      for (unsigned bx = 0; bx < gridDim.x; ++bx) t += part[(long long)c * gridDim.x + bx];
      out[c] = t;
    }
  }
}

__global__ void k_noise_diag(int n, int d, double nv, double ng, double* __restrict__ D) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * (d + 1)) return;
  D[e] = (e % (d + 1)) == 0 ? nv : ng;
}

}  // namespace

int ts_tn(dski_handle h, const double* A, int p, const double* B, int q, const double* w,
          double* C_dev) {
  const long long N = h->N;
  if (q == 1) {
    const int nchunk = (int)((N + GT_ROWS - 1) / GT_ROWS);
    double* part = wbuf(h->s_tnpart, (size_t)nchunk * p);
    if (!part) return DSKI_ERR_ALLOC;
    StageScope sc(h, ST_PRECOND, h->stream, 2);
    k_gemv_t1<<<nchunk, 256, 0, h->stream>>>(A, p, B, w, N, part);
    k_sum_chunks<<<(p + 7) / 8, 256, 0, h->stream>>>(part, nchunk, p, C_dev);
    DSKI_LAUNCHED();
    return DSKI_OK;
  }
  if (q <= 4) {
    const int nchunk = (int)((N + GV_ROWS - 1) / GV_ROWS);
    double* part = wbuf(h->s_tnpart, (size_t)nchunk * p * q);
    if (!part) return DSKI_ERR_ALLOC;
    StageScope sc(h, ST_PRECOND, h->stream, 2);
    if (q == 1)
      k_gemv_t<1><<<nchunk, 256, 0, h->stream>>>(A, p, B, q, w, N, part);
    else
      k_gemv_t<4><<<nchunk, 256, 0, h->stream>>>(A, p, B, q, w, N, part);
    k_sum_chunks<<<(p * q + 7) / 8, 256, 0, h->stream>>>(part, nchunk, p * q, C_dev);
    DSKI_LAUNCHED();
    return DSKI_OK;
  }
  // rows per chunk: enough blocks to fill the GPU twice, at least one sub-chunk
  const int tiles = ((p + TN_TP - 1) / TN_TP) * ((q + TN_TQ - 1) / TN_TQ);
  long long rows = (N + 2LL * h->sm_count * tiles - 1) / (2LL * h->sm_count * tiles);
  rows = std::max<long long>(TN_SUB, (rows + TN_SUB - 1) / TN_SUB * TN_SUB);
  const int chunk = (int)std::min<long long>(rows, 1 << 20);
  const int nchunk = (int)((N + chunk - 1) / chunk);
  double* part = wbuf(h->s_tnpart, (size_t)nchunk * p * q);   // own buffer: callers hold s_part
  if (!part) return DSKI_ERR_ALLOC;
  dim3 grd(nchunk, (p + TN_TP - 1) / TN_TP, (q + TN_TQ - 1) / TN_TQ);
  {
    StageScope sc(h, ST_PRECOND, h->stream, 2);
    k_ts_tn<<<grd, 256, 0, h->stream>>>(A, p, B, q, w, N, chunk, part);
    k_sum_chunks<<<(p * q + 7) / 8, 256, 0, h->stream>>>(part, nchunk, p * q, C_dev);
  }
  DSKI_LAUNCHED();
  return DSKI_OK;
}

int ts_nn(dski_handle h, const double* X, double alpha, const double* xscale, double beta,
          const double* A, int p, const double* C, int q, double* Y, const double* rowscale) {
  const long long N = h->N;
  const size_t smem = (size_t)p * q * sizeof(double);
  // C is staged in shared memory: up to 200 KB (GB300: 227 KB per block),
  // which holds the 128 x 128 factor of a rank-128 preconditioner
  if (smem > 200 * 1024) return set_error(DSKI_ERR_ARG, "ts_nn: p*q too large (%d x %d)", p, q);
  const int nbx = (int)std::min<long long>((N + 255) / 256, 4LL * h->sm_count);
  StageScope sc(h, ST_PRECOND, h->stream);
  if (q <= 4) {
    dim3 grd(nbx, (q + 3) / 4);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_ts_nn<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_ts_nn<4><<<grd, 256, smem, h->stream>>>(X, alpha, xscale, beta, A, p, C, q, Y, rowscale, N);
  } else {
    dim3 grd(nbx, (q + 7) / 8);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_ts_nn<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_ts_nn<8><<<grd, 256, smem, h->stream>>>(X, alpha, xscale, beta, A, p, C, q, Y, rowscale, N);
  }
  DSKI_LAUNCHED();
  return DSKI_OK;
}

int df_gemv_t(dski_handle h, const float* Qh, const float* Ql, int p, const double* B, int q,
              const double* w, double* C_dev) {
  const long long N = h->N;
  if (q > 4) return set_error(DSKI_ERR_ARG, "df_gemv_t: at most 4 columns per call");
  const int nchunk = (int)((N + GV_ROWS - 1) / GV_ROWS);
  double* part = wbuf(h->s_tnpart, (size_t)nchunk * p * q);
  if (!part) return DSKI_ERR_ALLOC;
  StageScope sc(h, ST_PRECOND, h->stream, 2);
  if (q == 1)
    k_df_gemv_t<1><<<nchunk, 256, 0, h->stream>>>(Qh, Ql, p, B, q, w, N, part);
  else
    k_df_gemv_t<4><<<nchunk, 256, 0, h->stream>>>(Qh, Ql, p, B, q, w, N, part);
  k_sum_chunks<<<(p * q + 7) / 8, 256, 0, h->stream>>>(part, nchunk, p * q, C_dev);
  DSKI_LAUNCHED();
  return DSKI_OK;
}

int split_q1(dski_handle h, pivchol_handle pc) {
  const size_t cnt = (size_t)pc->N * pc->rank;
  if (pc->Qh.ensure(cnt * 4) || pc->Ql.ensure(cnt * 4))
    return set_error(DSKI_ERR_ALLOC, "pivchol_build: allocation of the split Q1 failed");
  StageScope sc(h, ST_PIVCHOL, h->stream);
  k_qsplit<<<4 * h->sm_count, 256, 0, h->stream>>>(pc->Q1.as<double>(), (long long)cnt,
                                                   pc->Qh.as<float>(), pc->Ql.as<float>());
  DSKI_LAUNCHED();
  pc->split = true;
  return DSKI_OK;
}

// Z = D^-1/2 (Y - Q1 C), Y = D^-1/2 R, with the split Q1 (double-float).
__global__ void k_df_z(const double* __restrict__ R, const float* __restrict__ Qh,
                       const float* __restrict__ Ql, int rank, const double* __restrict__ C,
                       int s, const double* __restrict__ dis, double* __restrict__ Z,
                       long long N) {
  extern __shared__ float Cs2[];   // rank hi, rank lo
  const int c = blockIdx.y;
  for (int t = threadIdx.x; t < rank; t += blockDim.x) split_d(C[(long long)t * s + c], Cs2[t], Cs2[rank + t]);
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    float sh = 0.f, sl = 0.f;
    for (int t = 0; t < rank; ++t)
      df_fma(Qh[(long long)t * N + i], Ql[(long long)t * N + i], Cs2[t], Cs2[rank + t], sh, sl);
    const double y = dis[i] * R[(long long)c * N + i];
    Z[(long long)c * N + i] = dis[i] * ((y - (double)sh) - (double)sl);
  }
}

unsigned* tickets(dski_handle h, int count) {
  // Tickets are zeroed once at allocation; every user leaves them at zero.
  const size_t need = (size_t)count * sizeof(unsigned);
  if (h->s_ticket.bytes < need || !h->s_ticket.ptr) {
    h->s_ticket.release();
    if (h->s_ticket.ensure(std::max<size_t>(need, 4096)) != DSKI_OK) return nullptr;
    if (cudaMemsetAsync(h->s_ticket.ptr, 0, h->s_ticket.bytes, h->stream) != cudaSuccess)
      return nullptr;
  }
  return h->s_ticket.as<unsigned>();
}

int col_dots(dski_handle h, const double* a, const double* b, int s, double* out_dev,
             long long len) {
  const long long N = len > 0 ? len : h->N;
  const int nbx = (int)std::min<long long>((N + 1023) / 1024, 2LL * h->sm_count);
  double* part = wbuf(h->s_part, (size_t)nbx * s);
  unsigned* tk = tickets(h, 1);
  if (!part || !tk) return set_error(DSKI_ERR_ALLOC, "col_dots: workspace allocation failed");
  StageScope sc(h, ST_PCGVEC, h->stream);
  k_col_dots<<<dim3(nbx, s), 256, 0, h->stream>>>(a, b, N, s, part, tk, out_dev);
  DSKI_LAUNCHED();
  return DSKI_OK;
}

int precond_apply(dski_handle h, pivchol_handle pc, const double* R, double* Z, int s) {
  if (pc->grid_form) return grid_precond_apply(h, pc, R, Z, s);
  if (pc->split && pc->rank > 0) {
    double* C = wbuf(h->s_vec[5], (size_t)pc->rank * 4);
    if (!C) return DSKI_ERR_ALLOC;
    for (int c0 = 0; c0 < s; c0 += 4) {
      const int q = std::min(4, s - c0);
      const long long off = (long long)c0 * h->N;
      DSKI_TRY(df_gemv_t(h, pc->Qh.as<float>(), pc->Ql.as<float>(), pc->rank, R + off, q,
                         pc->dis.as<double>(), C));
      StageScope sc(h, ST_PRECOND, h->stream);
      const int nbx = (int)std::min<long long>((h->N + 255) / 256, 4LL * h->sm_count);
      k_df_z<<<dim3(nbx, q), 256, 2 * pc->rank * sizeof(float), h->stream>>>(
          R + off, pc->Qh.as<float>(), pc->Ql.as<float>(), pc->rank, C, q, pc->dis.as<double>(),
          Z + off, h->N);
      DSKI_LAUNCHED();
    }
    return DSKI_OK;
  }
  if (pc->rank == 0) {
    // M = D: Z = D^-1 R
    return ts_nn(h, R, 1.0, pc->dis.as<double>(), 0.0, nullptr, 0, nullptr, s, Z,
                 pc->dis.as<double>());
  }
  double* C = wbuf(h->s_vec[5], (size_t)pc->rank * s);
  if (!C) return DSKI_ERR_ALLOC;
  DSKI_TRY(ts_tn(h, pc->Q1.as<double>(), pc->rank, R, s, pc->dis.as<double>(), C));
  // Z = D^-1/2 (D^-1/2 R - Q1 C)
  return ts_nn(h, R, 1.0, pc->dis.as<double>(), -1.0, pc->Q1.as<double>(), pc->rank, C, s, Z,
               pc->dis.as<double>());
}

int noise_diag(dski_handle h, double nv, double ng, double* D_dev) {
  StageScope sc(h, ST_PCGVEC, h->stream);
  k_noise_diag<<<(unsigned)((h->N + 255) / 256), 256, 0, h->stream>>>(h->n, h->d, nv, ng, D_dev);
  DSKI_LAUNCHED();
  return DSKI_OK;
}

}  // namespace dski
