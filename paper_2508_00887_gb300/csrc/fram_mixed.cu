// Mixed-precision outer loop of FRAM (Alg. 1 of arXiv 2508.00887 with the
// precision split of Sec. 6 "Mixed-precision architecture"):
//
//   step 5  X = A N B (+ lambda K)   tcgen05 tensor cores, BF16 or TF32
//                                    operands, FP32 accumulation
//   step 6  D = SDSN(X, theta)       FP32 sweeps (Thm. 7: truncation residuals
//                                    of the sweep are projected away), then a
//                                    short FP64 polish of the last sweeps when
//                                    the residual gamma still exceeds polish_tol
//   step 7  N = (1 - alpha) N + alpha D          FP64
//   step 8  delta                                FP64
//   step 10 discretisation and objective         FP64 (shared with the FP64 path)
//
// Sweep budget: the FP32 phase runs at most max_sweeps - max_polish sweeps
// and stops early at gamma <= polish_tol; the FP64 polish then runs at most
// max_polish sweeps (stopping at gamma <= gamma_tol), so a capped solve does
// the same number of sweeps as the FP64 path.
//
// The update kernel also writes the next GEMM's low-precision operand: N^T in
// BF16 (or TF32-rounded FP32), so that both GEMM operands are K-major.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include "fram_ctx.h"
#include "fram_tc.h"

namespace fram {

namespace {

constexpr int kT = 32;  // transpose tile

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <int KIND>
__device__ __forceinline__ void store_lp(void* base, size_t idx, double v) {
  if (KIND == 0)
    static_cast<__nv_bfloat16*>(base)[idx] = __double2bfloat16(v);
  else
    static_cast<float*>(base)[idx] = tf32_round((float)v);
}

// dst (ld x ld, low precision) = src (ld x ld FP64).  Padding stays zero
// because src padding is zero.
template <int KIND>
__global__ void convert_kernel(const double* __restrict__ src, void* __restrict__ dst, size_t count) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x)
    store_lp<KIND>(dst, e, src[e]);
}

// dst[j][i] = lp(src[i][j]) over the full ld x ld square.
template <int KIND>
__global__ void transpose_lp_kernel(const double* __restrict__ src, void* __restrict__ dst, int ld) {
  __shared__ double tile[kT][kT + 1];
  const int tiles = ld / kT;
  for (int t = blockIdx.x; t < tiles * tiles; t += gridDim.x) {
    const int i0 = (t / tiles) * kT, j0 = (t % tiles) * kT;
    for (int r = threadIdx.y; r < kT; r += blockDim.y)
      tile[r][threadIdx.x] = src[(size_t)(i0 + r) * ld + j0 + threadIdx.x];
    __syncthreads();
    for (int r = threadIdx.y; r < kT; r += blockDim.y)
      store_lp<KIND>(dst, (size_t)(j0 + r) * ld + i0 + threadIdx.x, tile[threadIdx.x][r]);
    __syncthreads();
  }
}

// Alg. 1 steps 7-8 in FP64 on the n x n block, plus the transposed
// low-precision copy of the new N for the next gradient.  Deterministic
// delta: fixed tile ownership, fixed reduction trees, last-block combine.
// The update is written N + alpha (D - N), the same value as (1 - alpha) N +
// alpha D in exact arithmetic, and N_new - N = alpha (D - N), so that
// ||N_new - N||^2 = alpha^2 sum (D - N)^2: per element one subtraction and
// three FMAs instead of six FP64 operations (GB300's FP64 pipe bounds this
// kernel).
template <int KIND>
__device__ __forceinline__ void update_mixed_body(double* __restrict__ N,
                                                  const double* __restrict__ D, int ld, int n,
                                                  double alpha, void* __restrict__ Nt,
                                                  double* __restrict__ partials, unsigned* ticket,
                                                  IterStats* st, const int blk, const int nblk) {
  __shared__ double tile[kT][kT + 1];
  __shared__ double red[2][8];
  __shared__ int s_last;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const int tiles = (n + kT - 1) / kT;
  double d2 = 0.0, n2 = 0.0;
  for (int t = blk; t < tiles * tiles; t += nblk) {
    const int i0 = (t / tiles) * kT, j0 = (t % tiles) * kT;
    for (int r = ty; r < kT; r += 8) {
      const int i = i0 + r, j = j0 + tx;
      double nn = 0.0;
      if (i < n && j < n) {
        const size_t e = (size_t)i * ld + j;
        const double old = N[e];
        const double t = __dsub_rn(D[e], old);
        nn = __fma_rn(alpha, t, old);
        N[e] = nn;
        d2 = fma(t, t, d2);
        n2 = fma(nn, nn, n2);
      }
      tile[r][tx] = nn;
    }
    __syncthreads();
    for (int r = ty; r < kT; r += 8) {
      const int j = j0 + r, i = i0 + tx;
      if (i < n && j < n) store_lp<KIND>(Nt, (size_t)j * ld + i, tile[tx][r]);
    }
    __syncthreads();
  }
  d2 = warp_sum(d2);
  n2 = warp_sum(n2);
  const int warp = (ty * 32 + tx) >> 5, lane = tx;
  if (lane == 0) {
    red[0][warp] = d2;
    red[1][warp] = n2;
  }
  __syncthreads();
  if (warp == 0) {
    double a = lane < 8 ? red[0][lane] : 0.0, b = lane < 8 ? red[1][lane] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
      partials[2 * blk] = a;
      partials[2 * blk + 1] = b;
      __threadfence();
      s_last = (atomicAdd(ticket, 1u) == nblk - 1);
    }
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  {
    // All 256 threads of the last block read the partials (fixed stride,
    // fixed tree): one round of L2 latency instead of nblk / 32 in a row.
    const int tid = ty * 32 + tx;
    double a = 0.0, b = 0.0;
#pragma unroll 4
    for (int k = tid; k < nblk; k += 256) {
      a += __ldcg(&partials[2 * k]);
      b += __ldcg(&partials[2 * k + 1]);
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
      red[0][warp] = a;
      red[1][warp] = b;
    }
  }
  __syncthreads();
  if (warp == 0) {
    double a = lane < 8 ? red[0][lane] : 0.0, b = lane < 8 ? red[1][lane] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
      st->sum_d2 = alpha * alpha * a;
      st->sum_n2 = b;
      st->delta = alpha * sqrt(a) / sqrt(b);
      *ticket = 0u;
    }
  }
}

template <int KIND>
__global__ void __launch_bounds__(256) update_mixed_kernel(double* __restrict__ N,
                                                           const double* __restrict__ D, int ld,
                                                           int n, double alpha,
                                                           void* __restrict__ Nt,
                                                           double* __restrict__ partials,
                                                           unsigned* ticket, IterStats* st) {
  update_mixed_body<KIND>(N, D, ld, n, alpha, Nt, partials, ticket, st, (int)blockIdx.x,
                          (int)gridDim.x);
}

// The updates of many problems in one launch: problem q owns CTAs
// [blk0_q, blk0_q + nblk_q), the same number its solo launch uses, and each
// of those CTAs runs exactly what the solo CTA of that index runs (same
// tiles, same reduction tree), so N and delta are bit-identical to solo.
template <int KIND>
__global__ void __launch_bounds__(256) update_mixed_group_kernel(const UpdGroupProblem* probs,
                                                                 int nprob) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].blk0 <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const UpdGroupProblem& q = probs[lo];
  update_mixed_body<KIND>(q.N, q.D, q.ld, q.n, q.alpha, q.Nt, q.partials, q.ticket, q.st,
                          (int)blockIdx.x - q.blk0, q.nblk);
}

int update_grid(int n) {
  const int tiles = ((n + kT - 1) / kT) * ((n + kT - 1) / kT);
  return tiles < 1184 ? tiles : 1184;
}

int blocks_for(size_t count) {
  size_t b = (count + 255) / 256;
  return (int)(b < 2368 ? (b < 1 ? 1 : b) : 2368);
}

}  // namespace

// Buffers of the mixed path, each ld x ld x 4 bytes: A, B, N^T, T (low
// precision) and X/Y in FP32.
size_t mixed_bytes_for(int n) {
  const size_t ld = round_ld(n);
  return 5 * ld * ld * 4;
}

struct MixedBufs {
  void *A, *B, *Nt, *T;
  float* X32;
};

static MixedBufs carve_mixed(void* base, int ld) {
  const size_t m = (size_t)ld * ld * 4;
  char* p = static_cast<char*>(base);
  return MixedBufs{p, p + m, p + 2 * m, p + 3 * m, reinterpret_cast<float*>(p + 4 * m)};
}

int launch_convert_lp(const double* src, void* dst, int ld, int kind, cudaStream_t s) {
  const size_t count = (size_t)ld * ld;
  if (kind == 0)
    convert_kernel<0><<<blocks_for(count), 256, 0, s>>>(src, dst, count);
  else
    convert_kernel<1><<<blocks_for(count), 256, 0, s>>>(src, dst, count);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_transpose_lp(const double* src, void* dst, int ld, int kind, cudaStream_t s) {
  const int tiles = (ld / kT) * (ld / kT);
  const int grid = tiles < 1184 ? tiles : 1184;
  if (kind == 0)
    transpose_lp_kernel<0><<<grid, dim3(32, 8), 0, s>>>(src, dst, ld);
  else
    transpose_lp_kernel<1><<<grid, dim3(32, 8), 0, s>>>(src, dst, ld);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_update_mixed_group(UpdGroupProblem* hp, int count, int kind, void* dp,
                              size_t dp_bytes, cudaStream_t s) {
  if (count < 1) return 0;
  if ((size_t)count * sizeof(UpdGroupProblem) > dp_bytes) return -1;
  int total = 0;
  for (int q = 0; q < count; ++q) {
    hp[q].blk0 = total;
    hp[q].nblk = update_grid(hp[q].n);
    total += hp[q].nblk;
  }
  if (cudaMemcpyAsync(dp, hp, (size_t)count * sizeof(UpdGroupProblem), cudaMemcpyHostToDevice,
                      s) != cudaSuccess)
    return -1;
  const UpdGroupProblem* d = static_cast<const UpdGroupProblem*>(dp);
  if (kind == 0)
    update_mixed_group_kernel<0><<<total, dim3(32, 8), 0, s>>>(d, count);
  else
    update_mixed_group_kernel<1><<<total, dim3(32, 8), 0, s>>>(d, count);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_update_mixed(double* N, const double* D, int ld, int n, double alpha, void* Nt,
                        int kind, double* partials, unsigned* ticket, IterStats* st,
                        cudaStream_t s) {
  const int grid = update_grid(n);
  if (kind == 0)
    update_mixed_kernel<0><<<grid, dim3(32, 8), 0, s>>>(N, D, ld, n, alpha, Nt, partials, ticket,
                                                        st);
  else
    update_mixed_kernel<1><<<grid, dim3(32, 8), 0, s>>>(N, D, ld, n, alpha, Nt, partials, ticket,
                                                        st);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

#define MX_CUDA(x, what)                                     \
  do {                                                       \
    cudaError_t _e = (x);                                    \
    if (_e != cudaSuccess) return cuda_fail(c, _e, what);    \
  } while (0)
#define MX_LAUNCH(x, what)                                            \
  do {                                                                \
    int _k = (x);                                                     \
    if (_k < 0) return cuda_fail(c, cudaGetLastError(), what);        \
    c->launches += (uint64_t)_k;                                      \
  } while (0)

// Gradient only (step-level entry): operands already in ws.As/Bs/N (FP64,
// padded), result FP32 in the mixed X buffer.
fram_status mixed_gradient(fram_ctx* c, int n, bool has_K, double lam, int kind, float** X32) {
  Workspace& w = c->ws;
  const int ld = round_ld(n);
  MixedBufs b = carve_mixed(w.mixed, ld);
  MX_LAUNCH(launch_convert_lp(w.As, b.A, ld, kind, c->stream), "convert");
  MX_LAUNCH(launch_convert_lp(w.Bs, b.B, ld, kind, c->stream), "convert");
  MX_LAUNCH(launch_transpose_lp(w.N, b.Nt, ld, kind, c->stream), "transpose");
  MX_CUDA(cudaMemsetAsync(&w.scal->iter.gemm_err, 0, sizeof(int), c->stream), "memset");
  MX_LAUNCH(launch_gemm_tc(b.A, b.Nt, b.T, ld, n, kind, kind == 0 ? 1 : 2, nullptr, 0.0, nullptr,
                           &w.scal->iter.gemm_err, c->wait_limit_ns, c->stream),
            "tensor-core gemm");
  MX_LAUNCH(launch_gemm_tc(b.T, b.B, b.X32, ld, n, kind, 0, has_K ? w.Ks : nullptr, lam, nullptr,
                           &w.scal->iter.gemm_err, c->wait_limit_ns, c->stream),
            "tensor-core gemm");
  *X32 = b.X32;
  return FRAM_OK;
}

fram_status solve_mixed_loop(fram_ctx* c, int n, bool has_K, const fram_params& p,
                             fram_info* inf) {
  Workspace& w = c->ws;
  const int ld = round_ld(n);
  const int kind = p.precision == FRAM_PREC_MIXED_BF16 ? 0 : 1;
  MixedBufs b = carve_mixed(w.mixed, ld);
  MX_LAUNCH(launch_convert_lp(w.As, b.A, ld, kind, c->stream), "convert");
  MX_LAUNCH(launch_convert_lp(w.Bs, b.B, ld, kind, c->stream), "convert");
  MX_LAUNCH(launch_transpose_lp(w.N, b.Nt, ld, kind, c->stream), "transpose");
  const int cap32 = p.max_sweeps - p.max_polish > 1 ? p.max_sweeps - p.max_polish : 1;
  const double tol32 = p.polish_tol > p.gamma_tol ? p.polish_tol : p.gamma_tol;
  double prev_delta = INFINITY;

  static_assert(offsetof(DevScalars, xmax_key) == offsetof(DevScalars, iter) + sizeof(IterStats),
                "iteration stats and max key are cleared together");
  for (int t = 0; t < p.max_outer; ++t) {
    MX_CUDA(cudaMemsetAsync(&w.scal->iter, 0, sizeof(IterStats) + sizeof(unsigned long long),
                            c->stream),
            "memset");
    MX_CUDA(cudaEventRecord(c->evp[0], c->stream), "event");
    MX_LAUNCH(launch_gemm_tc(b.A, b.Nt, b.T, ld, n, kind, kind == 0 ? 1 : 2, nullptr, 0.0,
                             nullptr, &w.scal->iter.gemm_err, c->wait_limit_ns, c->stream),
              "tensor-core gemm");
    MX_LAUNCH(launch_gemm_tc(b.T, b.B, b.X32, ld, n, kind, 0, has_K ? w.Ks : nullptr, p.lambda,
                             &w.scal->xmax_key, &w.scal->iter.gemm_err, c->wait_limit_ns,
                             c->stream),
              "tensor-core gemm");
    MX_CUDA(cudaEventRecord(c->evp[1], c->stream), "event");
    SdsnLaunch L{};
    L.n = n;
    L.X = b.X32;
    L.ldx = ld;
    L.Y = b.X32;
    L.ldy = ld;
    L.in_fp32 = 1;
    L.out_fp32 = 1;
    L.mode = 0;
    L.theta = p.theta;
    L.gamma_tol = tol32;
    L.max_sweeps = cap32;
    L.xmax_key = &w.scal->xmax_key;
    L.stats = &w.scal->iter.sdsn;
    L.partials = w.sdsn_partials;
    L.barrier = &w.scal->bar;
    L.limit_ns = c->wait_limit_ns;
    MX_LAUNCH(launch_sdsn(L, c->num_sms, c->stream), "sdsn kernel");
    MX_CUDA(cudaEventRecord(c->evp[2], c->stream), "event");
    SdsnLaunch Pl = L;  // FP64 polish: continue from the FP32 result
    Pl.X = b.X32;
    Pl.Y = w.X;
    Pl.in_fp32 = 1;
    Pl.out_fp32 = 0;
    Pl.mode = 1;
    Pl.gamma_tol = p.gamma_tol;
    Pl.max_sweeps = p.max_polish;
    Pl.gate = &w.scal->iter.sdsn;
    Pl.gate_tol = tol32;
    Pl.stats = &w.scal->iter.polish;
    MX_LAUNCH(launch_sdsn(Pl, c->num_sms, c->stream), "sdsn polish kernel");
    MX_CUDA(cudaEventRecord(c->evp[3], c->stream), "event");
    MX_LAUNCH(launch_update_mixed(w.N, w.X, ld, n, p.alpha, b.Nt, kind, w.partials,
                                  &w.scal->ticket_update, &w.scal->iter, c->stream),
              "update kernel");
    MX_CUDA(cudaEventRecord(c->evp[4], c->stream), "event");
    MX_CUDA(cudaMemcpyAsync(&w.hscal->iter, &w.scal->iter, sizeof(IterStats),
                            cudaMemcpyDeviceToHost, c->stream),
            "readback");
    MX_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
    const IterStats& it = w.hscal->iter;
    if (it.gemm_err) {
      set_err(c, "tensor-core GEMM: a device-side wait exceeded its limit");
      return FRAM_ERR_TIMEOUT;
    }
    fram_status s1 = dev_status(c, it.sdsn.status, "SDSN");
    if (s1 != FRAM_OK) return s1;
    s1 = dev_status(c, it.polish.status, "SDSN polish");
    if (s1 != FRAM_OK) return s1;
    inf->outer_iters = t + 1;
    inf->ms_gemm += phase_ms(c, 0, 1);
    inf->ms_sdsn += phase_ms(c, 1, 2);
    inf->ms_polish += phase_ms(c, 2, 3);
    inf->ms_update += phase_ms(c, 3, 4);
    inf->total_sweeps += it.sdsn.sweeps + it.polish.sweeps;
    inf->polish_sweeps += it.polish.sweeps;
    inf->gamma = it.polish.gamma;
    inf->sdsn_converged_last = it.polish.gamma <= p.gamma_tol ? 1 : 0;
    inf->delta = it.delta;
    // Reading (ix): the BF16/TF32 gradient puts a floor under delta (delta
    // settles on a short cycle), so the mixed paths stop at mixed_delta_tol,
    // or earlier if delta stops contracting.
    if (it.delta <= p.delta_tol || it.delta <= p.mixed_delta_tol) break;
    if (p.stall_ratio > 0.0 && it.delta <= p.stall_below && it.delta > p.stall_ratio * prev_delta)
      break;
    prev_delta = it.delta;
  }
  return FRAM_OK;
}

}  // namespace fram
