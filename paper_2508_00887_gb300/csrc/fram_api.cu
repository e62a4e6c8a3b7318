// C ABI of the FRAM solver (include/fram.h): context, device workspace and
// the host side of Alg. 1 (arXiv 2508.00887).  Every arithmetic step runs in
// this library's kernels; the host only sequences launches and reads back a
// few scalars per outer iteration (delta and the SDSN status).
#include <cuda.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fram.h"
#include "fram_internal.cuh"
#include "fram_ctx.h"

using namespace fram;

// ------------------------------------------------------------ helpers
namespace fram {

void set_err(fram_ctx* c, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->last_error = buf;
}

fram_status cuda_fail(fram_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) {
    // A launcher refused without a CUDA error: the launch would exceed a
    // limit of this GPU (co-resident CTAs of a cooperative grid, shared
    // memory per CTA, cluster residency) or an attribute query failed.
    set_err(c, "%s: the launch exceeds this GPU's limits (co-resident CTAs, shared memory or "
               "cluster size) for this problem size", what);
    return FRAM_ERR_INVALID;
  }
  set_err(c, "%s: %s", what, cudaGetErrorString(e));
  cudaGetLastError();
  return FRAM_ERR_CUDA;
}

bool is_device_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

namespace {
using RangeFn = CUresult (*)(CUdeviceptr*, size_t*, CUdeviceptr);
RangeFn range_fn() {
  static const RangeFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<RangeFn>(p);
    cudaGetLastError();
    return static_cast<RangeFn>(nullptr);
  }();
  return fn;
}
}  // namespace

bool PtrClassifier::is_device(const void* p) {
  if (p == nullptr) return false;
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  auto it = std::upper_bound(ranges_.begin(), ranges_.end(), std::make_pair(a, UINTPTR_MAX));
  if (it != ranges_.begin() && a < std::prev(it)->second) return true;
  if (!is_device_ptr(p)) return false;
  CUdeviceptr base = 0;
  size_t size = 0;
  const RangeFn fn = range_fn();
  if (fn && fn(&base, &size, (CUdeviceptr)a) == CUDA_SUCCESS && size > 0) {
    const std::pair<uintptr_t, uintptr_t> r((uintptr_t)base, (uintptr_t)base + size);
    ranges_.insert(std::upper_bound(ranges_.begin(), ranges_.end(), r), r);
  }
  return true;
}

int round_ld(int n) { return ((n + 127) / 128) * 128; }

static void dfree(void*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void Workspace::release() {
  void** ptrs[] = {(void**)&As, (void**)&Bs, (void**)&Ks, (void**)&N, (void**)&T, (void**)&X,
                   (void**)&A0, (void**)&B0, (void**)&K0, (void**)&perm, &lap_ws,
                   (void**)&partials, (void**)&sdsn_partials, (void**)&scal, &mixed,
                   (void**)&sp_cnt, (void**)&sp_rowptr[0], (void**)&sp_rowptr[1],
                   (void**)&sp_col[0], (void**)&sp_col[1], (void**)&sp_val[0],
                   (void**)&sp_val[1]};
  for (void** p : ptrs) dfree(*p);
  sp_cap_n = 0;
  sp_cap_nnz[0] = sp_cap_nnz[1] = 0;
  sp_on[0] = sp_on[1] = false;
  if (hscal) cudaFreeHost(hscal);
  hscal = nullptr;
  cap_n = 0;
  cap_ld = 0;
  mixed_cap_n = 0;
  bytes = 0;
}

size_t Workspace::bytes_for(int n, int num_sms) {
  const size_t ld = round_ld(n);
  size_t b = 6 * ld * ld * sizeof(double);           // As Bs Ks N T X
  b += 3 * (size_t)n * n * sizeof(double);           // staging of host inputs
  b += (size_t)n * sizeof(int32_t) + lap_workspace_bytes(n);
  b += 8192 * sizeof(double);
  b += sdsn_partials_elems(n, num_sms) * sizeof(double);
  return b + 8 * 4096;
}

fram_status ensure_workspace(fram_ctx* c, int n) {
  Workspace& w = c->ws;
  if (n <= w.cap_n && w.scal != nullptr) return FRAM_OK;
  const size_t need = Workspace::bytes_for(n, c->num_sms);
  size_t others = c->serve_bytes;
  if (c->budget && need + others > c->budget) {
    set_err(c, "workspace for n=%d needs %zu bytes; HBM budget is %zu", n, need + others,
            c->budget);
    return FRAM_ERR_OOM;
  }
  w.release();
  const size_t ld = round_ld(n);
  const size_t mat = ld * ld * sizeof(double);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes ? bytes : 256);
  };
  A((void**)&w.As, mat);
  A((void**)&w.Bs, mat);
  A((void**)&w.Ks, mat);
  A((void**)&w.N, mat);
  A((void**)&w.T, mat);
  A((void**)&w.X, mat);
  A((void**)&w.A0, (size_t)n * n * sizeof(double));
  A((void**)&w.B0, (size_t)n * n * sizeof(double));
  A((void**)&w.K0, (size_t)n * n * sizeof(double));
  A((void**)&w.perm, (size_t)n * sizeof(int32_t));
  A(&w.lap_ws, lap_workspace_bytes(n));
  A((void**)&w.partials, 8192 * sizeof(double));
  A((void**)&w.sdsn_partials, sdsn_partials_elems(n, c->num_sms) * sizeof(double));
  A((void**)&w.scal, sizeof(DevScalars));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&w.hscal, sizeof(DevScalars));
  if (e == cudaSuccess) e = cudaMemsetAsync(w.scal, 0, sizeof(DevScalars), c->stream);
  if (e != cudaSuccess) {
    w.release();
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) {
      set_err(c, "cudaMalloc failed for n=%d workspace", n);
      return FRAM_ERR_OOM;
    }
    return cuda_fail(c, e, "workspace allocation");
  }
  w.cap_n = n;
  w.cap_ld = (int)ld;
  w.bytes = need;
  return FRAM_OK;
}

// Low-precision buffers of the mixed paths, allocated on first use.
fram_status ensure_mixed(fram_ctx* c, int n) {
  Workspace& w = c->ws;
  if (w.mixed != nullptr && n <= w.mixed_cap_n) return FRAM_OK;
  if (w.mixed) cudaFree(w.mixed);
  w.mixed = nullptr;
  w.mixed_cap_n = 0;
  const size_t need = mixed_bytes_for(n);
  if (c->budget && w.bytes + need + c->serve_bytes > c->budget) {
    set_err(c, "mixed-precision buffers for n=%d exceed the HBM budget", n);
    return FRAM_ERR_OOM;
  }
  cudaError_t e = cudaMalloc(&w.mixed, need);
  if (e != cudaSuccess) {
    w.mixed = nullptr;
    cudaGetLastError();
    set_err(c, "cudaMalloc failed for mixed buffers (n=%d)", n);
    return FRAM_ERR_OOM;
  }
  w.mixed_cap_n = n;
  return FRAM_OK;
}

// Stop tolerance of the exact projection: the requested gamma_tol, but not
// below what FP64 row sums of n terms can resolve.
double exact_tol(double gamma_tol, int n) {
  const double floor_tol = 8.0 * n * 2.220446049250313e-16;
  return gamma_tol > floor_tol ? gamma_tol : floor_tol;
}

fram_status check_params(fram_ctx* c, const fram_params& p) {
  if (!(p.alpha > 0.0 && p.alpha <= 1.0) || !(p.theta > 0.0) || !isfinite(p.theta) ||
      !isfinite(p.lambda) || !(p.delta_tol >= 0.0) || !(p.gamma_tol == p.gamma_tol) ||
      !(p.stall_ratio >= 0.0 && p.stall_ratio <= 1.0) || !(p.stall_below >= 0.0) ||
      !(p.mixed_delta_tol >= 0.0) ||
      p.max_outer < 1 || p.max_sweeps < 1 || p.max_polish < 0 || p.init < 0 || p.init > 2 ||
      p.precision < FRAM_PREC_FP64 || p.precision > FRAM_PREC_MIXED_BF16 ||
      p.projection < FRAM_PROJ_SDSN || p.projection > FRAM_PROJ_EXACT) {
    set_err(c, "invalid fram_params");
    return FRAM_ERR_INVALID;
  }
  if (p.projection == FRAM_PROJ_EXACT && p.precision != FRAM_PREC_FP64) {
    set_err(c, "the exact projection runs on the FP64 path only");
    return FRAM_ERR_INVALID;
  }
  return FRAM_OK;
}

double phase_ms(fram_ctx* c, int a, int b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, c->evp[a], c->evp[b]) != cudaSuccess) {
    cudaGetLastError();
    return 0.0;
  }
  return ms;
}

// Map a device status word onto the ABI.
fram_status dev_status(fram_ctx* c, int st, const char* where) {
  if (st == DEV_OK) return FRAM_OK;
  if (st == DEV_DEGENERATE) {
    set_err(c, "%s: max(X) <= 0, SDSN step 1 is undefined", where);
    return FRAM_ERR_DEGENERATE;
  }
  set_err(c, "%s: a device-side wait exceeded its limit", where);
  return FRAM_ERR_TIMEOUT;
}

// Stage an n x n (or n) input: device pointers are used in place, host
// buffers are copied into `staging`.
fram_status stage_in(fram_ctx* c, const double* src, size_t count, double* staging,
                     const double** out) {
  if (src == nullptr) {
    *out = nullptr;
    return FRAM_OK;
  }
  if (is_device_ptr(src)) {
    *out = src;
    return FRAM_OK;
  }
  cudaError_t e = cudaMemcpyAsync(staging, src, count * sizeof(double), cudaMemcpyHostToDevice,
                                  c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device copy");
  *out = staging;
  return FRAM_OK;
}

#define FR_TRY(x)                          \
  do {                                     \
    fram_status _s = (x);                  \
    if (_s != FRAM_OK) return _s;          \
  } while (0)
#define FR_CUDA(x, what)                              \
  do {                                                \
    cudaError_t _e = (x);                             \
    if (_e != cudaSuccess) return cuda_fail(c, _e, what); \
  } while (0)
#define FR_LAUNCH(x, what)                                              \
  do {                                                                  \
    int _k = (x);                                                       \
    if (_k < 0) return cuda_fail(c, cudaGetLastError(), what);          \
    c->launches += (uint64_t)_k;                                        \
  } while (0)

// Validate inputs and prescale them (Alg. 1 steps 2-3).
fram_status validate_and_scale(fram_ctx* c, int n, const double* A0, const double* B0,
                               const double* K0, double* scale_c) {
  Workspace& w = c->ws;
  const int ld = round_ld(n);
  FR_CUDA(cudaMemsetAsync(&w.scal->val, 0, sizeof(ValidateStats), c->stream), "memset");
  FR_LAUNCH(launch_validate(A0, B0, K0, n, &w.scal->val, c->stream), "validate kernel");
  FR_CUDA(cudaMemcpyAsync(&w.hscal->val, &w.scal->val, sizeof(ValidateStats),
                          cudaMemcpyDeviceToHost, c->stream),
          "readback");
  FR_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
  const ValidateStats& v = w.hscal->val;
  const char* names[3] = {"A", "B", "K"};
  for (int m = 0; m < 3; ++m)
    if (v.bad_value[m]) {
      set_err(c, "%s has negative or non-finite entries", names[m]);
      return FRAM_ERR_INVALID;
    }
  double mx[3], as[2];
  for (int m = 0; m < 3; ++m) memcpy(&mx[m], &v.maxbits[m], 8);
  for (int m = 0; m < 2; ++m) memcpy(&as[m], &v.asymbits[m], 8);
  for (int m = 0; m < 2; ++m)
    if (as[m] > 1e-12 * std::max(mx[m], 1.0)) {
      set_err(c, "%s is not symmetric (max |M - M^T| = %g)", names[m], as[m]);
      return FRAM_ERR_INVALID;
    }
  double cc = std::max(mx[0], mx[1]);
  if (K0) cc = std::max(cc, mx[2]);
  if (!(cc > 0.0)) {
    set_err(c, "all inputs are zero: SDSN step 1 is undefined");
    return FRAM_ERR_DEGENERATE;
  }
  // A / sqrt(c) and B / sqrt(c) as one multiply by the reciprocal (an FP64
  // division per element is a long sequence on GB300's FP64 pipe); the
  // batched and served paths scale the same way.
  const double inv_s = 1.0 / sqrt(cc);
  FR_LAUNCH(launch_scale(A0, n, inv_s, w.As, ld, c->stream), "scale kernel");
  FR_LAUNCH(launch_scale(B0, n, inv_s, w.Bs, ld, c->stream), "scale kernel");
  if (K0) FR_LAUNCH(launch_scale(K0, n, 1.0 / cc, w.Ks, ld, c->stream), "scale kernel");
  *scale_c = cc;
  return FRAM_OK;
}

// FP64 gradient operands in CSR when sparse enough (fraction of nonzeros at
// most c->sparse_density): CSR of A_s and of B_s^T.  Uses T as scratch for
// B_s^T, so it runs before the outer loop.
fram_status prepare_sparse(fram_ctx* c, int n) {
  Workspace& w = c->ws;
  w.sp_on[0] = w.sp_on[1] = false;
  if (!(c->sparse_density > 0.0) || n < 64) return FRAM_OK;
  const int ld = round_ld(n);
  auto grow = [&](void** p, size_t& cap, size_t need, size_t elem) -> bool {
    if (*p && cap >= need) return true;
    dfree(*p);
    cap = 0;
    if (cudaMalloc(p, (need ? need : 1) * elem) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cap = need;
    return true;
  };
  size_t capn = (size_t)w.sp_cap_n;
  if (!grow((void**)&w.sp_cnt, capn, (size_t)n, sizeof(int))) {
    set_err(c, "out of device memory for the sparse gradient");
    return FRAM_ERR_OOM;
  }
  size_t capr0 = (size_t)w.sp_cap_n, capr1 = (size_t)w.sp_cap_n;
  if (!grow((void**)&w.sp_rowptr[0], capr0, (size_t)n + 1, sizeof(int)) ||
      !grow((void**)&w.sp_rowptr[1], capr1, (size_t)n + 1, sizeof(int))) {
    set_err(c, "out of device memory for the sparse gradient");
    return FRAM_ERR_OOM;
  }
  w.sp_cap_n = n;
  const double* src[2] = {w.As, w.T};
  FR_LAUNCH(launch_transpose(w.Bs, w.T, ld, n, nullptr, 0.0, nullptr, c->stream), "transpose");
  int nnz[2];
  for (int m = 0; m < 2; ++m) {
    FR_LAUNCH(launch_csr_count(src[m], ld, n, w.sp_cnt, c->stream), "csr count");
    FR_LAUNCH(launch_csr_scan(w.sp_cnt, n, w.sp_rowptr[m], c->stream), "csr scan");
    FR_CUDA(cudaMemcpyAsync(&nnz[m], w.sp_rowptr[m] + n, sizeof(int), cudaMemcpyDeviceToHost,
                            c->stream),
            "readback");
  }
  FR_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
  for (int m = 0; m < 2; ++m) {
    if ((double)nnz[m] > c->sparse_density * (double)n * (double)n) continue;
    if (!w.sp_col[m] || !w.sp_val[m] || w.sp_cap_nnz[m] < (size_t)nnz[m]) {
      // column indices and values grow together, to the same capacity
      dfree(*(void**)&w.sp_col[m]);
      dfree(*(void**)&w.sp_val[m]);
      w.sp_cap_nnz[m] = 0;
      const size_t cap = nnz[m] > 0 ? (size_t)nnz[m] : 1;
      if (cudaMalloc((void**)&w.sp_col[m], cap * sizeof(int)) != cudaSuccess ||
          cudaMalloc((void**)&w.sp_val[m], cap * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        set_err(c, "out of device memory for the sparse gradient");
        return FRAM_ERR_OOM;
      }
      w.sp_cap_nnz[m] = cap;
    }
    FR_LAUNCH(launch_csr_fill(src[m], ld, n, w.sp_rowptr[m], w.sp_col[m], w.sp_val[m], c->stream),
              "csr fill");
    w.sp_on[m] = true;
  }
  return FRAM_OK;
}

// X = A_s N B_s (+ lam K_s) into w.X with max(X) into cmax (may be NULL):
// dense DGEMMs, or the CSR products when prepare_sparse switched them on
// (bit-identical results).
fram_status fp64_gradient(fram_ctx* c, int n, bool withK, double lam, unsigned long long* cmax) {
  Workspace& w = c->ws;
  const int ld = round_ld(n);
  if (w.sp_on[0])
    FR_LAUNCH(launch_spmm(w.sp_rowptr[0], w.sp_col[0], w.sp_val[0], n, w.N, ld, w.T, c->stream),
              "spmm");
  else
    FR_LAUNCH(launch_dgemm(w.As, w.N, w.T, ld, n, nullptr, 0.0, nullptr, c->stream), "gemm");
  if (w.sp_on[1]) {
    // X^T = B_s^T T^T, then X = (X^T)^T (+ lam K) with the max.
    FR_LAUNCH(launch_transpose(w.T, w.X, ld, n, nullptr, 0.0, nullptr, c->stream), "transpose");
    FR_LAUNCH(launch_spmm(w.sp_rowptr[1], w.sp_col[1], w.sp_val[1], n, w.X, ld, w.T, c->stream),
              "spmm");
    FR_LAUNCH(launch_transpose(w.T, w.X, ld, n, withK ? w.Ks : nullptr, lam, cmax, c->stream),
              "transpose");
  } else {
    FR_LAUNCH(launch_dgemm(w.T, w.Bs, w.X, ld, n, withK ? w.Ks : nullptr, lam, cmax, c->stream),
              "gemm");
  }
  return FRAM_OK;
}

// The full single-pair solve on device-resident (or staged) inputs.
fram_status solve_one(fram_ctx* c, int n, const double* A, const double* B, const double* K,
                      const fram_params& p, double* X_out, int32_t* perm_out, fram_info* info) {
  FR_TRY(ensure_workspace(c, n));
  Workspace& w = c->ws;
  const int ld = round_ld(n);
  FR_CUDA(cudaEventRecord(c->ev0, c->stream), "event");
  const double *A0, *B0, *K0;
  FR_TRY(stage_in(c, A, (size_t)n * n, w.A0, &A0));
  FR_TRY(stage_in(c, B, (size_t)n * n, w.B0, &B0));
  FR_TRY(stage_in(c, K, (size_t)n * n, w.K0, &K0));
  double cc = 0.0;
  FR_TRY(validate_and_scale(c, n, A0, B0, K0, &cc));

  const bool zero_init = p.init == 1 || (p.init == 0 && K0 != nullptr);
  FR_LAUNCH(launch_fill_assignment(w.N, n, ld, zero_init ? 0.0 : 1.0 / n, c->stream), "fill");

  fram_info inf;
  memset(&inf, 0, sizeof inf);
  double delta = INFINITY;
  fram_status rs = FRAM_OK;
  if (p.precision == FRAM_PREC_FP64) {
    FR_TRY(prepare_sparse(c, n));
    for (int t = 0; t < p.max_outer; ++t) {
      // The iteration stats and the max key, adjacent: one memset (the update
      // kernel rewrites delta and its sums every iteration).
      FR_CUDA(cudaMemsetAsync(&w.scal->iter, 0, sizeof(IterStats) + sizeof(unsigned long long),
                              c->stream),
              "memset");
      FR_CUDA(cudaEventRecord(c->evp[0], c->stream), "event");
      FR_TRY(fp64_gradient(c, n, K0 != nullptr, p.lambda, &w.scal->xmax_key));
      FR_CUDA(cudaEventRecord(c->evp[1], c->stream), "event");
      if (p.projection == FRAM_PROJ_EXACT) {
        // Step 6 variant: the exact FRA solution (T is free after the GEMMs).
        FR_LAUNCH(launch_fra(w.X, ld, w.T, ld, n, &w.scal->xmax_key, p.theta,
                             exact_tol(p.gamma_tol, n), p.max_sweeps, w.sdsn_partials,
                             &w.scal->bar, &w.scal->iter.sdsn, c->wait_limit_ns, c->num_sms,
                             c->stream),
                  "exact projection kernel");
      } else {
        SdsnLaunch L{};
        L.n = n;
        L.X = w.X;
        L.ldx = ld;
        L.Y = w.X;
        L.ldy = ld;
        L.theta = p.theta;
        L.gamma_tol = p.gamma_tol;
        L.max_sweeps = p.max_sweeps;
        L.xmax_key = &w.scal->xmax_key;
        L.stats = &w.scal->iter.sdsn;
        L.partials = w.sdsn_partials;
        L.barrier = &w.scal->bar;
        L.limit_ns = c->wait_limit_ns;
        FR_LAUNCH(launch_sdsn_fp64(L, c->num_sms, c->stream), "sdsn kernel");
      }
      FR_CUDA(cudaEventRecord(c->evp[2], c->stream), "event");
      FR_LAUNCH(launch_update(w.N, ld, w.X, ld, n, p.alpha, &w.scal->iter, w.partials,
                              &w.scal->ticket_update, c->stream),
                "update kernel");
      FR_CUDA(cudaEventRecord(c->evp[3], c->stream), "event");
      FR_CUDA(cudaMemcpyAsync(&w.hscal->iter, &w.scal->iter, sizeof(IterStats),
                              cudaMemcpyDeviceToHost, c->stream),
              "readback");
      FR_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
      const IterStats& it = w.hscal->iter;
      FR_TRY(dev_status(c, it.sdsn.status, "SDSN"));
      inf.outer_iters = t + 1;
      inf.ms_gemm += phase_ms(c, 0, 1);
      inf.ms_sdsn += phase_ms(c, 1, 2);
      inf.ms_update += phase_ms(c, 2, 3);
      inf.total_sweeps += it.sdsn.sweeps;
      inf.sdsn_converged_last = it.sdsn.converged;
      inf.gamma = it.sdsn.gamma;
      delta = it.delta;
      inf.delta = delta;
      if (delta <= p.delta_tol) break;
    }
  } else {
    FR_TRY(ensure_mixed(c, n));
    rs = solve_mixed_loop(c, n, K0 != nullptr, p, &inf);
    if (rs != FRAM_OK) return rs;
  }

  // Alg. 1 step 10 and eq. 1 on the unscaled inputs.
  FR_CUDA(cudaEventRecord(c->evp[0], c->stream), "event");
  FR_LAUNCH(launch_lap(w.N, ld, n, w.perm, &w.scal->lap, w.lap_ws, c->num_sms, c->wait_limit_ns,
                       c->stream, c->lap_searches), "lap kernels");
  FR_CUDA(cudaEventRecord(c->evp[1], c->stream), "event");
  FR_LAUNCH(launch_objective(A0, B0, K0, p.lambda, n, w.perm, &w.scal->obj, w.partials,
                             &w.scal->ticket_obj, c->stream),
            "objective kernel");
  if (X_out)
    FR_CUDA(cudaMemcpy2DAsync(X_out, (size_t)n * sizeof(double), w.N, (size_t)ld * sizeof(double),
                              (size_t)n * sizeof(double), n, cudaMemcpyDefault, c->stream),
            "copy X_out");
  FR_CUDA(cudaMemcpyAsync(perm_out, w.perm, (size_t)n * sizeof(int32_t), cudaMemcpyDefault,
                          c->stream),
          "copy perm_out");
  FR_CUDA(cudaMemcpyAsync(&w.hscal->lap, &w.scal->lap, sizeof(LapStats) + sizeof(ObjStats),
                          cudaMemcpyDeviceToHost, c->stream),
          "readback");
  FR_CUDA(cudaEventRecord(c->ev1, c->stream), "event");
  FR_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
  c->lap_ran = true;
  if (w.hscal->lap.status != 0) {
    set_err(c, "assignment search did not terminate");
    return FRAM_ERR_TIMEOUT;
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  inf.ms_rounding = phase_ms(c, 0, 1);
  inf.lap_augmentations = w.hscal->lap.augmented;
  inf.lap_auction_phases = w.hscal->lap.auction_phases;
  inf.assignment_value = w.hscal->lap.value;
  inf.objective = w.hscal->obj.objective;
  inf.match_error = w.hscal->obj.match_error;
  inf.ms_total = ms;
  if (info) *info = inf;
  return FRAM_OK;
}

}  // namespace fram

// ------------------------------------------------------------ C ABI
extern "C" {

void fram_default_params(fram_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->lambda = 1.0;
  p->alpha = 0.95;
  p->theta = 10.0;
  p->delta_tol = 1e-6;
  p->gamma_tol = 1e-14;
  p->polish_tol = 1e-6;
  p->mixed_delta_tol = 5e-4;
  p->stall_ratio = 0.9;
  p->stall_below = 1e-3;
  p->max_outer = 100;
  p->max_sweeps = 200;
  p->max_polish = 0;
  p->precision = FRAM_PREC_FP64;
  p->init = 0;
  p->projection = FRAM_PROJ_SDSN;
}

fram_status fram_create(fram_ctx** out, int device, size_t budget, void* stream) {
  if (!out) return FRAM_ERR_INVALID;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess) {
    cudaGetLastError();
    return FRAM_ERR_CUDA;
  }
  if (device < 0 || device >= count) return FRAM_ERR_INVALID;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return FRAM_ERR_CUDA;
  }
  fram_ctx* c = new fram_ctx();
  c->device = device;
  c->budget = budget;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&c->cc_major, cudaDevAttrComputeCapabilityMajor, device);
  cudaDeviceGetAttribute(&c->cc_minor, cudaDevAttrComputeCapabilityMinor, device);
  if (stream) {
    c->stream = static_cast<cudaStream_t>(stream);
    c->own_stream = false;
  } else if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return FRAM_ERR_CUDA;
  } else {
    c->own_stream = true;
  }
  bool ev_ok = cudaEventCreate(&c->ev0) == cudaSuccess && cudaEventCreate(&c->ev1) == cudaSuccess;
  for (int i = 0; i < 5 && ev_ok; ++i) ev_ok = cudaEventCreate(&c->evp[i]) == cudaSuccess;
  if (!ev_ok) {
    cudaGetLastError();
    fram_destroy(c);  // releases the events and stream made so far
    return FRAM_ERR_CUDA;
  }
  *out = c;
  return FRAM_OK;
}

fram_status fram_destroy(fram_ctx* c) {
  if (!c) return FRAM_OK;
  cudaSetDevice(c->device);
  serve_shutdown(c);
  cudaStreamSynchronize(c->stream);
  c->ws.release();
  batched_release(c);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  for (int i = 0; i < 5; ++i)
    if (c->evp[i]) cudaEventDestroy(c->evp[i]);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  cudaGetLastError();
  delete c;
  return FRAM_OK;
}

const char* fram_last_error(const fram_ctx* c) { return c ? c->last_error.c_str() : ""; }

uint64_t fram_kernel_launches(const fram_ctx* c) { return c ? c->launches.load() : 0; }

fram_status fram_set_wait_limit(fram_ctx* c, int limit_ms) {
  if (!c || limit_ms < 1) return FRAM_ERR_INVALID;
  c->wait_limit_ns = (uint64_t)limit_ms * 1000000ull;
  return FRAM_OK;
}

fram_status fram_selftest_wait_timeout(fram_ctx* c, int blocks) {
  if (!c) return FRAM_ERR_INVALID;
  c->last_error.clear();
  if (blocks < 1 || blocks > 64) {
    set_err(c, "fram_selftest_wait_timeout: 1 <= blocks <= 64");
    return FRAM_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  FR_TRY(ensure_workspace(c, 1));
  Workspace& w = c->ws;
  // Small grids are co-resident on any GPU, so every CTA reaches the barrier.
  FR_CUDA(cudaMemsetAsync(&w.scal->bar, 0, sizeof(GridBarrier), c->stream), "memset");
  FR_CUDA(cudaMemsetAsync(&w.scal->iter.sdsn.status, 0, sizeof(int), c->stream), "memset");
  FR_LAUNCH(launch_wait_selftest(&w.scal->bar, &w.scal->iter.sdsn.status, blocks,
                                 c->wait_limit_ns, c->stream),
            "wait self-test kernel");
  FR_CUDA(cudaMemcpyAsync(&w.hscal->iter.sdsn.status, &w.scal->iter.sdsn.status, sizeof(int),
                          cudaMemcpyDeviceToHost, c->stream),
          "readback");
  FR_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
  return dev_status(c, w.hscal->iter.sdsn.status, "self-test wait");
}

fram_status fram_solve(fram_ctx* c, int n, const double* A, const double* B, const double* K,
                       const fram_params* params, double* X_out, int32_t* perm_out,
                       fram_info* info) {
  if (!c) return FRAM_ERR_INVALID;
  c->last_error.clear();
  if (n < 1 || !A || !B || !perm_out) {
    set_err(c, "fram_solve: n >= 1 and non-NULL A, B, perm_out are required");
    return FRAM_ERR_INVALID;
  }
  fram_params p;
  if (params)
    p = *params;
  else
    fram_default_params(&p);
  FR_TRY(check_params(c, p));
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "set device");
  std::lock_guard<std::mutex> lk(c->mu);
  return solve_one(c, n, A, B, K, p, X_out, perm_out, info);
}

fram_status fram_set_lap_searches(fram_ctx* c, int searches) {
  if (!c) return FRAM_ERR_INVALID;
  c->last_error.clear();
  if (searches < 0 || searches > 16) {
    set_err(c, "fram_set_lap_searches: searches must lie in 0..16");
    return FRAM_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  c->lap_searches = searches;
  return FRAM_OK;
}

fram_status fram_lap_last_stats(const fram_ctx* c, int* augmented, int* repeats,
                                long long* steps) {
  if (!c || !c->lap_ran || !c->ws.hscal) return FRAM_ERR_INVALID;
  if (augmented) *augmented = c->ws.hscal->lap.augmented;
  if (repeats) *repeats = c->ws.hscal->lap.repeats;
  if (steps) *steps = c->ws.hscal->lap.steps;
  return FRAM_OK;
}

fram_status fram_set_sparse_density(fram_ctx* c, double max_density) {
  if (!c) return FRAM_ERR_INVALID;
  if (!(max_density >= 0.0 && max_density <= 1.0)) {
    set_err(c, "fram_set_sparse_density: the fraction must lie in [0, 1]");
    return FRAM_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  c->sparse_density = max_density;
  return FRAM_OK;
}

fram_status fram_node_affinity(fram_ctx* c, int n, int d, const double* F, const double* Ft,
                               double* K) {
  if (!c) return FRAM_ERR_INVALID;
  c->last_error.clear();
  if (n < 1 || d < 1 || !F || !Ft || !K || !is_device_ptr(F) || !is_device_ptr(Ft) ||
      !is_device_ptr(K)) {
    set_err(c, "fram_node_affinity: n, d >= 1 and device pointers F, Ft, K are required");
    return FRAM_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  FR_LAUNCH(launch_node_affinity(F, Ft, n, d, K, c->stream), "node affinity kernel");
  FR_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
  return FRAM_OK;
}

fram_status fram_gradient(fram_ctx* c, int n, const double* A, const double* Nm, const double* B,
                          const double* K, double lambda, double* X) {
  if (!c) return FRAM_ERR_INVALID;
  c->last_error.clear();
  if (n < 1 || !A || !Nm || !B || !X || !is_device_ptr(A) || !is_device_ptr(Nm) ||
      !is_device_ptr(B) || !is_device_ptr(X) || (K && !is_device_ptr(K))) {
    set_err(c, "fram_gradient: n >= 1 and device pointers A, N, B, X (and K) are required");
    return FRAM_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  FR_TRY(ensure_workspace(c, n));
  Workspace& w = c->ws;
  const int ld = round_ld(n);
  FR_LAUNCH(launch_scale(A, n, 1.0, w.As, ld, c->stream), "copy");
  FR_LAUNCH(launch_scale(B, n, 1.0, w.Bs, ld, c->stream), "copy");
  FR_LAUNCH(launch_scale(Nm, n, 1.0, w.N, ld, c->stream), "copy");
  if (K) FR_LAUNCH(launch_scale(K, n, 1.0, w.Ks, ld, c->stream), "copy");
  FR_TRY(prepare_sparse(c, n));
  FR_TRY(fp64_gradient(c, n, K != nullptr, lambda, nullptr));
  FR_CUDA(cudaMemcpy2DAsync(X, (size_t)n * sizeof(double), w.X, (size_t)ld * sizeof(double),
                            (size_t)n * sizeof(double), n, cudaMemcpyDeviceToDevice, c->stream),
          "copy X");
  FR_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
  return FRAM_OK;
}

fram_status fram_gradient_lowp(fram_ctx* c, int n, const double* A, const double* Nm,
                               const double* B, const double* K, double lambda, int precision,
                               float* X) {
  if (!c) return FRAM_ERR_INVALID;
  c->last_error.clear();
  if (n < 1 || !A || !Nm || !B || !X || !is_device_ptr(A) || !is_device_ptr(Nm) ||
      !is_device_ptr(B) || !is_device_ptr(X) || (K && !is_device_ptr(K)) ||
      (precision != FRAM_PREC_MIXED_BF16 && precision != FRAM_PREC_MIXED_TF32)) {
    set_err(c, "fram_gradient_lowp: n >= 1, device A, N, B, X (and K), and a mixed precision "
               "are required");
    return FRAM_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  FR_TRY(ensure_workspace(c, n));
  FR_TRY(ensure_mixed(c, n));
  Workspace& w = c->ws;
  const int ld = round_ld(n);
  FR_LAUNCH(launch_scale(A, n, 1.0, w.As, ld, c->stream), "copy");
  FR_LAUNCH(launch_scale(B, n, 1.0, w.Bs, ld, c->stream), "copy");
  FR_LAUNCH(launch_scale(Nm, n, 1.0, w.N, ld, c->stream), "copy");
  if (K) FR_LAUNCH(launch_scale(K, n, 1.0, w.Ks, ld, c->stream), "copy");
  float* X32 = nullptr;
  FR_TRY(mixed_gradient(c, n, K != nullptr, lambda, precision == FRAM_PREC_MIXED_BF16 ? 0 : 1,
                        &X32));
  FR_CUDA(cudaMemcpy2DAsync(X, (size_t)n * sizeof(float), X32, (size_t)ld * sizeof(float),
                            (size_t)n * sizeof(float), n, cudaMemcpyDeviceToDevice, c->stream),
          "copy X");
  FR_CUDA(cudaMemcpyAsync(&w.hscal->iter.gemm_err, &w.scal->iter.gemm_err, sizeof(int),
                          cudaMemcpyDeviceToHost, c->stream),
          "readback");
  FR_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
  if (w.hscal->iter.gemm_err) {
    set_err(c, "tensor-core GEMM: a device-side wait exceeded its limit");
    return FRAM_ERR_TIMEOUT;
  }
  return FRAM_OK;
}

fram_status fram_sdsn(fram_ctx* c, int n, const double* X, double* D, double theta,
                      double gamma_tol, int max_sweeps, int* sweeps_out, double* gamma_out) {
  if (!c) return FRAM_ERR_INVALID;
  c->last_error.clear();
  if (n < 1 || !X || !D || !is_device_ptr(X) || !is_device_ptr(D) || !(theta > 0.0) ||
      max_sweeps < 1) {
    set_err(c, "fram_sdsn: n >= 1, device X and D, theta > 0, max_sweeps >= 1 are required");
    return FRAM_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  FR_TRY(ensure_workspace(c, n));
  Workspace& w = c->ws;
  FR_CUDA(cudaMemsetAsync(&w.scal->xmax_key, 0, sizeof(unsigned long long), c->stream), "memset");
  FR_CUDA(cudaMemsetAsync(&w.scal->iter.sdsn, 0, sizeof(SdsnStats), c->stream), "memset");
  FR_LAUNCH(launch_max(X, n, n, &w.scal->xmax_key, c->stream), "max kernel");
  SdsnLaunch L{};
  L.n = n;
  L.X = X;
  L.ldx = n;
  L.Y = D;
  L.ldy = n;
  L.theta = theta;
  L.gamma_tol = gamma_tol;
  L.max_sweeps = max_sweeps;
  L.xmax_key = &w.scal->xmax_key;
  L.stats = &w.scal->iter.sdsn;
  L.partials = w.sdsn_partials;
  L.barrier = &w.scal->bar;
  L.limit_ns = c->wait_limit_ns;
  FR_LAUNCH(launch_sdsn_fp64(L, c->num_sms, c->stream), "sdsn kernel");
  FR_CUDA(cudaMemcpyAsync(&w.hscal->iter.sdsn, &w.scal->iter.sdsn, sizeof(SdsnStats),
                          cudaMemcpyDeviceToHost, c->stream),
          "readback");
  FR_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
  const SdsnStats& st = w.hscal->iter.sdsn;
  FR_TRY(dev_status(c, st.status, "SDSN"));
  if (sweeps_out) *sweeps_out = st.sweeps;
  if (gamma_out) *gamma_out = st.gamma;
  return FRAM_OK;
}

fram_status fram_sdsn_f32(fram_ctx* c, int n, const float* X, int ldx, float* D, int ldd,
                          double theta, double gamma_tol, int max_sweeps, int* sweeps_out,
                          double* gamma_out) {
  if (!c) return FRAM_ERR_INVALID;
  c->last_error.clear();
  if (n < 1 || ldx < n || ldd < n || !X || !D || !is_device_ptr(X) || !is_device_ptr(D) ||
      !(theta > 0.0) || max_sweeps < 1) {
    set_err(c, "fram_sdsn_f32: n >= 1, ldx >= n, ldd >= n, device X and D, theta > 0, "
               "max_sweeps >= 1 are required");
    return FRAM_ERR_INVALID;
  }
  if (X == D && ldx != ldd) {
    set_err(c, "fram_sdsn_f32: in place (D == X) needs ldd == ldx");
    return FRAM_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  FR_TRY(ensure_workspace(c, n));
  Workspace& w = c->ws;
  FR_CUDA(cudaMemsetAsync(&w.scal->xmax_key, 0, sizeof(unsigned long long), c->stream), "memset");
  FR_CUDA(cudaMemsetAsync(&w.scal->iter.sdsn, 0, sizeof(SdsnStats), c->stream), "memset");
  FR_LAUNCH(launch_max_f32(X, ldx, n, &w.scal->xmax_key, c->stream), "max kernel");
  SdsnLaunch L{};
  L.n = n;
  L.X = X;
  L.ldx = ldx;
  L.Y = D;
  L.ldy = ldd;
  L.in_fp32 = 1;
  L.out_fp32 = 1;
  L.theta = theta;
  L.gamma_tol = gamma_tol;
  L.max_sweeps = max_sweeps;
  L.xmax_key = &w.scal->xmax_key;
  L.stats = &w.scal->iter.sdsn;
  L.partials = w.sdsn_partials;
  L.barrier = &w.scal->bar;
  L.limit_ns = c->wait_limit_ns;
  FR_LAUNCH(launch_sdsn(L, c->num_sms, c->stream), "sdsn kernel");
  FR_CUDA(cudaMemcpyAsync(&w.hscal->iter.sdsn, &w.scal->iter.sdsn, sizeof(SdsnStats),
                          cudaMemcpyDeviceToHost, c->stream),
          "readback");
  FR_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
  const SdsnStats& st = w.hscal->iter.sdsn;
  FR_TRY(dev_status(c, st.status, "SDSN"));
  if (sweeps_out) *sweeps_out = st.sweeps;
  if (gamma_out) *gamma_out = st.gamma;
  return FRAM_OK;
}

fram_status fram_fra_exact(fram_ctx* c, int n, const double* X, double* D, double theta,
                           double tol, int max_sweeps, int* sweeps_out, double* res_out) {
  if (!c) return FRAM_ERR_INVALID;
  c->last_error.clear();
  if (n < 1 || !X || !D || !is_device_ptr(X) || !is_device_ptr(D) || !(theta > 0.0) ||
      !isfinite(theta) || max_sweeps < 1 || !(tol >= 0.0)) {
    set_err(c, "fram_fra_exact: n >= 1, device X and D, theta > 0, tol >= 0, max_sweeps >= 1");
    return FRAM_ERR_INVALID;
  }
  if (2 * (size_t)n * sizeof(double) > 200 * 1024) {
    set_err(c, "fram_fra_exact: n = %d exceeds the limit of 12800", n);
    return FRAM_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  FR_TRY(ensure_workspace(c, n));
  Workspace& w = c->ws;
  const int ld = round_ld(n);
  FR_LAUNCH(launch_scale(X, n, 1.0, w.X, ld, c->stream), "copy");
  FR_CUDA(cudaMemsetAsync(&w.scal->xmax_key, 0, sizeof(unsigned long long), c->stream), "memset");
  FR_CUDA(cudaMemsetAsync(&w.scal->iter.sdsn, 0, sizeof(SdsnStats), c->stream), "memset");
  FR_LAUNCH(launch_max(w.X, ld, n, &w.scal->xmax_key, c->stream), "max kernel");
  FR_LAUNCH(launch_fra(w.X, ld, w.T, ld, n, &w.scal->xmax_key, theta, tol, max_sweeps,
                       w.sdsn_partials, &w.scal->bar, &w.scal->iter.sdsn, c->wait_limit_ns,
                       c->num_sms, c->stream),
            "exact projection kernel");
  FR_CUDA(cudaMemcpy2DAsync(D, (size_t)n * sizeof(double), w.X, (size_t)ld * sizeof(double),
                            (size_t)n * sizeof(double), n, cudaMemcpyDeviceToDevice, c->stream),
          "copy D");
  FR_CUDA(cudaMemcpyAsync(&w.hscal->iter.sdsn, &w.scal->iter.sdsn, sizeof(SdsnStats),
                          cudaMemcpyDeviceToHost, c->stream),
          "readback");
  FR_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
  const SdsnStats& st = w.hscal->iter.sdsn;
  FR_TRY(dev_status(c, st.status, "exact projection"));
  if (sweeps_out) *sweeps_out = st.sweeps;
  if (res_out) *res_out = st.gamma;
  return FRAM_OK;
}

fram_status fram_sdsn_grouped(fram_ctx* c, int count, const int* n, const double* const* X,
                              double* const* D, double theta, double gamma_tol, int max_sweeps,
                              int* sweeps_out, double* gamma_out) {
  if (!c) return FRAM_ERR_INVALID;
  c->last_error.clear();
  if (count < 1 || count > 64 || !n || !X || !D || !(theta > 0.0) || max_sweeps < 1) {
    set_err(c, "fram_sdsn_grouped: 1 <= count <= 64, theta > 0, max_sweeps >= 1 are required");
    return FRAM_ERR_INVALID;
  }
  int nmax = 0, blocks = 0;
  for (int i = 0; i < count; ++i) {
    if (n[i] < 1 || !X[i] || !D[i] || !is_device_ptr(X[i]) || !is_device_ptr(D[i])) {
      set_err(c, "fram_sdsn_grouped: problem %d needs n >= 1 and device X, D", i);
      return FRAM_ERR_INVALID;
    }
    nmax = std::max(nmax, n[i]);
    blocks += sdsn_grid_blocks(n[i], c->num_sms);
  }
  if (blocks > c->num_sms) {
    set_err(c, "fram_sdsn_grouped: the sub-grids need %d CTAs, more than one wave", blocks);
    return FRAM_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  // Per-problem scratch: partials, stats, barriers, max keys.
  size_t per = sdsn_partials_elems(nmax, c->num_sms) * sizeof(double);
  per = (per + 255) & ~(size_t)255;
  const size_t hdr = 256;
  char* buf = nullptr;
  FR_CUDA(cudaMalloc(&buf, count * (per + hdr) + sdsn_group_desc_bytes(count)), "scratch");
  struct Hdr {
    SdsnStats st;
    GridBarrier bar;
    unsigned long long key;
  };
  std::vector<SdsnLaunch> L(count);
  fram_status rs = FRAM_OK;
  FR_CUDA(cudaMemsetAsync(buf, 0, count * hdr, c->stream), "memset");
  for (int i = 0; i < count && rs == FRAM_OK; ++i) {
    Hdr* h = reinterpret_cast<Hdr*>(buf + i * hdr);
    if (launch_max(X[i], n[i], n[i], &h->key, c->stream) < 0) rs = FRAM_ERR_CUDA;
    c->launches += 1;
    L[i].n = n[i];
    L[i].X = X[i];
    L[i].ldx = n[i];
    L[i].Y = D[i];
    L[i].ldy = n[i];
    L[i].theta = theta;
    L[i].gamma_tol = gamma_tol;
    L[i].max_sweeps = max_sweeps;
    L[i].xmax_key = &h->key;
    L[i].stats = &h->st;
    L[i].partials = reinterpret_cast<double*>(buf + count * hdr + i * per);
    L[i].barrier = &h->bar;
    L[i].limit_ns = c->wait_limit_ns;
  }
  if (rs == FRAM_OK &&
      launch_sdsn_group(L.data(), count, c->num_sms, buf + count * (hdr + per),
                        sdsn_group_desc_bytes(count), c->num_sms, c->stream) < 0)
    rs = FRAM_ERR_CUDA;
  std::vector<Hdr> hh(count);
  if (rs == FRAM_OK) {
    c->launches += 1;
    if (cudaMemcpy2DAsync(hh.data(), sizeof(Hdr), buf, hdr, sizeof(Hdr), count,
                          cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      rs = FRAM_ERR_CUDA;
  }
  if (rs == FRAM_ERR_CUDA) set_err(c, "fram_sdsn_grouped: %s", cudaGetErrorString(cudaGetLastError()));
  cudaStreamSynchronize(c->stream);
  cudaFree(buf);
  if (rs != FRAM_OK) return rs;
  for (int i = 0; i < count; ++i) {
    fram_status s1 = dev_status(c, hh[i].st.status, "grouped SDSN");
    if (s1 != FRAM_OK) return s1;
    if (sweeps_out) sweeps_out[i] = hh[i].st.sweeps;
    if (gamma_out) gamma_out[i] = hh[i].st.gamma;
  }
  return FRAM_OK;
}

fram_status fram_assign(fram_ctx* c, int n, const double* W, int32_t* perm, double* value_out,
                        int* auction_phases_out) {
  if (!c) return FRAM_ERR_INVALID;
  c->last_error.clear();
  if (n < 1 || !W || !perm || !is_device_ptr(W) || !is_device_ptr(perm)) {
    set_err(c, "fram_assign: n >= 1 and device W, perm are required");
    return FRAM_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  FR_TRY(ensure_workspace(c, n));
  Workspace& w = c->ws;
  FR_LAUNCH(launch_lap(W, n, n, perm, &w.scal->lap, w.lap_ws, c->num_sms, c->wait_limit_ns,
                       c->stream, c->lap_searches), "lap kernels");
  FR_CUDA(cudaMemcpyAsync(&w.hscal->lap, &w.scal->lap, sizeof(LapStats), cudaMemcpyDeviceToHost,
                          c->stream),
          "readback");
  FR_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
  c->lap_ran = true;
  if (w.hscal->lap.status != 0) {
    set_err(c, "assignment search did not terminate");
    return FRAM_ERR_TIMEOUT;
  }
  if (value_out) *value_out = w.hscal->lap.value;
  if (auction_phases_out) *auction_phases_out = w.hscal->lap.auction_phases;
  return FRAM_OK;
}

}  // extern "C"
