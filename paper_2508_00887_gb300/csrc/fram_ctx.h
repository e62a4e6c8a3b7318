// Host-side context and workspace of the FRAM library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/fram.h"
#include "fram_internal.cuh"

namespace fram {

// Device scalars of one solve.  `lap` and `obj` are adjacent: they are read
// back with one copy.  `iter` and `xmax_key` are adjacent: the mixed loop
// clears both with one memset per outer iteration.
struct DevScalars {
  IterStats iter;
  unsigned long long xmax_key;
  ValidateStats val;
  LapStats lap;
  ObjStats obj;
  GridBarrier bar;
  unsigned ticket_update;
  unsigned ticket_obj;
};

// Device workspace of the single-pair path, grown on demand.  Matrices use a
// leading dimension ld = n rounded up to 128 with zero padding.
struct Workspace {
  int cap_n = 0, cap_ld = 0;
  size_t bytes = 0;
  double *As = nullptr, *Bs = nullptr, *Ks = nullptr;  // prescaled inputs
  double *N = nullptr, *T = nullptr, *X = nullptr;     // assignment, A*N, gradient/SDSN
  double *A0 = nullptr, *B0 = nullptr, *K0 = nullptr;  // staged host inputs
  int32_t* perm = nullptr;
  void* lap_ws = nullptr;
  double* partials = nullptr;       // block partials of update / objective
  double* sdsn_partials = nullptr;  // SDSN row/column/tile partials
  DevScalars* scal = nullptr;
  DevScalars* hscal = nullptr;      // pinned host mirror
  void* mixed = nullptr;            // low-precision shadows (mixed paths)
  int mixed_cap_n = 0;
  // Sparse gradient (FP64 path): CSR of A_s and of B_s^T, grown on demand.
  int* sp_cnt = nullptr;            // [n] row counts
  int* sp_rowptr[2] = {nullptr, nullptr};
  int* sp_col[2] = {nullptr, nullptr};
  double* sp_val[2] = {nullptr, nullptr};
  int sp_cap_n = 0;
  size_t sp_cap_nnz[2] = {0, 0};
  bool sp_on[2] = {false, false};   // this solve uses CSR for A / for B
  void release();
  static size_t bytes_for(int n, int num_sms);
};

}  // namespace fram

struct fram_ctx {
  int device = 0, num_sms = 0, cc_major = 0, cc_minor = 0;
  size_t budget = 0;
  std::atomic<size_t> serve_bytes{0};  // device bytes held by serving slots
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t evp[5] = {};  // phase boundaries inside one outer iteration
  std::string last_error;
  std::atomic<uint64_t> launches{0};
  uint64_t wait_limit_ns = fram::kWaitLimitNs;
  double sparse_density = 0.2;  // FP64 gradient uses CSR up to this fraction of nonzeros
  int lap_searches = 0;         // concurrent LAP searches (0 = default, 1 = sequential)
  bool lap_ran = false;         // an assignment has run (fram_lap_last_stats)
  std::mutex mu;        // serialises the synchronous entry points
  std::mutex serve_mu;  // guards creation of the serving scheduler
  fram::Workspace ws;
  void* batched = nullptr;
  void* serve = nullptr;
};

namespace fram {

void set_err(fram_ctx* c, const char* fmt, ...);
fram_status cuda_fail(fram_ctx* c, cudaError_t e, const char* what);
bool is_device_ptr(const void* p);
// is_device_ptr for many pointers in one call: remembers the address range
// of every device allocation it has classified (cuMemGetAddressRange), so a
// pointer inside a known range needs no driver query.  Valid while those
// allocations stay alive, i.e. within one API call.
class PtrClassifier {
 public:
  bool is_device(const void* p);

 private:
  std::vector<std::pair<uintptr_t, uintptr_t>> ranges_;  // [base, end), sorted by base
};
int round_ld(int n);
fram_status ensure_workspace(fram_ctx* c, int n);
fram_status ensure_mixed(fram_ctx* c, int n);
fram_status check_params(fram_ctx* c, const fram_params& p);
fram_status dev_status(fram_ctx* c, int st, const char* where);
// Elapsed ms between phase events a and b of the current iteration.
double phase_ms(fram_ctx* c, int a, int b);
fram_status stage_in(fram_ctx* c, const double* src, size_t count, double* staging,
                     const double** out);
fram_status solve_one(fram_ctx* c, int n, const double* A, const double* B, const double* K,
                      const fram_params& p, double* X_out, int32_t* perm_out, fram_info* info);

// Mixed-precision outer loop (fram_mixed.cu).
size_t mixed_bytes_for(int n);
fram_status prepare_sparse(fram_ctx* c, int n);
fram_status fp64_gradient(fram_ctx* c, int n, bool withK, double lam, unsigned long long* cmax);
fram_status solve_mixed_loop(fram_ctx* c, int n, bool has_K, const fram_params& p,
                             fram_info* inf);
fram_status mixed_gradient(fram_ctx* c, int n, bool has_K, double lam, int kind, float** X32);

// Batched and serving state (fram_batched.cu, fram_serve.cu).
void batched_release(fram_ctx* c);
void serve_shutdown(fram_ctx* c);

}  // namespace fram
