// Internal launchers of the mixed-precision path (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fram_internal.cuh"

namespace fram {

// C = A * Bop^T on ld x ld K-major operands with tcgen05 tensor cores.
// kind: 0 = BF16 operands, 1 = TF32 (FP32 storage).  out_kind: 0 = FP32,
// 1 = BF16, 2 = TF32-rounded FP32.  Optional lambda*K term and max(C) over
// the leading n x n block.  err receives DEV_TIMEOUT if a wait expired.
int launch_gemm_tc(const void* A, const void* Bop, void* C, int ld, int n, int kind, int out_kind,
                   const double* Kmat, double lam, unsigned long long* cmax, int* err,
                   uint64_t limit_ns, cudaStream_t s);

// One problem of a grouped tensor-core GEMM launch (C = A * Bop^T, ld x ld,
// 128 x 128 tiles, no K term).  Tensor maps first: the array is copied to
// 64-byte-aligned device memory and read by the TMA unit from there.
struct GemmGroupProblem {  // CUtensorMap members keep it 64-byte aligned
  CUtensorMap ma, mb;
  void* C;
  unsigned long long* cmax;  // optional max(C) over the leading n x n block
  int* err;                  // DEV_TIMEOUT if a wait of the launch expired
  int ld, n;
  int tile0;                 // set by the launcher
};

// Fill q's tensor maps and pointers (host only; no device work).  False on
// a misaligned operand or a failed encode.
bool make_group_problem(GemmGroupProblem* q, const void* A, const void* Bop, void* C, int ld,
                        int n, int kind, unsigned long long* cmax, int* err);
// All `count` problems (same kind and out_kind) in one persistent launch;
// dp: device array of count GemmGroupProblem (64-byte aligned), written here.
int launch_gemm_tc_group(GemmGroupProblem* hp, int count, int kind, int out_kind, void* dp,
                         size_t dp_bytes, uint64_t limit_ns, cudaStream_t s);

// FP64 (ld x ld) -> BF16 (kind 0) or TF32-rounded FP32 (kind 1), same layout.
int launch_convert_lp(const double* src, void* dst, int ld, int kind, cudaStream_t s);
// dst[j][i] = lp(src[i][j]) over ld x ld.
int launch_transpose_lp(const double* src, void* dst, int ld, int kind, cudaStream_t s);
// One problem of a grouped mixed update launch (see launch_update_mixed).
struct UpdGroupProblem {
  double* N;
  const double* D;
  void* Nt;
  double* partials;
  unsigned* ticket;
  IterStats* st;
  double alpha;
  int ld, n;
  int blk0, nblk;  // set by the launcher
};
// All `count` updates (same kind) in one launch, each bit-identical to its
// solo launch; dp: device array of count UpdGroupProblem, written here.
int launch_update_mixed_group(UpdGroupProblem* hp, int count, int kind, void* dp,
                              size_t dp_bytes, cudaStream_t s);

// Mixed update: N <- (1-alpha) N + alpha D (FP64), writes N^T in low precision
// and delta into st (deterministic last-block combine; ticket starts at 0).
int launch_update_mixed(double* N, const double* D, int ld, int n, double alpha, void* Nt,
                        int kind, double* partials, unsigned* ticket, IterStats* st,
                        cudaStream_t s);

}  // namespace fram
