// Internal launchers of the mixed-precision path (not part of the C ABI).
#pragma once

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

// FP64 (ld x ld) -> BF16 (kind 0) or TF32-rounded FP32 (kind 1), same layout.
int launch_convert_lp(const double* src, void* dst, int ld, int kind, cudaStream_t s);
// dst[j][i] = lp(src[i][j]) over ld x ld.
int launch_transpose_lp(const double* src, void* dst, int ld, int kind, cudaStream_t s);
// Mixed update: N <- (1-alpha) N + alpha D (FP64), writes N^T in low precision
// and delta into st (deterministic last-block combine; ticket starts at 0).
int launch_update_mixed(double* N, const double* D, int ld, int n, double alpha, void* Nt,
                        int kind, double* partials, unsigned* ticket, IterStats* st,
                        cudaStream_t s);

}  // namespace fram
