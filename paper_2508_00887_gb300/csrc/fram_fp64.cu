// FP64 kernels of the FRAM outer iteration (Alg. 1 of arXiv 2508.00887):
// input validation (Sec. 3 graph model), prescaling (Alg. 1 steps 2-3),
// initial assignment (step 1), the gradient GEMMs (step 5, eq. 3), the damped
// update with the delta criterion (steps 7-8) and the objective at the final
// permutation (eq. 1, Sec. 7 matching error).
//
// Reductions are deterministic: fixed per-thread ranges, fixed shuffle trees
// and a last-block combine in block order, so repeated runs give identical
// bits.
#include <math.h>

#include "fram_internal.cuh"

namespace fram {

namespace {

constexpr int kRowThreads = 256;

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = lane < NT / 32 ? red[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;  // valid in warp 0
}

template <int NT>
__device__ __forceinline__ double block_max(double v, double* red) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = lane < NT / 32 ? red[lane] : 0.0;
    r = warp_max(r);
  }
  return r;
}

// ---------------------------------------------------------------- validate
// Finite and >= 0 checks, the max, and the largest asymmetry |M_ij - M_ji|
// (A and B).  One 32 x 32 tile pair per step: tile (bi, bj), bi <= bj, and
// its mirror (bj, bi), both read coalesced into shared memory, so the
// transposed element is a shared-memory read.  The checks and the maxima run
// on bit patterns (integer instructions; nonnegative doubles order like their
// bits); only the asymmetry takes an FP64 subtraction.
constexpr int kVT = 32;

__device__ __forceinline__ void check_entry(double a, int& bad, unsigned long long& mx) {
  unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const bool nonfinite = ((u >> 52) & 0x7FFull) == 0x7FFull;
  const bool negative = (u >> 63) != 0ull && (u << 1) != 0ull;  // -0.0 counts as 0
  if (nonfinite || negative) {
    bad = 1;
    return;
  }
  if ((u << 1) == 0ull) u = 0ull;
  mx = u > mx ? u : mx;
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v,
                                                            unsigned long long* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  unsigned long long r = 0ull;
  if (warp == 0) {
    r = lane < kRowThreads / 32 ? red[lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, r, o);
      r = w > r ? w : r;
    }
  }
  return r;  // valid in thread 0
}

__global__ void __launch_bounds__(kRowThreads) validate_kernel(const double* __restrict__ A,
                                                               const double* __restrict__ B,
                                                               const double* __restrict__ K, int n,
                                                               ValidateStats* st) {
  __shared__ double t0[kVT][kVT + 1], t1[kVT][kVT + 1];
  __shared__ unsigned long long red[kRowThreads / 32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int T = (n + kVT - 1) / kVT;
  const double* mats[3] = {A, B, K};
  for (int which = 0; which < 3; ++which) {
    const double* M = mats[which];
    if (M == nullptr) continue;
    unsigned long long mx = 0ull, as = 0ull;
    int bad = 0;
    for (int p = blockIdx.x; p < T * T; p += gridDim.x) {
      const int bi = p / T, bj = p % T;
      if (bi > bj) continue;  // the same for the whole block
      __syncthreads();        // the previous pair's reads are done
      for (int r = ty; r < kVT; r += kRowThreads / 32) {
        const int i = bi * kVT + r, j = bj * kVT + tx;
        t0[r][tx] = (i < n && j < n) ? M[(size_t)i * n + j] : 0.0;
        const int i2 = bj * kVT + r, j2 = bi * kVT + tx;
        t1[r][tx] = (i2 < n && j2 < n) ? M[(size_t)i2 * n + j2] : 0.0;
      }
      __syncthreads();
      for (int r = ty; r < kVT; r += kRowThreads / 32) {
        const int i = bi * kVT + r, j = bj * kVT + tx;
        if (i < n && j < n) {
          const double a = t0[r][tx];
          check_entry(a, bad, mx);
          if (which < 2) {
            const double t = t1[tx][r];  // M[j][i]
            const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
            const unsigned long long ut = (unsigned long long)__double_as_longlong(t);
            if (((ua >> 52) & 0x7FFull) != 0x7FFull && ((ut >> 52) & 0x7FFull) != 0x7FFull) {
              const unsigned long long d =
                  (unsigned long long)__double_as_longlong(a - t) & 0x7FFFFFFFFFFFFFFFull;
              as = d > as ? d : as;
            }
          }
        }
        const int i2 = bj * kVT + r, j2 = bi * kVT + tx;
        if (bi != bj && i2 < n && j2 < n) check_entry(t1[r][tx], bad, mx);
      }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(&st->bad_value[which], 1);
    const unsigned long long bmx = block_max_u64(mx, red);
    if (threadIdx.x == 0 && bmx) atomicMax(&st->maxbits[which], bmx);
    if (which < 2) {
      const unsigned long long bas = block_max_u64(as, red);
      if (threadIdx.x == 0 && bas) atomicMax(&st->asymbits[which], bas);
    }
  }
}

// ---------------------------------------------------------------- scale
// dst (ld x ld, zero padding) = src (n x n contiguous) * v.
__global__ void scale_kernel(const double* __restrict__ src, int n, double v,
                             double* __restrict__ dst, int ld) {
  for (int i = blockIdx.x; i < ld; i += gridDim.x) {
    for (int j = threadIdx.x; j < ld; j += blockDim.x) {
      double o = 0.0;
      if (i < n && j < n) {
        const double a = src[(size_t)i * n + j];
        o = a * v;
      }
      dst[(size_t)i * ld + j] = o;
    }
  }
}

__global__ void fill_kernel(double* __restrict__ N, int n, int ld, double value) {
  for (int i = blockIdx.x; i < ld; i += gridDim.x)
    for (int j = threadIdx.x; j < ld; j += blockDim.x)
      N[(size_t)i * ld + j] = (i < n && j < n) ? value : 0.0;
}

// ---------------------------------------------------------------- DGEMM
// C = A * B (+ lam * K inside n x n) for ld x ld operands, ld % 64 == 0,
// zero padding outside n x n.  64x64 block tile, k-step 16, 256 threads with
// a 4x4 register tile each.  The epilogue folds max(C) over n x n into an
// ordered-key atomic (SDSN step 1 needs max X).
constexpr int GT = 64, GKS = 16;

__global__ void __launch_bounds__(256) dgemm_kernel(const double* __restrict__ A,
                                                    const double* __restrict__ B,
                                                    double* __restrict__ C, int ld, int n,
                                                    const double* __restrict__ K, double lam,
                                                    unsigned long long* cmax) {
  __shared__ double As[GKS][GT + 2];
  __shared__ double Bs[GKS][GT + 2];
  __shared__ double red[8];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = 0; k0 < ld; k0 += GKS) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      const int m = e >> 4, k = e & 15;
      As[k][m] = A[(size_t)(row0 + m) * ld + k0 + k];
      const int kb = e >> 6, c = e & 63;
      Bs[kb][c] = B[(size_t)(k0 + kb) * ld + col0 + c];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GKS; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double lmax = -INFINITY;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx + 16 * j;
      double v = acc[i][j];
      if (r < n && c < n) {
        if (K != nullptr) v = v + lam * K[(size_t)r * ld + c];
        lmax = fmax(lmax, v);
      }
      C[(size_t)r * ld + c] = v;
    }
  }
  if (cmax != nullptr) {
    const double bm = block_max<256>(lmax, red);
    if (tid == 0 && bm > -INFINITY) atomicMax(cmax, ordered_key(bm));
  }
}

// ---------------------------------------------------------------- update
// Alg. 1 steps 7-8: N <- (1 - alpha) N + alpha D over n x n, and
// delta = ||N_new - N_old||_F / ||N_new||_F with a deterministic combine.
__global__ void __launch_bounds__(kRowThreads) update_kernel(double* __restrict__ N, int ldn,
                                                             const double* __restrict__ D, int ldd,
                                                             int n, double alpha,
                                                             double* __restrict__ partials,
                                                             unsigned* ticket, IterStats* st) {
  __shared__ double red[kRowThreads / 32];
  __shared__ int s_last;
  const double beta = 1.0 - alpha;
  double d2 = 0.0, n2 = 0.0;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    double* nrow = N + (size_t)i * ldn;
    const double* drow = D + (size_t)i * ldd;
    for (int j = threadIdx.x; j < n; j += kRowThreads) {
      const double old = nrow[j];
      const double nn = __dadd_rn(__dmul_rn(beta, old), __dmul_rn(alpha, drow[j]));
      const double d = __dsub_rn(nn, old);
      nrow[j] = nn;
      d2 = fma(d, d, d2);
      n2 = fma(nn, nn, n2);
    }
  }
  const double bd = block_sum<kRowThreads>(d2, red);
  const double bn = block_sum<kRowThreads>(n2, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = bd;
    partials[2 * blockIdx.x + 1] = bn;
    __threadfence();
    s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double sd = 0.0, sn = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kRowThreads) {
    sd += __ldcg(&partials[2 * b]);
    sn += __ldcg(&partials[2 * b + 1]);
  }
  sd = block_sum<kRowThreads>(sd, red);
  sn = block_sum<kRowThreads>(sn, red);
  if (threadIdx.x == 0) {
    st->sum_d2 = sd;
    st->sum_n2 = sn;
    st->delta = sqrt(sd) / sqrt(sn);
    *ticket = 0u;
  }
}

// ---------------------------------------------------------------- objective
// eq. 1 at the permutation: Phi = 1/2 sum_ij A_ij B_{p(i) p(j)} (+ lam sum_i
// K_{i p(i)}), and the Sec. 7 matching error 1/2 sqrt(sum (A_ij - B_p(i)p(j))^2),
// on the unscaled n x n inputs.
__global__ void __launch_bounds__(kRowThreads) objective_kernel(
    const double* __restrict__ A, const double* __restrict__ B, const double* __restrict__ K,
    double lam, int n, const int32_t* __restrict__ perm, double* __restrict__ partials,
    unsigned* ticket, ObjStats* st) {
  __shared__ double red[kRowThreads / 32];
  __shared__ int s_last;
  double s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int pi = perm[i];
    const double* arow = A + (size_t)i * n;
    const double* brow = B + (size_t)pi * n;
    for (int j = threadIdx.x; j < n; j += kRowThreads) {
      const double a = arow[j];
      const double b = brow[perm[j]];
      s1 = fma(a, b, s1);
      const double d = a - b;
      s2 = fma(d, d, s2);
    }
    if (K != nullptr && threadIdx.x == 0) s3 += K[(size_t)i * n + pi];
  }
  s1 = block_sum<kRowThreads>(s1, red);
  s2 = block_sum<kRowThreads>(s2, red);
  s3 = block_sum<kRowThreads>(s3, red);
  if (threadIdx.x == 0) {
    partials[3 * blockIdx.x] = s1;
    partials[3 * blockIdx.x + 1] = s2;
    partials[3 * blockIdx.x + 2] = s3;
    __threadfence();
    s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double t1 = 0.0, t2 = 0.0, t3 = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kRowThreads) {
    t1 += __ldcg(&partials[3 * b]);
    t2 += __ldcg(&partials[3 * b + 1]);
    t3 += __ldcg(&partials[3 * b + 2]);
  }
  t1 = block_sum<kRowThreads>(t1, red);
  t2 = block_sum<kRowThreads>(t2, red);
  t3 = block_sum<kRowThreads>(t3, red);
  if (threadIdx.x == 0) {
    st->objective = 0.5 * t1 + lam * t3;
    st->match_error = 0.5 * sqrt(t2);
    *ticket = 0u;
  }
}

// Node-attribute affinity K = F Ft^T (eq. 1's node term, eq. 3's lambda F F~^T)
// for n x d row-major F, Ft and an n x n row-major K: 64 x 64 output tiles,
// 4 x 4 per thread, d staged through shared memory in chunks of 16 with zero
// fill past n and d.  Each entry sums over k in increasing order.
constexpr int NT_T = 64, NT_K = 16;

__global__ void __launch_bounds__(256) nt_gemm_kernel(const double* __restrict__ F,
                                                      const double* __restrict__ Ft, int n, int d,
                                                      double* __restrict__ K) {
  __shared__ double sa[NT_K][NT_T + 1];
  __shared__ double sb[NT_K][NT_T + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = blockIdx.y * NT_T, c0 = blockIdx.x * NT_T;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < d; k0 += NT_K) {
    for (int e = threadIdx.x; e < NT_T * NT_K; e += 256) {
      const int r = e / NT_K, k = e % NT_K;
      const bool kin = k0 + k < d;
      sa[k][r] = (r0 + r < n && kin) ? F[(size_t)(r0 + r) * d + k0 + k] : 0.0;
      sb[k][r] = (c0 + r < n && kin) ? Ft[(size_t)(c0 + r) * d + k0 + k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NT_K; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = sa[k][ty + 16 * q];
        b[q] = sb[k][tx + 16 * q];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[q][p] = fma(a[q], b[p], acc[q][p]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int r = r0 + ty + 16 * q, c = c0 + tx + 16 * p;
      if (r < n && c < n) K[(size_t)r * n + c] = acc[q][p];
    }
}

template <typename T>
__global__ void max_kernel(const T* __restrict__ X, int ldx, int n, unsigned long long* out) {
  __shared__ double red[kRowThreads / 32];
  double m = -INFINITY;
  for (int i = blockIdx.x; i < n; i += gridDim.x)
    for (int j = threadIdx.x; j < n; j += kRowThreads)
      m = fmax(m, (double)X[(size_t)i * ldx + j]);
  const double bm = block_max<kRowThreads>(m, red);
  if (threadIdx.x == 0 && bm > -INFINITY) atomicMax(out, ordered_key(bm));
}

// Waits at a grid barrier sized for gridDim.x + 1 CTAs: nothing can complete
// it, so every CTA leaves through the time limit and records DEV_TIMEOUT.
__global__ void wait_selftest_kernel(GridBarrier* bar, int* status, uint64_t limit_ns) {
  __shared__ int s_flag;
  unsigned gen = 0;
  grid_sync(bar, gridDim.x + 1, gen, limit_ns, status, &s_flag);
}

int grid_rows(int rows) { return rows < 1 ? 1 : (rows < 1184 ? rows : 1184); }

}  // namespace

// ---------------------------------------------------------------- launchers
int launch_validate(const double* A, const double* B, const double* K, int n, ValidateStats* st,
                    cudaStream_t s) {
  const int T = (n + kVT - 1) / kVT;
  validate_kernel<<<grid_rows(T * T), kRowThreads, 0, s>>>(A, B, K, n, st);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_scale(const double* src, int n, double v, double* dst, int ld, cudaStream_t s) {
  scale_kernel<<<grid_rows(ld), kRowThreads, 0, s>>>(src, n, v, dst, ld);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_fill_assignment(double* N, int n, int ld, double value, cudaStream_t s) {
  fill_kernel<<<grid_rows(ld), kRowThreads, 0, s>>>(N, n, ld, value);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_dgemm(const double* A, const double* B, double* C, int ld, int n, const double* K,
                 double lam, unsigned long long* cmax_key, cudaStream_t s) {
  if (ld % GT != 0) return -1;
  dim3 grid(ld / GT, ld / GT);
  dgemm_kernel<<<grid, 256, 0, s>>>(A, B, C, ld, n, K, lam, cmax_key);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_node_affinity(const double* F, const double* Ft, int n, int d, double* K,
                         cudaStream_t s) {
  const int tiles = (n + NT_T - 1) / NT_T;
  nt_gemm_kernel<<<dim3(tiles, tiles), 256, 0, s>>>(F, Ft, n, d, K);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_max(const double* X, int ldx, int n, unsigned long long* out, cudaStream_t s) {
  max_kernel<double><<<grid_rows(n), kRowThreads, 0, s>>>(X, ldx, n, out);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_max_f32(const float* X, int ldx, int n, unsigned long long* out, cudaStream_t s) {
  max_kernel<float><<<grid_rows(n), kRowThreads, 0, s>>>(X, ldx, n, out);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

size_t update_partials_elems(int n) { return 3 * (size_t)grid_rows(n); }

int launch_update(double* N, int ldn, const double* D, int ldd, int n, double alpha, IterStats* st,
                  double* partials, unsigned* ticket, cudaStream_t s) {
  update_kernel<<<grid_rows(n), kRowThreads, 0, s>>>(N, ldn, D, ldd, n, alpha, partials, ticket,
                                                     st);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_wait_selftest(GridBarrier* bar, int* status, int blocks, uint64_t limit_ns,
                         cudaStream_t s) {
  wait_selftest_kernel<<<blocks, 32, 0, s>>>(bar, status, limit_ns);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_objective(const double* A, const double* B, const double* K, double lam, int n,
                     const int32_t* perm, ObjStats* st, double* partials, unsigned* ticket,
                     cudaStream_t s) {
  objective_kernel<<<grid_rows(n), kRowThreads, 0, s>>>(A, B, K, lam, n, perm, partials, ticket,
                                                        st);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace fram
