// Internal declarations shared by the FRAM CUDA translation units.
// Nothing here is part of the public C ABI (include/fram.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace fram {

// Device-side status codes (written into a status word by kernels).
enum DevStatus : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_DEGENERATE = 2 };

// Default limit for every device-side wait (grid barriers, flags).
constexpr uint64_t kWaitLimitNs = 4000000000ull;  // 4 s

// ------------------------------------------------------------ host helpers
// A launch fact computed once per device (a kernel attribute set, an
// occupancy, the SM count): function attributes are per device, and several
// contexts -- on several devices, or the serving thread beside the caller's
// -- may ask at once.  compute() returns the value to keep; only positive
// values are kept, so a failed query (<= 0) is retried on the next call.
constexpr int kMaxDevices = 64;

struct DeviceCache {
  std::mutex mu;
  int val[kMaxDevices] = {};
};

template <typename F>
int device_cached(DeviceCache& c, F compute) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return compute();
  std::lock_guard<std::mutex> lk(c.mu);
  if (c.val[dev] > 0) return c.val[dev];
  const int v = compute();
  if (v > 0) c.val[dev] = v;
  return v;
}

// ------------------------------------------------------------ device helpers
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile_s32(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

// FP64 a + b and a - b issued as fma.f64 with a 1.0 that the compiler cannot
// see (callers read it from their kernel arguments), so that it cannot fold
// them back into add.f64.  Exact: a * 1 is exact, so the fma rounds a + b
// once, as add.f64 does, signed zeros and infinities included.  On this GPU
// fma.f64 issues at 1.89 operations per SM per clock against 1.59 for
// add.f64 (measured with eight independent chains per thread).
__device__ __forceinline__ double add64(double a, double b, double one) {
  double d;
  asm("fma.rn.f64 %0, %1, %2, %3;" : "=d"(d) : "d"(a), "d"(one), "d"(b));
  return d;
}
__device__ __forceinline__ double sub64(double a, double b, double one) {  // a - b
  double d;
  asm("fma.rn.f64 %0, %1, %2, %3;" : "=d"(d) : "d"(b), "d"(-one), "d"(a));
  return d;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Max of nonnegative doubles through their bit patterns (monotone for +0..+inf).
// -0.0 and negatives are mapped to +0 first.
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  double c = v > 0.0 ? v : 0.0;
  atomicMax(addr, (unsigned long long)__double_as_longlong(c));
}

// Order-preserving map of a double onto uint64 (for atomicMax of any sign);
// key 0 sorts below every value and means "no value".
__host__ __device__ __forceinline__ unsigned long long ordered_key(double v) {
#ifdef __CUDA_ARCH__
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
#else
  unsigned long long b;
  __builtin_memcpy(&b, &v, 8);
#endif
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__host__ __device__ __forceinline__ double from_ordered_key(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double v;
  __builtin_memcpy(&v, &b, 8);
  return v;
#endif
}

// Grid-wide barrier for a co-resident (cooperatively launched) grid.
// State must be zeroed before the launch.  Every wait is limited in time:
// on expiry the block records DEV_TIMEOUT, raises `abort`, and returns false;
// blocks that see `abort` also return false.  Callers stop on false.
struct GridBarrier {
  unsigned count;
  unsigned gen;
  int abort;
  int pad;
};

__device__ __forceinline__ bool grid_sync(GridBarrier* b, unsigned nblocks, unsigned& gen,
                                          uint64_t limit_ns, int* status, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = gen + 1;
    __threadfence();
    const unsigned prev = atomicAdd(&b->count, 1u);
    if (prev == nblocks - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicExch(&b->gen, target);
    } else {
      const uint64_t t0 = globaltimer_ns();
      while (true) {
        if ((int)(ld_acquire_u32(&b->gen) - target) >= 0) break;
        if (ld_volatile_s32(&b->abort)) { ok = 0; break; }
        if (globaltimer_ns() - t0 > limit_ns) {
          atomicCAS(status, DEV_OK, DEV_TIMEOUT);
          atomicExch(&b->abort, 1);
          ok = 0;
          break;
        }
        __nanosleep(40);
      }
    }
    __threadfence();
    gen = target;
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// Barrier on a counter that only grows: the k-th barrier of the launch waits
// until the counter reaches k * nblocks.  Time-limited (see GridBarrier).
__device__ __forceinline__ bool grid_sync_epoch(GridBarrier* b, unsigned target,
                                                uint64_t limit_ns, int* status, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    // The barrier above orders the CTA's writes before thread 0's release.
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&b->count) : "memory");
    if ((int)(ld_acquire_u32(&b->count) - target) < 0) {
      const uint64_t t0 = globaltimer_ns();
      unsigned polls = 0;
      while ((int)(ld_acquire_u32(&b->count) - target) < 0) {
        if ((++polls & 63u) == 0) {
          if (ld_volatile_s32(&b->abort)) {
            ok = 0;
            break;
          }
          if (globaltimer_ns() - t0 > limit_ns) {
            atomicCAS(status, DEV_OK, DEV_TIMEOUT);
            atomicExch(&b->abort, 1);
            ok = 0;
            break;
          }
        }
      }
    }
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// ------------------------------------------------------------ SDSN state
struct SdsnStats {
  int sweeps;
  int converged;
  int status;   // DevStatus
  int pad;
  double gamma;
  double xmax;
};

// Per-iteration scalars of the outer loop, read back by the host.
struct IterStats {
  SdsnStats sdsn;     // SDSN of this iteration (FP64 path) or its FP32 phase (mixed)
  SdsnStats polish;   // FP64 polish phase (mixed paths)
  double delta;
  double sum_d2;
  double sum_n2;
  int gemm_err;       // tensor-core GEMM wait expired (mixed paths)
  int pad;
};

struct LapStats {
  int augmented;       // augmenting paths of the exact completion
  int status;          // 0 ok, 1 the search did not terminate
  int auction_phases;  // epsilon-scaling phases completed, -1 if the auction did not run
  int repeats;         // concurrent completion: searches repeated after a conflicting commit
  double value;
  long long steps;     // Dijkstra steps of the last completion pass, repeated searches included
};

struct ObjStats {
  double objective;
  double match_error;
};

struct ValidateStats {
  unsigned long long maxbits[3];   // max of A, B, K (nonneg doubles as bits)
  unsigned long long asymbits[2];  // max |A - A^T|, |B - B^T|
  int bad_value[3];                // negative or non-finite entries seen
  int pad;
};

// ------------------------------------------------------------ launchers
// Each returns the number of kernels it launched (>= 0) or -1 on a launch
// error (cudaGetLastError() holds the cause).

int launch_validate(const double* A, const double* B, const double* K, int n,
                    ValidateStats* st, cudaStream_t s);
// dst (ld x ld, zero padding) = src (n x n contiguous) * v.
int launch_scale(const double* src, int n, double v, double* dst, int ld, cudaStream_t s);
int launch_fill_assignment(double* N, int n, int ld, double value, cudaStream_t s);
int launch_dgemm(const double* A, const double* B, double* C, int ld, int n, const double* K,
                 double lam, unsigned long long* cmax_bits, cudaStream_t s);
// Sparse-graph gradient (FP64 path): CSR build and products.
int launch_csr_count(const double* M, int ld, int n, int* rowcnt, cudaStream_t s);
int launch_csr_scan(const int* rowcnt, int n, int* rowptr, cudaStream_t s);
int launch_csr_fill(const double* M, int ld, int n, const int* rowptr, int* col, double* val,
                    cudaStream_t s);
int launch_spmm(const int* rowptr, const int* col, const double* val, int n, const double* D,
                int ld, double* C, cudaStream_t s);
int launch_transpose(const double* Src, double* Dst, int ld, int n, const double* Kmat,
                     double lam, unsigned long long* cmax, cudaStream_t s);
int launch_node_affinity(const double* F, const double* Ft, int n, int d, double* K,
                         cudaStream_t s);
int launch_max(const double* X, int ldx, int n, unsigned long long* key, cudaStream_t s);
int launch_max_f32(const float* X, int ldx, int n, unsigned long long* key, cudaStream_t s);

struct SdsnLaunch {
  int n;
  const void* X;  int ldx;     // FP64 or FP32 gradient
  void* Y;        int ldy;     // output (may alias X when the types match)
  int in_fp32 = 0;             // X is FP32
  int out_fp32 = 0;            // Y and the sweep arithmetic are FP32
  int mode = 0;                // 0: scale X (Alg. 2 step 1); 1: continue from Y0 = X
  int barrier_zeroed = 0;      // the caller zeroed *barrier already (grouped launches)
  double theta, gamma_tol;
  int max_sweeps;
  const unsigned long long* xmax_key;   // max(X) as an ordered key (mode 0)
  const SdsnStats* gate = nullptr;      // skip the sweeps if gate->gamma <= gate_tol
  double gate_tol = 0.0;
  SdsnStats* stats;
  double* partials;            // workspace, sdsn_partials_elems(n, ...) doubles
  GridBarrier* barrier;        // zeroed by the launcher
  uint64_t limit_ns;
};
size_t sdsn_partials_elems(int n, int max_blocks);
// Exact FRA projection (FP64): Y holds X on entry and D on return (ld-strided),
// Yt is n x n scratch, ws holds fra_workspace_elems doubles.  stats->gamma
// gets the row residual max_i |sum_j D_ij - 1| of the returned D.
size_t fra_workspace_elems(int n, int num_sms);
int launch_fra(double* Y, int ldy, double* Yt, int ldt, int n, const unsigned long long* xmax_key,
               double theta, double tol, int max_sweeps, double* ws, GridBarrier* bar,
               SdsnStats* stats, uint64_t limit_ns, int num_sms, cudaStream_t s);
int launch_sdsn_fp64(const SdsnLaunch& L, int num_sms, cudaStream_t s);
// FP32 SDSN of one problem on chip (2 <= n <= 1024, mode 0, no gate): one
// or two warps up to n = 64, one thread-block cluster above.  1 launched, 0
// not applicable (use the grid form), -1 error.
int launch_sdsn_cluster(const SdsnLaunch& L, cudaStream_t s);
// On-chip class of a problem, in [0, kSdsnClusterClasses) (0: neither form
// applies); problems of one class can share one grouped launch, each on its
// own cluster or CTA.
constexpr int kSdsnClusterClasses = 9;
int sdsn_cluster_class(const SdsnLaunch& L);
int launch_sdsn_cluster_group(const SdsnLaunch* L, int count, void* ddesc, size_t ddesc_bytes,
                              cudaStream_t s);
size_t sdsn_cluster_desc_bytes();
// The mixed paths' FP64 polish (FP32 input, mode 1) for 2 <= n <= 64 in one
// CTA of warps: 1 launched, 0 not applicable (use the grid form), -1 error;
// and many such polishes at once (every problem must apply).
int launch_sdsn_polish_small(const SdsnLaunch& L, cudaStream_t s);
int launch_sdsn_polish_small_group(const SdsnLaunch* L, int count, void* ddesc,
                                   size_t ddesc_bytes, cudaStream_t s);
bool sdsn_polish_small_applies(const SdsnLaunch& L);
int launch_sdsn(const SdsnLaunch& L, int num_sms, cudaStream_t s);
// Several problems (same precision pair) in one cooperative launch of at most
// max_blocks CTAs; ddesc is device scratch of sdsn_group_desc_bytes(count).
int launch_sdsn_group(const SdsnLaunch* L, int count, int max_blocks, void* ddesc,
                      size_t ddesc_bytes, int num_sms, cudaStream_t s);
size_t sdsn_group_desc_bytes(int count);
// CTAs of the single-problem SDSN grid for size n (what fram_sdsn uses).
int sdsn_grid_blocks(int n, int num_sms);

int launch_update(double* N, int ldn, const double* D, int ldd, int n, double alpha,
                  IterStats* st, double* partials, unsigned* ticket, cudaStream_t s);
size_t update_partials_elems(int n);

// searches: concurrent searches of the cluster completion (n >= 1024);
// 0 = the default, 1 = one search at a time.
int launch_lap(const double* W, int ldw, int n, int32_t* perm, LapStats* st, void* ws,
               int num_sms, uint64_t limit_ns, cudaStream_t s, int searches = 0);
size_t lap_workspace_bytes(int n);

int launch_wait_selftest(GridBarrier* bar, int* status, int blocks, uint64_t limit_ns,
                         cudaStream_t s);

int launch_objective(const double* A, const double* B, const double* K, double lam, int n,
                     const int32_t* perm, ObjStats* st, double* partials, unsigned* ticket,
                     cudaStream_t s);

}  // namespace fram
