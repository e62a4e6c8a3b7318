// Batched FRAM for many small pairs (n <= 64) in one persistent launch.
//
// Each CTA takes pairs from a work queue (one atomic per pair, pairs sorted
// by decreasing n on the host) and runs the whole of Alg. 1 + Alg. 2 + eq. 2
// of arXiv 2508.00887 for that pair in shared memory:
//   validation and prescale (Sec. 3; Alg. 1 steps 2-3), N0 = 11^T/n (reading
//   (i)), per outer iteration the two gradient products (step 5, FFMA/DFMA on
//   64 x 64 zero-padded tiles), SDSN (Alg. 2, eq. 7), the FP64 update and
//   delta (steps 7-8), then the Hungarian assignment (eq. 2; one warp, row
//   argmax warm start + shortest augmenting paths with the columns' state in
//   registers) and the objective (eq. 1, Sec. 7) on the unscaled inputs.
// T = double is the FP64 path (same arithmetic as the single-pair FP64
// path); T = float runs the gradient and SDSN in FP32 and keeps N, the
// update and delta in FP64, with the mixed paths' rounding-floor stop.
// Nothing in the kernel waits on another CTA.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "fram_ctx.h"

namespace fram {

namespace {

constexpr int NMAX = 64;
constexpr int LDS = NMAX + 1;

struct BatchDesc {
  int n;
  int index;           // position in the caller's arrays (host bookkeeping)
  long long off_mat;   // element offset of the pair's n x n blocks
  long long off_vec;   // element offset of the pair's n-vectors
};

struct BatchInfo {
  int outer_iters, total_sweeps, status, lap_aug;
  double delta, gamma, objective, match_error, assignment_value;
};

struct BatchArgs {
  const BatchDesc* desc;
  int count;
  const double* A;
  const double* B;
  double* Nout;
  int32_t* perm;
  BatchInfo* info;
  unsigned* queue;
  double lam, alpha, theta, delta_tol, gamma_tol, mixed_delta_tol, stall_ratio, stall_below;
  int max_outer, max_sweeps, use_stall;
  int team_split;  // team kernel: pairs with n > team_split run on two warps (tile edge 64)
};

enum : int { PAIR_OK = 0, PAIR_INVALID = 1, PAIR_DEGENERATE = 2 };

// Shared memory of one CTA: five tiles (A, B, N, T, X/Y), the FP64 copy of
// N (FP64 path only: the FP32 path keeps N in FP32 and fits two CTAs per
// SM), the SDSN vectors and partials, the row potentials and reductions.
template <typename T>
__host__ __device__ constexpr size_t batched_smem_bytes(int nt) {
  return 5 * (size_t)NMAX * LDS * sizeof(T) +
         (sizeof(T) == 8 ? (size_t)NMAX * NMAX * sizeof(double) : 0) +
         4 * (size_t)NMAX * sizeof(T) + (size_t)(nt / 64) * NMAX * sizeof(T) +
         (size_t)NMAX * sizeof(double) + 64 * sizeof(double);
}

// Block reductions over NT threads in a fixed order; warp 0 combines the
// warp results and red[32] broadcasts the total (FP64 instructions are
// scarce on this GPU, so the second level runs in one warp only).
template <int NT>
__device__ __forceinline__ double bsum_level2(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double r = lane < NT / 32 ? red[lane] : 0.0;
    r = warp_sum(r);
    if (lane == 0) red[32] = r;
  }
  __syncthreads();
  return red[32];
}

template <int NT>
__device__ __forceinline__ double bsum(double v, double* red) {
  return bsum_level2<NT>(warp_sum(v), red);
}

// FP32 warp sums, FP64 across warps.
template <int NT>
__device__ __forceinline__ double bsum_f(float v, double* red) {
  return bsum_level2<NT>((double)warp_sum(v), red);
}

template <int NT>
__device__ __forceinline__ double bmax(double v, double* red) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double r = lane < NT / 32 ? red[lane] : -INFINITY;
    r = warp_max(r);
    if (lane == 0) red[32] = r;
  }
  __syncthreads();
  return red[32];
}

__device__ __forceinline__ double relu_d(double y) {
  const long long b = __double_as_longlong(y);
  return __longlong_as_double(b & ~(b >> 63));
}
__device__ __forceinline__ float relu_d(float y) {
  const int b = __float_as_int(y);
  return __int_as_float(b & ~(b >> 31));
}

// C[i][j] = sum_{k<n} Aop[i][k] * Bop[k][j] over the 64 x 64 padded tile.
// Returns the thread's max over i, j < n when want_max.
template <typename T, int NT>
__device__ __forceinline__ T small_gemm(const T* __restrict__ Aop, const T* __restrict__ Bop,
                                        T* __restrict__ C, int n, bool want_max) {
  constexpr int RY = NT / 16;        // rows per step
  constexpr int RA = NMAX / RY;      // row repeats
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[RA][4];
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int k = 0; k < n; ++k) {
    T av[RA], bv[4];
#pragma unroll
    for (int a = 0; a < RA; ++a) av[a] = Aop[(ty + RY * a) * LDS + k];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = Bop[k * LDS + tx + 16 * b];
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
  }
  T mx = T(-INFINITY);
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = ty + RY * a, j = tx + 16 * b;
      C[i * LDS + j] = acc[a][b];
      if (want_max && i < n && j < n) mx = acc[a][b] > mx ? acc[a][b] : mx;
    }
  return mx;
}

// Per-sweep scalars, formed once by thread 0 (FP64 instructions are scarce
// on this GPU, so no other thread touches them): S = sum Y, gamma = S/n - 1,
// the stop flag gamma <= gamma_tol, and c1 = 1/n + S/n^2 in the working type.
template <typename T>
struct SweepCtl {
  double S, g;
  double delta, prev_delta;  // outer-iteration test state (thread 0)
  double inv_sq, inv_n;      // per-pair scalars
  T c1;
  int conv, stop;
};

// One pass of SDSN on Ys (n x n): FIRST scales by `scale`; otherwise the fused
// P1+P2 sweep with arow/bcol.  Leaves row sums in rs, column sums in cs and
// the sweep scalars in *ctl, visible to every thread on return.
template <typename T, int NT, bool FIRST>
__device__ __forceinline__ void small_sdsn_pass(T* Ys, T* rs, T* cs, const T* arow,
                                                const T* bcol, T* cpart, SweepCtl<T>* ctl, int n,
                                                T scale, double inv_n, double inv_n2,
                                                double gtol) {
  constexpr int G = NT / 64;  // row groups
  const int tid = threadIdx.x, c = tid & 63, rg = tid >> 6;
  if (c < n) {
    T acc = T(0);
    const T bc = FIRST ? T(0) : bcol[c];
    for (int r = rg; r < n; r += G) {
      T y = Ys[r * LDS + c];
      y = FIRST ? y * scale : relu_d((y + arow[r]) - bc);
      Ys[r * LDS + c] = y;
      acc += y;
    }
    cpart[rg * NMAX + c] = acc;
  }
  __syncthreads();
  {
    const int r = tid / G, part = tid % G;  // G consecutive lanes per row
    T s = T(0);
    if (r < n)
      for (int j = part; j < n; j += G) s += Ys[r * LDS + j];
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (part == 0 && r < n) rs[r] = s;
  }
  if (tid < n) {
    T s = T(0);
#pragma unroll
    for (int g = 0; g < G; ++g) s += cpart[g * NMAX + tid];
    cs[tid] = s;
  }
  __syncthreads();
  if (tid < 32) {
    double s = 0.0;
    if (tid < n) s += (double)rs[tid];
    if (tid + 32 < n) s += (double)rs[tid + 32];
    s = warp_sum(s);
    if (tid == 0) {
      const double g = s * inv_n - 1.0;
      ctl->S = s;
      ctl->g = g;
      ctl->conv = g <= gtol;
      ctl->c1 = (T)(inv_n + s * inv_n2);
    }
  }
  __syncthreads();
}

// Warp 0: Hungarian on W (n x n, row stride NMAX) for maximum sum.  Lane l
// owns columns l and l + 32; row potentials live in shared memory.
template <typename TW>
__device__ void small_lap(const TW* W, int ldw, int n, double* u, int* rowcol, int* argc,
                          double* rowmax, int* aug_out) {
  const int lane = threadIdx.x & 31;
  // Row argmax (ties -> lowest column).
  for (int i = 0; i < n; ++i) {
    double best = -INFINITY;
    int bj = 0x7fffffff;
    for (int j = lane; j < n; j += 32) {
      const double x = (double)W[i * ldw + j];
      if (x > best) { best = x; bj = j; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      if (ob > best || (ob == best && oj < bj)) { best = ob; bj = oj; }
    }
    if (lane == 0) {
      argc[i] = bj;
      rowmax[i] = best;
    }
  }
  __syncwarp();
  // Column state in registers: slot s <-> column lane + 32 s.
  int colrow[2] = {-1, -1};
  double v[2] = {0.0, 0.0};
  for (int i = 0; i < n; ++i) {  // lowest row claiming a column keeps it
    const int j = argc[i];
    if ((j & 31) == lane && colrow[j >> 5] == -1) colrow[j >> 5] = i;
  }
  for (int i = lane; i < n; i += 32) u[i] = -rowmax[i];
  __syncwarp();
  for (int i = 0; i < n; ++i) {
    const int j = argc[i];
    const int owner = __shfl_sync(0xffffffffu, colrow[(j >> 5) & 1], j & 31);
    if (lane == 0) rowcol[i] = owner == i ? j : -1;
  }
  __syncwarp();
  int aug = 0;
  for (int root = 0; root < n; ++root) {
    if (rowcol[root] != -1) continue;
    ++aug;
    double minv[2] = {INFINITY, INFINITY};
    int used[2] = {0, 0}, way[2] = {-1, -1};
    int i0 = root, j0 = -1, j1 = -1;
    for (int step = 0; step <= n; ++step) {
      const double ui = u[i0];
      double best = INFINITY;
      int bj = 0x7fffffff;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int j = lane + 32 * s;
        if (j < n && !used[s]) {
          const double cur = -(double)W[i0 * ldw + j] - ui - v[s];
          if (cur < minv[s]) { minv[s] = cur; way[s] = j0; }
          if (minv[s] < best) { best = minv[s]; bj = j; }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (ob < best || (ob == best && oj < bj)) { best = ob; bj = oj; }
      }
      const double delta = best;
      j1 = bj;
      __syncwarp();
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int j = lane + 32 * s;
        if (j < n) {
          if (used[s]) {
            v[s] -= delta;
            u[colrow[s]] += delta;
          } else {
            minv[s] -= delta;
          }
        }
      }
      if (lane == 0) u[root] += delta;
      if ((j1 & 31) == lane) used[j1 >> 5] = 1;
      __syncwarp();
      j0 = j1;
      const int nxt = __shfl_sync(0xffffffffu, colrow[(j1 >> 5) & 1], j1 & 31);
      if (nxt == -1) break;
      i0 = nxt;
    }
    // Augment along the predecessor chain.
    int j = j1;
    while (j != -1) {
      const int jp = __shfl_sync(0xffffffffu, way[(j >> 5) & 1], j & 31);
      const int r = jp == -1 ? root : __shfl_sync(0xffffffffu, colrow[(jp >> 5) & 1], jp & 31);
      if ((j & 31) == lane) colrow[j >> 5] = r;
      if (lane == 0) rowcol[r] = j;
      j = jp;
    }
    __syncwarp();
  }
  if (lane == 0) *aug_out = aug;
  __syncwarp();
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 2 : 1) batched_kernel(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* As = reinterpret_cast<T*>(smem);
  T* Bs = As + NMAX * LDS;
  T* Nc = Bs + NMAX * LDS;
  T* Ts = Nc + NMAX * LDS;
  T* Ys = Ts + NMAX * LDS;
  double* N64 = reinterpret_cast<double*>(Ys + NMAX * LDS);  // FP64 path only
  T* rs = reinterpret_cast<T*>(N64 + (sizeof(T) == 8 ? NMAX * NMAX : 0));
  T* cs = rs + NMAX;
  T* arow = cs + NMAX;
  T* bcol = arow + NMAX;
  T* cpart = bcol + NMAX;
  double* u = reinterpret_cast<double*>(cpart + (NT / 64) * NMAX);
  double* red = u + NMAX;  // [0,32) reductions, [32] broadcast slot
  __shared__ int s_pair, s_aug;
  __shared__ SweepCtl<T> ctl;
  __shared__ int rowcol[NMAX], argc[NMAX];
  __shared__ double rowmax[NMAX];
  const int tid = threadIdx.x, c = tid & 63, rg = tid >> 6;
  constexpr int G = NT / 64;

  while (true) {
    __syncthreads();
    if (tid == 0) s_pair = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int pi = s_pair;
    if (pi >= a.count) break;
    const BatchDesc d = a.desc[pi];
    const int n = d.n;
    const double* Ag = a.A + d.off_mat;
    const double* Bg = a.B + d.off_mat;
    BatchInfo info{};

    // Validation (Sec. 3 graph model, reading (vii)) and max for the prescale,
    // on bit patterns: a finite value >= 0 has sign 0 and exponent < 0x7ff,
    // and such values order like their bits.  Only entries that differ from
    // their transpose pay for an FP64 subtraction.
    unsigned long long mAb = 0, mBb = 0;
    double asA = 0.0, asB = 0.0;
    int badi = 0;
    for (int e = tid; e < n * n; e += NT) {
      const int i = e / n, j = e - i * n;
      const unsigned long long xb = (unsigned long long)__double_as_longlong(Ag[e]);
      const unsigned long long yb = (unsigned long long)__double_as_longlong(Bg[e]);
      // valid: finite and >= 0, i.e. +0..+max finite, or -0
      const bool okx = xb < 0x7ff0000000000000ull || xb == 0x8000000000000000ull;
      const bool oky = yb < 0x7ff0000000000000ull || yb == 0x8000000000000000ull;
      if (!okx || !oky) {
        badi = 1;
        continue;
      }
      mAb = mAb > (xb & 0x7fffffffffffffffull) ? mAb : (xb & 0x7fffffffffffffffull);
      mBb = mBb > (yb & 0x7fffffffffffffffull) ? mBb : (yb & 0x7fffffffffffffffull);
      const unsigned long long xtb = (unsigned long long)__double_as_longlong(Ag[j * n + i]);
      const unsigned long long ytb = (unsigned long long)__double_as_longlong(Bg[j * n + i]);
      if (xtb != xb && xtb < 0x7ff0000000000000ull)
        asA = fmax(asA, fabs(__longlong_as_double((long long)xb) -
                             __longlong_as_double((long long)xtb)));
      if (ytb != yb && ytb < 0x7ff0000000000000ull)
        asB = fmax(asB, fabs(__longlong_as_double((long long)yb) -
                             __longlong_as_double((long long)ytb)));
    }
    const double bad = bmax<NT>(badi ? 1.0 : 0.0, red);
    const double mA = bmax<NT>(__longlong_as_double((long long)mAb), red);
    const double mB = bmax<NT>(__longlong_as_double((long long)mBb), red);
    asA = bmax<NT>(asA, red);
    asB = bmax<NT>(asB, red);
    const double cc = fmax(mA, mB);
    if (bad > 0.0 || asA > 1e-12 * fmax(mA, 1.0) || asB > 1e-12 * fmax(mB, 1.0)) {
      info.status = PAIR_INVALID;
    } else if (!(cc > 0.0)) {
      info.status = PAIR_DEGENERATE;
    }
    if (info.status != PAIR_OK) {
      if (tid == 0) a.info[pi] = info;
      continue;
    }
    // Alg. 1 steps 2-3 and the initial N (reading (i)), zero-padded tiles.
    // Scalars once, in thread 0: 1/sqrt(c) scales both graphs by one multiply.
    if (tid == 0) {
      ctl.inv_sq = 1.0 / sqrt(cc);
      ctl.inv_n = 1.0 / n;
    }
    __syncthreads();
    const double inv_n = ctl.inv_n, n0 = inv_n;
    const T inv_n_t = (T)inv_n, inv_sq_t = (T)ctl.inv_sq;
    for (int e = tid; e < NMAX * NMAX; e += NT) {
      const int i = e >> 6, j = e & 63;
      const bool in = i < n && j < n;
      As[i * LDS + j] = in ? (T)Ag[i * n + j] * inv_sq_t : T(0);
      Bs[i * LDS + j] = in ? (T)Bg[i * n + j] * inv_sq_t : T(0);
      Nc[i * LDS + j] = in ? inv_n_t : T(0);
      if (sizeof(T) == 8) N64[i * NMAX + j] = in ? n0 : 0.0;
    }
    __syncthreads();

    const double inv_n2 = inv_n * inv_n;
    const double gtol = a.gamma_tol;
    double delta = INFINITY, g = INFINITY;
    if (tid == 0) ctl.prev_delta = INFINITY;
    int t = 0, sweeps_total = 0;
    while (t < a.max_outer) {
      // Step 5: T = A N, X = T B.
      small_gemm<T, NT>(As, Nc, Ts, n, false);
      __syncthreads();
      const T lm = small_gemm<T, NT>(Ts, Bs, Ys, n, true);
      const double m = bmax<NT>((double)lm, red);
      if (tid == 0) {
        ctl.conv = !(m > 0.0);  // degenerate: max X <= 0
        ctl.c1 = (T)((a.theta / 2.0) / m);
      }
      __syncthreads();
      if (ctl.conv) {
        info.status = PAIR_DEGENERATE;
        break;
      }
      // Step 6: SDSN.
      small_sdsn_pass<T, NT, true>(Ys, rs, cs, arow, bcol, cpart, &ctl, n, ctl.c1, inv_n, inv_n2,
                                   gtol);
      int k = 0;
      while (true) {
        if (k > 0 && ctl.conv) break;  // gamma of the last clamped result (reading (iii))
        if (k >= a.max_sweeps) break;
        const T c1 = ctl.c1;
        if (tid < n) {
          arow[tid] = c1 - rs[tid] * inv_n_t;
          bcol[tid] = cs[tid] * inv_n_t;
        }
        __syncthreads();
        small_sdsn_pass<T, NT, false>(Ys, rs, cs, arow, bcol, cpart, &ctl, n, T(1), inv_n, inv_n2,
                                      gtol);
        ++k;
      }
      if (k > 0) g = ctl.g;
      sweeps_total += k;
      // Steps 7-8.  FP64 path: N in FP64.  FP32 path: N in FP32 with each
      // thread's few squared terms summed in FP32 and the block sums and the
      // delta test in FP64.
      double d2 = 0.0, nn2 = 0.0;
      float d2f = 0.0f, nn2f = 0.0f;
      if (c < n) {
        if (sizeof(T) == 8) {
          for (int r = rg; r < n; r += G) {
            const double old = N64[r * NMAX + c];
            const double nn = __dadd_rn(__dmul_rn(1.0 - a.alpha, old),
                                        __dmul_rn(a.alpha, (double)Ys[r * LDS + c]));
            const double dd = __dsub_rn(nn, old);
            N64[r * NMAX + c] = nn;
            Nc[r * LDS + c] = (T)nn;
            d2 = fma(dd, dd, d2);
            nn2 = fma(nn, nn, nn2);
          }
        } else {
          const float al = (float)a.alpha, bl = (float)(1.0 - a.alpha);
          for (int r = rg; r < n; r += G) {
            const float old = (float)Nc[r * LDS + c];
            const float nn = fmaf(bl, old, al * (float)Ys[r * LDS + c]);
            const float dd = nn - old;
            Nc[r * LDS + c] = (T)nn;
            d2f = fmaf(dd, dd, d2f);
            nn2f = fmaf(nn, nn, nn2f);
          }
        }
      }
      if (sizeof(T) == 8) {
        d2 = bsum<NT>(d2, red);
        nn2 = bsum<NT>(nn2, red);
      } else {
        d2 = bsum_f<NT>(d2f, red);
        nn2 = bsum_f<NT>(nn2f, red);
      }
      ++t;
      // Alg. 1 steps 7-8 test (and the mixed stop rules), thread 0 only.
      if (tid == 0) {
        const double dl = sqrt(d2) / sqrt(nn2);
        int stop = dl <= a.delta_tol || (a.use_stall && dl <= a.mixed_delta_tol);
        if (a.use_stall && a.stall_ratio > 0.0 && dl <= a.stall_below &&
            dl > a.stall_ratio * ctl.prev_delta)
          stop = 1;
        ctl.prev_delta = dl;
        ctl.delta = dl;
        ctl.stop = stop;
      }
      __syncthreads();
      delta = ctl.delta;
      if (ctl.stop) break;
    }
    __syncthreads();
    if (info.status != PAIR_OK) {
      if (tid == 0) a.info[pi] = info;
      continue;
    }
    // Step 10 (eq. 2): warp 0, on N as kept (FP64 path: FP64 copy).
    if (tid < 32) {
      if (sizeof(T) == 8)
        small_lap(N64, NMAX, n, u, rowcol, argc, rowmax, &s_aug);
      else
        small_lap(Nc, LDS, n, u, rowcol, argc, rowmax, &s_aug);
    }
    __syncthreads();
    // Objective (eq. 1) and matching error (Sec. 7) on the unscaled inputs.
    double s1 = 0.0, s2 = 0.0;
    for (int e = tid; e < n * n; e += NT) {
      const int i = e / n, j = e - i * n;
      const double x = Ag[e];
      const double y = Bg[rowcol[i] * n + rowcol[j]];
      s1 = fma(x, y, s1);
      s2 = fma(x - y, x - y, s2);
    }
    double av = 0.0;
    if (tid < n)
      av = sizeof(T) == 8 ? N64[tid * NMAX + rowcol[tid]] : (double)Nc[tid * LDS + rowcol[tid]];
    s1 = bsum<NT>(s1, red);
    s2 = bsum<NT>(s2, red);
    av = bsum<NT>(av, red);
    int32_t* pout = a.perm + d.off_vec;
    for (int i = tid; i < n; i += NT) pout[i] = rowcol[i];
    if (a.Nout != nullptr) {
      double* no = a.Nout + d.off_mat;
      for (int e = tid; e < n * n; e += NT) {
        const int i = e / n, j = e - i * n;
        no[e] = sizeof(T) == 8 ? N64[i * NMAX + j] : (double)Nc[i * LDS + j];
      }
    }
    if (tid == 0) {
      info.outer_iters = t;
      info.total_sweeps = sweeps_total;
      info.delta = delta;
      info.gamma = g;
      info.objective = 0.5 * s1;
      info.match_error = 0.5 * sqrt(s2);
      info.assignment_value = av;
      info.lap_aug = s_aug;
      a.info[pi] = info;
    }
  }
}

// ------------------------------------------------------------ team kernel
// The FP32 form for the keypoint-sized pairs: a CTA of 4 warps holds two
// teams of two warps.  A pair with n <= 32 runs on ONE warp (tile edge 32),
// a pair with 32 < n <= 64 on a team of two (tile edge 64).  Lane c owns
// column c of the tile: its column of N and of the SDSN iterate stay in
// registers for the whole solve, so a sweep (eq. 7) keeps the column sums in
// the lane, forms the row sums by one transposed shuffle tree (two warps add
// their halves through shared memory) and synchronises with __syncwarp or a
// 64-thread named barrier -- no CTA-wide barrier.  The products of step 5
// read A^T and (A N)^T rows as broadcasts; S and gamma are FP32 double-floats
// (TwoSum), so no FP64 instruction runs per sweep.
constexpr int kTeamCT = 128;

template <int TE>
struct TeamLayout {
  static constexpr int SA = TE + 4;  // rows of A^T, (A N)^T and N: 16-byte aligned
  static constexpr int SB = TE + 1;  // B: conflict-free column reads
  static constexpr size_t a = 0;
  static constexpr size_t b = a + (size_t)TE * SA * 4;
  static constexpr size_t t = (b + (size_t)TE * SB * 4 + 15) & ~size_t(15);
  static constexpr size_t part = t + (size_t)TE * SA * 4;  // [2][TE] row partials
  static constexpr size_t arow = part + 2 * (size_t)TE * 4;  // [TE] next sweep's a_i
  static constexpr size_t red = arow + (size_t)TE * 4;       // 8 doubles
  static constexpr size_t u = red + 64;
  static constexpr size_t rowmax = u + (size_t)TE * 8;
  static constexpr size_t rowcol = rowmax + (size_t)TE * 8;
  static constexpr size_t argc = rowcol + (size_t)TE * 4;
  static constexpr size_t misc = argc + (size_t)TE * 4;  // 16 ints
  static constexpr size_t bytes = misc + 64;
};
constexpr size_t kTeamBytes = TeamLayout<64>::bytes;
static_assert(2 * TeamLayout<32>::bytes <= kTeamBytes, "two warp regions in a team region");

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Double-float sum over the 32 lanes (xor butterfly; every lane ends with
// the same hi + lo, because TwoSum recovers the exact error in any order).
__device__ __forceinline__ void warp_sum_df(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
    float s, e;
    two_sum_f(hi, oh, s, e);
    hi = s;
    lo = (lo + ol) + e;
  }
  float s, e;
  two_sum_f(hi, lo, s, e);
  hi = s;
  lo = e;
}

// Transposed sums of y[0..32) over the 32 lanes: each stage halves the
// entries a lane carries (the lane whose offset bit is set keeps the upper
// half), so lane l ends with the warp's total of entry l.  31 shuffles for 32
// row sums; fixed order; y is read, not modified.
template <int OFF, int TE>
__device__ __forceinline__ float team_rows32(const float (&y)[TE], int lane) {
  float v[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const bool hi = lane & 16;
    const float send = hi ? y[OFF + m] : y[OFF + m + 16];
    const float keep = hi ? y[OFF + m + 16] : y[OFF + m];
    v[m] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int w = 8, o = 8; o > 0; w >>= 1, o >>= 1) {
#pragma unroll
    for (int m = 0; m < w; ++m) {
      const bool hi = lane & o;
      const float send = hi ? v[m] : v[m + w];
      const float keep = hi ? v[m + w] : v[m];
      v[m] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

template <int TE>
__device__ __forceinline__ void team_sync(int bar_id) {
  if (TE == 32)
    __syncwarp();
  else
    asm volatile("bar.sync %0, 64;" ::"r"(bar_id) : "memory");
}

// Team-wide max / sum: warp shuffles, then (TE = 64) the two warps through
// shared memory in a fixed order.
template <int TE>
__device__ __forceinline__ double team_max(double v, double* red, int wt, int bar_id) {
  v = warp_max(v);
  if (TE == 32) return v;
  if ((threadIdx.x & 31) == 0) red[wt] = v;
  team_sync<TE>(bar_id);
  const double r = fmax(red[0], red[1]);
  team_sync<TE>(bar_id);
  return r;
}
template <int TE>
__device__ __forceinline__ double team_sum(double v, double* red, int wt, int bar_id) {
  v = warp_sum(v);
  if (TE == 32) return v;
  if ((threadIdx.x & 31) == 0) red[wt] = v;
  team_sync<TE>(bar_id);
  const double r = red[0] + red[1];
  team_sync<TE>(bar_id);
  return r;
}

// FP32 sums per warp, FP64 across the two warps (as the CTA form's bsum_f).
template <int TE>
__device__ __forceinline__ double team_sum_f(float v, double* red, int wt, int bar_id) {
  const double w = (double)warp_sum(v);
  if (TE == 32) return w;
  if ((threadIdx.x & 31) == 0) red[wt] = w;
  team_sync<TE>(bar_id);
  const double r = red[0] + red[1];
  team_sync<TE>(bar_id);
  return r;
}

template <int TE>
__device__ void team_solve(const BatchArgs& a, int pi, unsigned char* region, int wt, int bar_id) {
  using Lay = TeamLayout<TE>;
  constexpr int SA = Lay::SA, SB = Lay::SB;
  float* AsT = reinterpret_cast<float*>(region + Lay::a);
  float* Bs = reinterpret_cast<float*>(region + Lay::b);
  float* TsT = reinterpret_cast<float*>(region + Lay::t);
  float* part = reinterpret_cast<float*>(region + Lay::part);
  float* arow = reinterpret_cast<float*>(region + Lay::arow);
  double* red = reinterpret_cast<double*>(region + Lay::red);
  double* u = reinterpret_cast<double*>(region + Lay::u);
  double* rowmax = reinterpret_cast<double*>(region + Lay::rowmax);
  int* rowcol = reinterpret_cast<int*>(region + Lay::rowcol);
  int* argc = reinterpret_cast<int*>(region + Lay::argc);
  int* misc = reinterpret_cast<int*>(region + Lay::misc);
  const int lane = threadIdx.x & 31;
  const int c = TE == 32 ? lane : lane + 32 * wt;  // this lane's column
  const BatchDesc d = a.desc[pi];
  const int n = d.n;
  const double* Ag = a.A + d.off_mat;
  const double* Bg = a.B + d.off_mat;
  BatchInfo info{};

  // Validation (Sec. 3, reading (vii)) and the prescale's max, on bit
  // patterns as in the CTA form.
  unsigned long long mAb = 0, mBb = 0;
  double asA = 0.0, asB = 0.0;
  int badi = 0;
  for (int e = c; e < n * n; e += TE) {
    const int i = e / n, j = e - i * n;
    const unsigned long long xb = (unsigned long long)__double_as_longlong(Ag[e]);
    const unsigned long long yb = (unsigned long long)__double_as_longlong(Bg[e]);
    const bool okx = xb < 0x7ff0000000000000ull || xb == 0x8000000000000000ull;
    const bool oky = yb < 0x7ff0000000000000ull || yb == 0x8000000000000000ull;
    if (!okx || !oky) {
      badi = 1;
      continue;
    }
    mAb = mAb > (xb & 0x7fffffffffffffffull) ? mAb : (xb & 0x7fffffffffffffffull);
    mBb = mBb > (yb & 0x7fffffffffffffffull) ? mBb : (yb & 0x7fffffffffffffffull);
    const unsigned long long xtb = (unsigned long long)__double_as_longlong(Ag[j * n + i]);
    const unsigned long long ytb = (unsigned long long)__double_as_longlong(Bg[j * n + i]);
    if (xtb != xb && xtb < 0x7ff0000000000000ull)
      asA = fmax(asA, fabs(__longlong_as_double((long long)xb) - __longlong_as_double((long long)xtb)));
    if (ytb != yb && ytb < 0x7ff0000000000000ull)
      asB = fmax(asB, fabs(__longlong_as_double((long long)yb) - __longlong_as_double((long long)ytb)));
  }
  const double bad = team_max<TE>(badi ? 1.0 : 0.0, red, wt, bar_id);
  const double mA = team_max<TE>(__longlong_as_double((long long)mAb), red, wt, bar_id);
  const double mB = team_max<TE>(__longlong_as_double((long long)mBb), red, wt, bar_id);
  asA = team_max<TE>(asA, red, wt, bar_id);
  asB = team_max<TE>(asB, red, wt, bar_id);
  const double cc = fmax(mA, mB);
  if (bad > 0.0 || asA > 1e-12 * fmax(mA, 1.0) || asB > 1e-12 * fmax(mB, 1.0))
    info.status = PAIR_INVALID;
  else if (!(cc > 0.0))
    info.status = PAIR_DEGENERATE;
  if (info.status != PAIR_OK) {
    if (c == 0) a.info[pi] = info;
    return;
  }
  // Alg. 1 steps 2-3 and N0 = 11^T/n (reading (i)); zero padding.
  const double inv_n = 1.0 / n;
  const float inv_n_f = (float)inv_n, inv_n2_f = (float)(inv_n * inv_n);
  const float inv_sq = (float)(1.0 / sqrt(cc));
  for (int i = 0; i < TE; ++i) {
    const bool in = i < n && c < n;
    AsT[c * SA + i] = in ? (float)Ag[i * n + c] * inv_sq : 0.f;  // A^T[c][i] = A[i][c]
    Bs[i * SB + c] = in ? (float)Bg[i * n + c] * inv_sq : 0.f;
  }
  float ncol[TE], y[TE];
#pragma unroll
  for (int i = 0; i < TE; ++i) ncol[i] = (i < n && c < n) ? inv_n_f : 0.f;
  team_sync<TE>(bar_id);
  const double thr = (double)n * (1.0 + a.gamma_tol);
  const float thr_hi = (float)thr, thr_lo = (float)(thr - (double)thr_hi);
  const float al = (float)a.alpha, bl = (float)(1.0 - a.alpha);
  double prev_delta = INFINITY, delta = INFINITY, g = INFINITY;
  float Shi = 0.f, Slo = 0.f;
  int t = 0, sweeps_total = 0;
  while (t < a.max_outer) {
    // Step 5, T = A N: column c of T from column c of N and rows of A^T.
    // Column c of N goes to row c of the (A N)^T region first, which only
    // this lane reads and then overwrites with column c of T: the k loop can
    // then index it at run time (a register array cannot be), which keeps
    // the loop rolled and the kernel's code small.
    team_sync<TE>(bar_id);  // the previous iteration's reads of (A N)^T are done
    float4* const own = reinterpret_cast<float4*>(TsT + c * SA);  // (A N)^T[c][i] = T[i][c]
#pragma unroll
    for (int q = 0; q < TE / 4; ++q)
      own[q] = make_float4(ncol[4 * q], ncol[4 * q + 1], ncol[4 * q + 2], ncol[4 * q + 3]);
#pragma unroll
    for (int i = 0; i < TE; ++i) y[i] = 0.f;
#pragma unroll 1
    for (int k4 = 0; k4 < n; k4 += 4) {
      const float4 n4 = own[k4 >> 2];
      const float nk4[4] = {n4.x, n4.y, n4.z, n4.w};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int k = k4 + h;
        if (k < n) {
          const float nk = nk4[h];
          const float4* ar = reinterpret_cast<const float4*>(AsT + k * SA);
#pragma unroll
          for (int q = 0; q < TE / 4; ++q) {
            const float4 av = ar[q];
            y[4 * q] = fmaf(av.x, nk, y[4 * q]);
            y[4 * q + 1] = fmaf(av.y, nk, y[4 * q + 1]);
            y[4 * q + 2] = fmaf(av.z, nk, y[4 * q + 2]);
            y[4 * q + 3] = fmaf(av.w, nk, y[4 * q + 3]);
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < TE / 4; ++q)
      own[q] = make_float4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3]);
    team_sync<TE>(bar_id);
    // X = T B: column c of X from column c of B and rows of T^T.
#pragma unroll
    for (int i = 0; i < TE; ++i) y[i] = 0.f;
#pragma unroll 2
    for (int k = 0; k < n; ++k) {
      const float bk = Bs[k * SB + c];
      const float4* tr = reinterpret_cast<const float4*>(TsT + k * SA);
#pragma unroll
      for (int q = 0; q < TE / 4; ++q) {
        const float4 tv = tr[q];
        y[4 * q] = fmaf(tv.x, bk, y[4 * q]);
        y[4 * q + 1] = fmaf(tv.y, bk, y[4 * q + 1]);
        y[4 * q + 2] = fmaf(tv.z, bk, y[4 * q + 2]);
        y[4 * q + 3] = fmaf(tv.w, bk, y[4 * q + 3]);
      }
    }
    float lm = -INFINITY;
    if (c < n)
#pragma unroll
      for (int i = 0; i < TE; ++i)
        if (i < n) lm = fmaxf(lm, y[i]);
    const double m = team_max<TE>((double)lm, red, wt, bar_id);
    if (!(m > 0.0)) {
      info.status = PAIR_DEGENERATE;
      break;
    }
    // Step 6: SDSN (Alg. 2).  k = 0 is step 1, then the sweeps of eq. 7.
    const float scale = (float)((a.theta / 2.0) / m);
    int k = 0;
    float cS1 = 0.f, bc = 0.f;
    while (true) {
      if (k == 0) {
#pragma unroll
        for (int i = 0; i < TE; ++i) y[i] *= scale;
      } else {
        // a_i = 1/n + S/n^2 - r_i/n, formed once per row by the lane that
        // owns the row (-inf on padding rows, which stay 0).
#pragma unroll
        for (int q = 0; q < TE / 4; ++q) {
          const float4 a4 = reinterpret_cast<const float4*>(arow)[q];
          const float aa[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
          for (int h = 0; h < 4; ++h) y[4 * q + h] = fmaxf((y[4 * q + h] + aa[h]) - bc, 0.f);
        }
      }
      ++k;
      // Sums of the new Y: column (in the lane, four interleaved partial
      // sums in a fixed order: a chain of TE / 4 additions, not TE), rows
      // (transposed tree).
      float c4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < TE; ++i) c4[i & 3] += y[i];
      const float cs = (c4[0] + c4[1]) + (c4[2] + c4[3]);
      // After the trees lane l holds the warp's sum of row l (and, TE = 64,
      // of row 32 + l): every row by exactly one lane.
      const float v0 = team_rows32<0>(y, lane);
      const float v1 = TE == 64 ? team_rows32<TE == 64 ? 32 : 0>(y, lane) : 0.f;
      team_sync<TE>(bar_id);  // every lane has read the previous a_i and row sums
      part[wt * TE + lane] = v0;
      if (TE == 64) part[wt * TE + 32 + lane] = v1;
      team_sync<TE>(bar_id);
      // S over all rows as a double-float, the same in every lane of the team.
      float shi, slo = 0.f;
      if (TE == 32) {
        shi = v0;
      } else {
        two_sum_f(part[lane] + part[TE + lane], part[32 + lane] + part[TE + 32 + lane], shi, slo);
      }
      warp_sum_df(shi, slo);
      Shi = shi;
      Slo = slo;
      bc = c < n ? cs * inv_n_f : INFINITY;  // padding column: stays 0
      cS1 = inv_n_f + (shi * inv_n2_f + slo * inv_n2_f);
      {
        // Row 32 wt + lane of the tile (row `lane` for one warp): its sum
        // over both warps' columns, then its a_i for the next sweep.
        const int row = (TE == 64 ? 32 * wt : 0) + lane;
        const float rsum = TE == 64 ? part[row] + part[TE + row] : v0;
        arow[row] = row < n ? cS1 - rsum * inv_n_f : -INFINITY;
      }
      team_sync<TE>(bar_id);  // every a_i is written
      const bool below = shi < thr_hi || (shi == thr_hi && slo <= thr_lo);
      if (k > 1 && below) break;  // gamma of the last clamped result (reading (iii))
      if (k > a.max_sweeps) break;
    }
    const int sweeps = k - 1;
    if (sweeps > 0) g = ((double)Shi + (double)Slo) * inv_n - 1.0;
    sweeps_total += sweeps;
    // Steps 7-8 (FP32 N as in the CTA form; delta's block sums in FP64).
    float d2f = 0.f, nn2f = 0.f;
    if (c < n) {
#pragma unroll
      for (int i = 0; i < TE; ++i) {
        if (i < n) {
          const float old = ncol[i];
          const float nn = fmaf(bl, old, al * y[i]);
          const float dd = nn - old;
          ncol[i] = nn;
          d2f = fmaf(dd, dd, d2f);
          nn2f = fmaf(nn, nn, nn2f);
        }
      }
    }
    const double d2 = team_sum_f<TE>(d2f, red, wt, bar_id);
    const double nn2 = team_sum_f<TE>(nn2f, red, wt, bar_id);
    ++t;
    const double dl = sqrt(d2) / sqrt(nn2);
    bool stop = dl <= a.delta_tol || (a.use_stall && dl <= a.mixed_delta_tol);
    if (a.use_stall && a.stall_ratio > 0.0 && dl <= a.stall_below && dl > a.stall_ratio * prev_delta)
      stop = true;
    prev_delta = dl;
    delta = dl;
    if (stop) break;
  }
  if (info.status != PAIR_OK) {
    if (c == 0) a.info[pi] = info;
    team_sync<TE>(bar_id);
    return;
  }
  // Step 10 (eq. 2): N into shared memory (over A^T, no longer needed), then
  // the Hungarian of the CTA form on one warp.
  team_sync<TE>(bar_id);
#pragma unroll
  for (int i = 0; i < TE; ++i) AsT[i * SA + c] = ncol[i];
  team_sync<TE>(bar_id);
  if (wt == 0 || TE == 32) small_lap(AsT, SA, n, u, rowcol, argc, rowmax, &misc[0]);
  team_sync<TE>(bar_id);
  // Objective (eq. 1) and matching error (Sec. 7) on the unscaled inputs.
  double s1 = 0.0, s2 = 0.0;
  for (int e = c; e < n * n; e += TE) {
    const int i = e / n, j = e - i * n;
    const double x = Ag[e];
    const double yv = Bg[rowcol[i] * n + rowcol[j]];
    s1 = fma(x, yv, s1);
    s2 = fma(x - yv, x - yv, s2);
  }
  const double av = c < n ? (double)AsT[c * SA + rowcol[c]] : 0.0;
  s1 = team_sum<TE>(s1, red, wt, bar_id);
  s2 = team_sum<TE>(s2, red, wt, bar_id);
  const double avs = team_sum<TE>(av, red, wt, bar_id);
  if (c < n) a.perm[d.off_vec + c] = rowcol[c];
  if (a.Nout != nullptr && c < n) {
    double* no = a.Nout + d.off_mat;
#pragma unroll
    for (int i = 0; i < TE; ++i)
      if (i < n) no[i * n + c] = (double)ncol[i];
  }
  if (c == 0) {
    info.outer_iters = t;
    info.total_sweeps = sweeps_total;
    info.delta = delta;
    info.gamma = g;
    info.objective = 0.5 * s1;
    info.match_error = 0.5 * sqrt(s2);
    info.assignment_value = avs;
    info.lap_aug = misc[0];
    a.info[pi] = info;
  }
  team_sync<TE>(bar_id);
}

__global__ void __launch_bounds__(kTeamCT, 2) batched_team_kernel(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_pi[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int team = warp >> 1, wt = warp & 1;
  unsigned char* region = smem + team * kTeamBytes;
  const int bar_id = 1 + team;  // named barrier of the team's 64 threads
  while (true) {
    if (wt == 0 && lane == 0) s_pi[team] = (int)atomicAdd(a.queue, 1u);
    team_sync<64>(bar_id);
    const int pi = s_pi[team];
    team_sync<64>(bar_id);
    if (pi >= a.count) break;
    if (a.desc[pi].n > a.team_split) {
      team_solve<64>(a, pi, region, wt, bar_id);
    } else {
      // Pairs are queued longest first: every later pair also has n <=
      // team_split <= 32, so the second warp takes its own.
      int pj = pi;
      if (wt == 1) {
        if (lane == 0) pj = (int)atomicAdd(a.queue, 1u);
        pj = __shfl_sync(0xffffffffu, pj, 0);
      }
      if (pj < a.count) team_solve<32>(a, pj, region + wt * TeamLayout<32>::bytes, 0, bar_id);
    }
  }
}

// Gather caller matrices (device pointers, table by processing position)
// into the packed input buffers.
__global__ void gather_kernel(const double* const* srcA, const double* const* srcB,
                              const BatchDesc* desc, int count, double* A, double* B) {
  for (int p = blockIdx.x; p < count; p += gridDim.x) {
    const BatchDesc d = desc[p];
    const double* sa = srcA[p];
    const double* sb = srcB[p];
    for (int e = threadIdx.x; e < d.n * d.n; e += blockDim.x) {
      A[d.off_mat + e] = sa[e];
      B[d.off_mat + e] = sb[e];
    }
  }
}

// Scatter packed outputs to caller device buffers.
__global__ void scatter_kernel(const BatchDesc* desc, int count, const double* Nout,
                               const int32_t* perm, double* const* dstX, int32_t* const* dstP) {
  for (int p = blockIdx.x; p < count; p += gridDim.x) {
    const BatchDesc d = desc[p];
    if (dstX != nullptr && dstX[p] != nullptr)
      for (int e = threadIdx.x; e < d.n * d.n; e += blockDim.x) dstX[p][e] = Nout[d.off_mat + e];
    for (int i = threadIdx.x; i < d.n; i += blockDim.x) dstP[p][i] = perm[d.off_vec + i];
  }
}

// Device state of the batched path, grown on demand.
struct BatchedState {
  size_t cap_mat = 0, cap_vec = 0, cap_count = 0;
  double *A = nullptr, *B = nullptr, *N = nullptr;
  int32_t* perm = nullptr;
  BatchDesc* desc = nullptr;
  BatchDesc* tdesc = nullptr;   // autotuner: strided sample of the queue
  size_t cap_tdesc = 0;
  BatchInfo* info = nullptr;
  void** ptrs = nullptr;        // device tables by position: A, B, X, perm (4 x count)
  unsigned* queue = nullptr;
  size_t hcap_mat = 0, hcap_vec = 0, hcap_count = 0;
  double *hA = nullptr, *hB = nullptr, *hN = nullptr;
  int32_t* hperm = nullptr;
  BatchDesc* hdesc = nullptr;
  BatchInfo* hinfo = nullptr;
  void** hptrs = nullptr;
  int tuned_nt[2] = {0, 0};     // autotuned kernel variant per precision (0 = not tuned)
  int forced = 0;               // fram_set_batched_kernel: 0 = autotune
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  // signature of the captured graph
  int g_nt = 0, g_scatter = -1;
  void* g_ptrs = nullptr;
  BatchArgs g_args{};
};

template <typename T>
void set_attrs() {
  static DeviceCache done;
  device_cached(done, [] {
    cudaFuncSetAttribute(batched_kernel<T, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)batched_smem_bytes<T>(128));
    cudaFuncSetAttribute(batched_kernel<T, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)batched_smem_bytes<T>(256));
    cudaFuncSetAttribute(batched_kernel<T, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)batched_smem_bytes<T>(512));
    return 1;
  });
}

// Resident CTAs per SM for a block size (queried once).
template <typename T>
int batched_occupancy(int nt) {
  static DeviceCache occ[3];
  const int k = nt == 128 ? 0 : (nt == 256 ? 1 : 2);
  return device_cached(occ[k], [nt] {
    int v = 0;
    cudaError_t e =
        nt == 128 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, batched_kernel<T, 128>, 128,
                                                                  batched_smem_bytes<T>(128))
        : nt == 256 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, batched_kernel<T, 256>, 256,
                                                                    batched_smem_bytes<T>(256))
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, batched_kernel<T, 512>, 512,
                                                                    batched_smem_bytes<T>(512));
    return (e == cudaSuccess && v > 0) ? v : 1;
  });
}

template <typename T>
int launch_batched(const BatchArgs& a, int nt, int num_sms, cudaStream_t s) {
  set_attrs<T>();
  const int slots = batched_occupancy<T>(nt) * num_sms;
  int grid = slots < a.count ? slots : a.count;
  if (grid < 1) grid = 1;
  switch (nt) {
    case 128:
      batched_kernel<T, 128><<<grid, 128, batched_smem_bytes<T>(128), s>>>(a);
      break;
    case 256:
      batched_kernel<T, 256><<<grid, 256, batched_smem_bytes<T>(256), s>>>(a);
      break;
    default:
      batched_kernel<T, 512><<<grid, 512, batched_smem_bytes<T>(512), s>>>(a);
      break;
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// Team kernel (FP32): two teams of two warps per CTA, persistent.
int launch_batched_team(const BatchArgs& a, int num_sms, cudaStream_t s) {
  static DeviceCache occ;
  const int per_sm = device_cached(occ, [] {
    if (cudaFuncSetAttribute(batched_team_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * kTeamBytes)) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, batched_team_kernel, kTeamCT,
                                                      2 * kTeamBytes) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    return v > 0 ? v : -1;
  });
  if (per_sm < 1) return -1;
  // Persistent: every CTA resident at once, none beyond two pairs per CTA.
  int grid = per_sm * num_sms;
  if (grid > (a.count + 1) / 2) grid = (a.count + 1) / 2;
  if (grid < 1) grid = 1;
  batched_team_kernel<<<grid, kTeamCT, 2 * kTeamBytes, s>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// Kernel variants of the batched path.  CTA form: one pair per CTA of 128,
// 256 or 512 threads (FP64 and FP32).  Team form (FP32 only): tile edge 32
// on one warp for n <= 32 and 64 on two warps above, or 64 for every pair.
enum BatchVariant : int { BV_CTA128 = 1, BV_CTA256, BV_CTA512, BV_TEAM_SPLIT, BV_TEAM64 };

int launch_batched_variant(bool fp32, BatchArgs a, int v, int num_sms, cudaStream_t s) {
  switch (v) {
    case BV_TEAM_SPLIT:
      a.team_split = 32;
      return fp32 ? launch_batched_team(a, num_sms, s) : -1;
    case BV_TEAM64:
      a.team_split = 0;
      return fp32 ? launch_batched_team(a, num_sms, s) : -1;
    default: {
      const int nt = v == BV_CTA128 ? 128 : v == BV_CTA256 ? 256 : 512;
      return fp32 ? launch_batched<float>(a, nt, num_sms, s)
                  : launch_batched<double>(a, nt, num_sms, s);
    }
  }
}

// Grow a device (pinned host when host == true) buffer to `need` elements.
template <typename P>
bool grow(P** ptr, size_t& cap, size_t need, bool host = false) {
  if (need <= cap && *ptr) return true;
  if (*ptr) host ? cudaFreeHost(*ptr) : cudaFree(*ptr);
  *ptr = nullptr;
  cap = 0;
  const size_t bytes = (need ? need : 1) * sizeof(P);
  cudaError_t e = host ? cudaMallocHost(reinterpret_cast<void**>(ptr), bytes)
                       : cudaMalloc(reinterpret_cast<void**>(ptr), bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return false;
  }
  cap = need;
  return true;
}

}  // namespace

void batched_release(fram_ctx* c) {
  BatchedState* b = static_cast<BatchedState*>(c->batched);
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  void* dptr[] = {b->A, b->B, b->N, b->perm, b->desc, b->tdesc, b->info, b->ptrs, b->queue};
  for (void* p : dptr)
    if (p) cudaFree(p);
  void* hptr[] = {b->hA, b->hB, b->hN, b->hperm, b->hdesc, b->hinfo, b->hptrs};
  for (void* p : hptr)
    if (p) cudaFreeHost(p);
  delete b;
  c->batched = nullptr;
}

// Solve the pairs `idx` (all with n <= 64) of one fram_solve_batched call in
// one persistent launch.  Inputs and outputs must each be all-host or
// all-device.
fram_status solve_small_batch(fram_ctx* c, const std::vector<int>& idx, const int* n,
                              const double* const* A, const double* const* B,
                              const fram_params& p, double* const* X_out,
                              int32_t* const* perm_out, fram_info* infos) {
  if (!c->batched) c->batched = new BatchedState();
  BatchedState& S = *static_cast<BatchedState*>(c->batched);
  const int count = (int)idx.size();
  if (count == 0) return FRAM_OK;
  const bool fp32 = p.precision != FRAM_PREC_FP64;
  const bool wantX = X_out != nullptr;
  std::vector<int> order(idx);  // longest pairs first for the work queue
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return n[x] > n[y]; });
  std::vector<BatchDesc> desc(count);
  size_t mat = 0, vec = 0;
  int in_dev = 0, out_dev = 0;
  PtrClassifier pc;  // thousands of pointers, few allocations
  for (int k = 0; k < count; ++k) {
    const int i = order[k];
    desc[k] = BatchDesc{n[i], i, (long long)mat, (long long)vec};
    mat += (size_t)n[i] * n[i];
    vec += (size_t)n[i];
    in_dev += (pc.is_device(A[i]) ? 1 : 0) + (pc.is_device(B[i]) ? 1 : 0);
    const bool xnone = !wantX || X_out[i] == nullptr;
    const bool xdev = !xnone && pc.is_device(X_out[i]);
    const bool xd = xnone || xdev;
    const bool xh = xnone || !xdev;
    const bool pd = pc.is_device(perm_out[i]);
    out_dev += (pd && xd) ? 1 : ((!pd && xh) ? 0 : -count - 1);
  }
  if (in_dev != 0 && in_dev != 2 * count) {
    set_err(c, "fram_solve_batched: inputs must be all host or all device buffers");
    return FRAM_ERR_INVALID;
  }
  if (out_dev != 0 && out_dev != count) {
    set_err(c, "fram_solve_batched: outputs must be all host or all device buffers");
    return FRAM_ERR_INVALID;
  }
  const bool dev_in = in_dev != 0, dev_out = out_dev != 0;
  const size_t need_bytes = 3 * mat * 8 + vec * 4 +
                            (size_t)count * (sizeof(BatchDesc) + sizeof(BatchInfo) + 32);
  if (c->budget && c->ws.bytes + need_bytes + c->serve_bytes > c->budget) {
    set_err(c, "batched buffers (%zu bytes) exceed the HBM budget", need_bytes);
    return FRAM_ERR_OOM;
  }
  bool ok = true;
  size_t cm = S.cap_mat, cv = S.cap_vec, cc = S.cap_count;
  ok = ok && grow(&S.A, cm = S.cap_mat, mat) && grow(&S.B, cm = S.cap_mat, mat) &&
       grow(&S.N, S.cap_mat, mat);
  ok = ok && grow(&S.perm, cv, vec);
  ok = ok && grow(&S.desc, cc = S.cap_count, (size_t)count) &&
       grow(&S.info, cc = S.cap_count, (size_t)count) &&
       grow(&S.ptrs, S.cap_count, (size_t)4 * count);
  ok = ok && (S.queue || cudaMalloc(&S.queue, 256) == cudaSuccess);
  S.cap_vec = cv;
  size_t hm = S.hcap_mat, hc = S.hcap_count;
  ok = ok && grow(&S.hA, hm = S.hcap_mat, mat, true) && grow(&S.hB, hm = S.hcap_mat, mat, true) &&
       grow(&S.hN, S.hcap_mat, mat, true);
  ok = ok && grow(&S.hperm, S.hcap_vec, vec, true);
  ok = ok && grow(&S.hdesc, hc = S.hcap_count, (size_t)count, true) &&
       grow(&S.hinfo, hc = S.hcap_count, (size_t)count, true) &&
       grow(&S.hptrs, S.hcap_count, (size_t)4 * count, true);
  (void)cm;
  (void)cc;
  (void)hm;
  (void)hc;
  if (!ok) {
    batched_release(c);
    set_err(c, "batched buffers: allocation failed");
    return FRAM_ERR_OOM;
  }
  cudaStream_t s = c->stream;
#define BT_CUDA(x, what)                                   \
  do {                                                     \
    cudaError_t _e = (x);                                  \
    if (_e != cudaSuccess) return cuda_fail(c, _e, what);  \
  } while (0)
  memcpy(S.hdesc, desc.data(), count * sizeof(BatchDesc));
  for (int k = 0; k < count; ++k) {
    const int i = desc[k].index;
    S.hptrs[k] = const_cast<double*>(A[i]);
    S.hptrs[count + k] = const_cast<double*>(B[i]);
    S.hptrs[2 * count + k] = wantX ? X_out[i] : nullptr;
    S.hptrs[3 * count + k] = perm_out[i];
  }
  BT_CUDA(cudaMemcpyAsync(S.desc, S.hdesc, count * sizeof(BatchDesc), cudaMemcpyHostToDevice, s),
          "copy descriptors");
  BT_CUDA(cudaMemcpyAsync(S.ptrs, S.hptrs, 4 * count * sizeof(void*), cudaMemcpyHostToDevice, s),
          "copy pointer tables");
  if (dev_in) {
    gather_kernel<<<std::min(count, 2 * c->num_sms), 256, 0, s>>>(
        reinterpret_cast<const double* const*>(S.ptrs),
        reinterpret_cast<const double* const*>(S.ptrs + count), S.desc, count, S.A, S.B);
    if (cudaPeekAtLastError() != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "gather");
    c->launches += 1;
  } else {
    // Pack the host inputs into the pinned staging arena: a memory-bound
    // loop, split over up to 8 threads by byte offset for large batches.
    auto pack = [&](int k0, int k1) {
      for (int k = k0; k < k1; ++k) {
        const BatchDesc& d = desc[k];
        memcpy(S.hA + d.off_mat, A[d.index], (size_t)d.n * d.n * 8);
        memcpy(S.hB + d.off_mat, B[d.index], (size_t)d.n * d.n * 8);
      }
    };
    const unsigned hw = std::thread::hardware_concurrency();
    const int nth = mat * 16 >= (16u << 20) ? (int)std::min(8u, hw > 1 ? hw : 1u) : 1;
    if (nth <= 1) {
      pack(0, count);
    } else {
      std::vector<std::thread> th;
      int k0 = 0;
      for (int t = 1; t <= nth && k0 < count; ++t) {
        const size_t until = mat * (size_t)t / (size_t)nth;  // cumulative element bound
        int k1 = k0;
        while (k1 < count && (t == nth || (size_t)desc[k1].off_mat < until)) ++k1;
        if (k1 > k0) {
          try {
            th.emplace_back(pack, k0, k1);
          } catch (...) {  // no thread to be had: this one packs the rest
            pack(k0, count);
            k0 = count;
            break;
          }
        }
        k0 = k1;
      }
      for (auto& x : th) x.join();
    }
    BT_CUDA(cudaMemcpyAsync(S.A, S.hA, mat * 8, cudaMemcpyHostToDevice, s), "copy inputs");
    BT_CUDA(cudaMemcpyAsync(S.B, S.hB, mat * 8, cudaMemcpyHostToDevice, s), "copy inputs");
  }
  BatchArgs a{};
  a.desc = S.desc;
  a.count = count;
  a.A = S.A;
  a.B = S.B;
  a.Nout = wantX ? S.N : nullptr;
  a.perm = S.perm;
  a.info = S.info;
  a.queue = S.queue;
  a.lam = p.lambda;
  a.alpha = p.alpha;
  a.theta = p.theta;
  a.delta_tol = p.delta_tol;
  a.gamma_tol = fp32 ? std::max(p.polish_tol, p.gamma_tol) : p.gamma_tol;
  a.mixed_delta_tol = p.mixed_delta_tol;
  a.stall_ratio = p.stall_ratio;
  a.stall_below = p.stall_below;
  a.max_outer = p.max_outer;
  a.max_sweeps = p.max_sweeps;
  a.use_stall = fp32 ? 1 : 0;

  // Autotuner: on the first batched call per precision, time each kernel
  // variant (block size of the CTA form; tile edge split of the team form)
  // on a sample of the batch and keep the fastest.  The sample takes every
  // stride-th pair of the queue, so it has the batch's length mix (a prefix
  // would hold only the longest pairs), and up to 32 pairs per SM: with
  // fewer, the last pairs' latency decides and favours the wider teams over
  // the form with the higher throughput.  Each variant runs twice and its
  // faster run counts (once when the sample holds 1024 pairs or more: such a
  // run is long enough to time to about 1%).
  int& nt = S.tuned_nt[fp32 ? 1 : 0];
  if (S.forced >= BV_TEAM_SPLIT && !fp32) {
    set_err(c, "fram_solve_batched: the team kernel runs the mixed precisions only");
    return FRAM_ERR_INVALID;
  }
  if (S.forced != 0) nt = S.forced;
  if (nt == 0) {
    const int m = std::min(count, 32 * c->num_sms);
    const int stride = count / m;
    if (!grow(&S.tdesc, S.cap_tdesc, (size_t)m)) {
      batched_release(c);
      set_err(c, "batched buffers: allocation failed");
      return FRAM_ERR_OOM;
    }
    std::vector<BatchDesc> sample(m);
    for (int j = 0; j < m; ++j) sample[j] = desc[(size_t)j * stride];
    BT_CUDA(cudaMemcpyAsync(S.tdesc, sample.data(), m * sizeof(BatchDesc),
                            cudaMemcpyHostToDevice, s),
            "copy tuning descriptors");
    BT_CUDA(cudaStreamSynchronize(s), "synchronize");  // sample is a stack vector
    float best = 1e30f;
    BatchArgs t = a;
    t.desc = S.tdesc;
    t.count = m;
    std::vector<int> cands = {BV_CTA128, BV_CTA256, BV_CTA512};
    if (fp32) {
      cands.push_back(BV_TEAM_SPLIT);
      cands.push_back(BV_TEAM64);
    }
    for (int cand : cands) {
      for (int rep = 0; rep < (m >= 1024 ? 1 : 2); ++rep) {
        BT_CUDA(cudaMemsetAsync(S.queue, 0, 4, s), "memset");
        BT_CUDA(cudaEventRecord(c->ev0, s), "event");
        if (launch_batched_variant(fp32, t, cand, c->num_sms, s) < 0)
          return cuda_fail(c, cudaGetLastError(), "batched kernel");
        BT_CUDA(cudaEventRecord(c->ev1, s), "event");
        BT_CUDA(cudaEventSynchronize(c->ev1), "synchronize");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        c->launches += 1;
        if (ms < best) {
          best = ms;
          nt = cand;
        }
      }
    }
  }
  // Queue reset + persistent kernel (+ scatter to device outputs), captured
  // into a CUDA graph once per configuration and replayed; the data of each
  // call lives in device buffers the graph reads.
  const bool scatter = dev_out;
  const bool same = S.graph && S.g_nt == nt && S.g_scatter == (int)scatter &&
                    S.g_ptrs == (void*)S.ptrs && memcmp(&S.g_args, &a, sizeof a) == 0;
  if (!same) {
    if (S.graph) cudaGraphExecDestroy(S.graph);
    S.graph = nullptr;
    if (!S.cap_stream &&
        cudaStreamCreateWithFlags(&S.cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return cuda_fail(c, cudaGetLastError(), "capture stream");
    cudaGraph_t g = nullptr;
    BT_CUDA(cudaStreamBeginCapture(S.cap_stream, cudaStreamCaptureModeThreadLocal),
            "begin capture");
    cudaMemsetAsync(S.queue, 0, 4, S.cap_stream);
    launch_batched_variant(fp32, a, nt, c->num_sms, S.cap_stream);
    if (scatter)
      scatter_kernel<<<std::min(count, 2 * c->num_sms), 256, 0, S.cap_stream>>>(
          S.desc, count, S.N, S.perm,
          wantX ? reinterpret_cast<double* const*>(S.ptrs + 2 * count) : nullptr,
          reinterpret_cast<int32_t* const*>(S.ptrs + 3 * count));
    cudaError_t ce = cudaStreamEndCapture(S.cap_stream, &g);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "end capture");
    ce = cudaGraphInstantiate(&S.graph, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
      S.graph = nullptr;
      return cuda_fail(c, ce, "graph instantiate");
    }
    S.g_nt = nt;
    S.g_scatter = scatter;
    S.g_ptrs = S.ptrs;
    S.g_args = a;
  }
  BT_CUDA(cudaGraphLaunch(S.graph, s), "graph launch");
  c->launches += scatter ? 2 : 1;
  if (!scatter) {
    if (wantX) BT_CUDA(cudaMemcpyAsync(S.hN, S.N, mat * 8, cudaMemcpyDeviceToHost, s), "copy N");
    BT_CUDA(cudaMemcpyAsync(S.hperm, S.perm, vec * 4, cudaMemcpyDeviceToHost, s), "copy perm");
  }
  BT_CUDA(cudaMemcpyAsync(S.hinfo, S.info, count * sizeof(BatchInfo), cudaMemcpyDeviceToHost, s),
          "copy info");
  BT_CUDA(cudaStreamSynchronize(s), "synchronize");
  fram_status worst = FRAM_OK;
  for (int k = 0; k < count; ++k) {
    const BatchDesc& d = desc[k];
    const BatchInfo& bi = S.hinfo[k];
    if (!scatter) {
      memcpy(perm_out[d.index], S.hperm + d.off_vec, (size_t)d.n * 4);
      if (wantX && X_out[d.index])
        memcpy(X_out[d.index], S.hN + d.off_mat, (size_t)d.n * d.n * 8);
    }
    if (infos) {
      fram_info& f = infos[d.index];
      memset(&f, 0, sizeof f);
      f.outer_iters = bi.outer_iters;
      f.total_sweeps = bi.total_sweeps;
      f.lap_augmentations = bi.lap_aug;
      f.lap_auction_phases = -1;
      f.delta = bi.delta;
      f.gamma = bi.gamma;
      f.sdsn_converged_last = bi.gamma <= a.gamma_tol ? 1 : 0;
      f.objective = bi.objective;
      f.match_error = bi.match_error;
      f.assignment_value = bi.assignment_value;
    }
    if (bi.status == PAIR_INVALID && worst == FRAM_OK) {
      set_err(c, "fram_solve_batched: pair %d is outside the graph model", d.index);
      worst = FRAM_ERR_INVALID;
    } else if (bi.status == PAIR_DEGENERATE && worst == FRAM_OK) {
      set_err(c, "fram_solve_batched: pair %d is degenerate (max(X) <= 0)", d.index);
      worst = FRAM_ERR_DEGENERATE;
    }
  }
  return worst;
}

}  // namespace fram

extern "C" fram_status fram_set_batched_kernel(fram_ctx* c, int variant) {
  using namespace fram;
  if (!c) return FRAM_ERR_INVALID;
  if (variant < 0 || variant > BV_TEAM64) {
    set_err(c, "fram_set_batched_kernel: variant must be 0 (autotune) .. %d", (int)BV_TEAM64);
    return FRAM_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  if (!c->batched) c->batched = new BatchedState();
  BatchedState& S = *static_cast<BatchedState*>(c->batched);
  S.forced = variant;
  S.tuned_nt[0] = S.tuned_nt[1] = 0;  // re-tune (or take the forced one) on the next call
  return FRAM_OK;
}

extern "C" int fram_batched_kernel(const fram_ctx* c, int precision) {
  using namespace fram;
  if (!c || !c->batched) return 0;
  const BatchedState& S = *static_cast<const BatchedState*>(c->batched);
  return S.tuned_nt[precision != FRAM_PREC_FP64 ? 1 : 0];
}

extern "C" fram_status fram_solve_batched(fram_ctx* c, int count, const int* n,
                                          const double* const* A, const double* const* B,
                                          const fram_params* params, double* const* X_out,
                                          int32_t* const* perm_out, fram_info* infos) {
  using namespace fram;
  if (!c) return FRAM_ERR_INVALID;
  c->last_error.clear();
  if (count < 0 || (count > 0 && (!n || !A || !B || !perm_out))) {
    set_err(c, "fram_solve_batched: count >= 0 and non-NULL n, A, B, perm_out are required");
    return FRAM_ERR_INVALID;
  }
  fram_params p;
  if (params)
    p = *params;
  else
    fram_default_params(&p);
  {
    fram_status st = check_params(c, p);
    if (st != FRAM_OK) return st;
    if (p.projection != FRAM_PROJ_SDSN) {
      set_err(c, "fram_solve_batched: the exact projection is available through fram_solve only");
      return FRAM_ERR_INVALID;
    }
  }
  for (int i = 0; i < count; ++i)
    if (n[i] < 1 || !A[i] || !B[i] || !perm_out[i]) {
      set_err(c, "fram_solve_batched: pair %d needs n >= 1 and non-NULL A, B, perm_out", i);
      return FRAM_ERR_INVALID;
    }
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "set device");
  std::lock_guard<std::mutex> lk(c->mu);
  std::vector<int> small;
  for (int i = 0; i < count; ++i)
    if (n[i] <= NMAX) small.push_back(i);
  fram_status st = solve_small_batch(c, small, n, A, B, p, X_out, perm_out, infos);
  if (st != FRAM_OK) return st;
  for (int i = 0; i < count; ++i)
    if (n[i] > NMAX) {
      st = solve_one(c, n[i], A[i], B[i], nullptr, p, X_out ? X_out[i] : nullptr, perm_out[i],
                     infos ? &infos[i] : nullptr);
      if (st != FRAM_OK) return st;
    }
  return FRAM_OK;
}
