// Discretisation (eq. 2 / Alg. 1 step 10 of arXiv 2508.00887):
//   perm = argmax_{P in Pi_n} <P, W>   (= argmin ||P - W||_F over permutations)
//
//  1. Row argmax, one warp per row (ties -> lowest column).  If the row
//     argmaxes already form a permutation it is optimal: the sum of row
//     maxima bounds every assignment from above.  This is the common case
//     once FRAM has converged, because N is then close to a permutation.
//     Column potentials v_j = min_i (rowmax_i - W_ij) keep every argmax
//     pair tight and start the completion from tighter duals.
//  2. Exact completion from that start (step 4) with a budget of 64 n
//     Dijkstra steps.  Almost every FRAM output finishes here.
//  3. A W whose rows all prefer the same few columns and differ by little
//     else can need far more steps from the argmax start.  Past the budget, a forward auction with
//     epsilon-scaling (Bertsekas 1988) computes near-optimal column prices p
//     in one cooperative launch and the completion restarts from them.  It runs in the
//     asynchronous Gauss-Seidel form: each CTA bids for its own rows with one
//     64-bit atomicMax on a (quantised price, row) key, and a row it outbids
//     is its to place next, so a chain of displacements costs one bid each
//     and no CTA waits on another inside a phase.  Prices only rise, so a bid
//     computed from stale prices is a lower bid and epsilon-complementary
//     slackness still holds for the winner.
//  4. Exact completion.  With column potentials v (those of step 1, or -p
//     after step 3) a pair is kept only if its column minimises c_ij - v_j
//     for the cost c = -W; one CTA (a cluster of 8 from n = 1024) then
//     places the other rows by shortest augmenting paths (the Hungarian
//     method of Kuhn 1955 in the Jonker-Volgenant form).  The auction only shortens these paths; the result is exact
//     either way.
#include <cooperative_groups.h>
#include <math.h>

#include "fram_internal.cuh"

namespace cg = cooperative_groups;

namespace fram {

namespace {

constexpr int kLapThreads = 1024;
constexpr int kOwnerBits = 20;
constexpr unsigned long long kNoOwner = (1ull << kOwnerBits) - 1;  // n < 2^20 - 1
constexpr int kQuantBits = 36;   // price quantum = (max W - min W) * 2^-36
constexpr int kPriceBits = 44;   // quantised prices < 2^44 (256x the value range)
constexpr int kPhases = 12;      // epsilon = range * 4^-phase, phase = 1..12

// Concurrent completion (lap_solve_conc_kernel), one per pass.
struct ConcCtl {
  int lock;          // 0 free, 1 held by a committing cluster
  unsigned seq;      // commits published so far (release store)
  int next_row;      // work queue over the rows
  int commits;       // augmenting paths applied
  int aborts;        // searches repeated after a conflicting commit
  int err;           // 1: a search did not terminate or a wait expired
  long long steps;   // Dijkstra steps of every search, repeated ones included
  long long applied_steps;  // steps of the applied searches (the step budget)
};

struct LapCtl {
  GridBarrier bar;
  unsigned long long wmax_key;  // ordered keys of max / min over W
  unsigned long long wmin_key;
  double dq;                    // price quantum
  int nfree;                    // rows whose argmax column is taken by a lower row
  int phases;                   // auction phases completed
  int status;                   // DEV_TIMEOUT if an auction wait expired
  int need_auction;             // the first completion ran out of its step budget
  ConcCtl cc[2];                // concurrent completion, by pass
};

struct LapWs {
  int* argc;       // [n] row argmax column
  int* owner;      // [n] lowest row claiming column j as argmax (INT_MAX if none)
  int* colrow;     // [n] row matched to column j, -1 if free
  int* rowcol;     // [n] column matched to row i, -1 if free
  int* way;        // [n] completion: row that reached column j
  int* cand;       // [n] candidate column of row i from step 1 or 2, -1 if none
  unsigned* cseq;  // [n] concurrent completion: last commit that changed column j
  double* rowmax;  // [n]
  double* u;       // [n] row potentials of the kept pairs
  double* v;       // [n] column potentials
  unsigned long long* key;   // [n] auction: (quantised price << 20) | owner row;
                             //     completion label keys when they do not fit on chip
  unsigned long long* tkey;  // [n] completion test keys when they do not fit on chip
  double* wmat;              // [n] W[colrow[j]][j] when it does not fit on chip
  LapCtl* ctl;
};

__host__ __device__ inline size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

__host__ __device__ inline LapWs carve(void* base, int n) {
  LapWs w;
  char* p = static_cast<char*>(base);
  const size_t ib = al256((size_t)n * sizeof(int)), db = al256((size_t)n * sizeof(double));
  int** ia[] = {&w.argc, &w.owner, &w.colrow, &w.rowcol, &w.way, &w.cand,
                reinterpret_cast<int**>(&w.cseq)};
  for (int** q : ia) {
    *q = reinterpret_cast<int*>(p);
    p += ib;
  }
  double** da[] = {&w.rowmax, &w.u, &w.v};
  for (double** q : da) {
    *q = reinterpret_cast<double*>(p);
    p += db;
  }
  w.key = reinterpret_cast<unsigned long long*>(p);
  p += db;
  w.tkey = reinterpret_cast<unsigned long long*>(p);
  p += db;
  w.wmat = reinterpret_cast<double*>(p);
  p += db;
  w.ctl = reinterpret_cast<LapCtl*>(p);
  return w;
}

__global__ void lap_init_kernel(LapWs w, int n) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    w.owner[j] = 0x7fffffff;
    w.cand[j] = -1;
    w.key[j] = kNoOwner;
    w.tkey[j] = ~0ull;  // column potential key (lap_colpot_kernel)
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    LapCtl c{};
    c.wmax_key = 0ull;
    c.wmin_key = ~0ull;
    *w.ctl = c;
  }
}

// Row max and argmax (ties -> lowest column), the lowest row claiming each
// argmax column, and the range of W.
__global__ void lap_rowmax_kernel(const double* __restrict__ W, int ldw, int n, LapWs w) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const double* row = W + (size_t)i * ldw;
    double best = -INFINITY, lo = INFINITY;
    int bj = 0x7fffffff;
#pragma unroll 8
    for (int j = lane; j < n; j += 32) {  // unrolled: the loads issue together
      const double x = row[j];
      if (x > best) {
        best = x;
        bj = j;
      }
      lo = fmin(lo, x);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      if (ob > best || (ob == best && oj < bj)) {
        best = ob;
        bj = oj;
      }
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    }
    if (lane == 0) {
      if (bj == 0x7fffffff) bj = 0;
      w.argc[i] = bj;
      w.rowmax[i] = best;
      atomicMin(&w.owner[bj], i);
      atomicMax(&w.ctl->wmax_key, ordered_key(best));
      atomicMin(&w.ctl->wmin_key, ordered_key(lo));
    }
  }
}

// Number of rows that lose their argmax column to a lower row; price quantum.
// Column potentials for the argmax start: v_j = min_i (rowmax_i - W_ij) >= 0.
// Every argmax pair stays tight (its column gets v = 0, and W_ik + v_k <=
// rowmax_i for every k), so these are feasible duals for the kept pairs,
// and a column no row prefers starts closer to being reached.  On FRAM's N
// this roughly halves the Dijkstra steps of the completion (on the diffuse
// matrices of near-uniform rows, by ~2.6x).  Row block blockIdx.y of every
// column, combined with atomicMin on order-preserving keys (exact, so the
// result does not depend on the order).
__global__ void lap_colpot_kernel(const double* __restrict__ W, int ldw, int n, LapWs w,
                                  int rows_per) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int i0 = blockIdx.y * rows_per, i1 = min(n, i0 + rows_per);
  if (i0 >= i1) return;
  double m = INFINITY;
#pragma unroll 8
  for (int i = i0; i < i1; ++i) m = fmin(m, w.rowmax[i] - W[(size_t)i * ldw + j]);
  atomicMin(&w.tkey[j], ordered_key(m));
}

__global__ void lap_conflicts_kernel(LapWs w, int n) {
  int cnt = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    cnt += w.owner[w.argc[i]] != i;
  cnt = warp_sum(cnt);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&w.ctl->nfree, cnt);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double range = from_ordered_key(w.ctl->wmax_key) - from_ordered_key(w.ctl->wmin_key);
    w.ctl->dq = (range > 0.0 && range < INFINITY) ? ldexp(range, -kQuantBits) : 0.0;
  }
}

// The auction runs when the first completion ran out of budget and W has a
// finite, nonzero range.
__device__ __forceinline__ bool auction_on(const LapCtl* c) {
  return ld_volatile_s32(&c->need_auction) && c->dq > 0.0;
}

// Top two values of W_ij - p_j with the argmax (ties -> lowest column) and
// the key read for it.
struct Top2 {
  double v1, v2;
  int j1;
  unsigned long long k1;
};

__device__ __forceinline__ void top2_merge(Top2& a, double ov1, int oj1, unsigned long long ok1,
                                           double ov2) {
  if (ov1 > a.v1 || (ov1 == a.v1 && oj1 < a.j1)) {
    a.v2 = fmax(a.v1, ov2);
    a.v1 = ov1;
    a.j1 = oj1;
    a.k1 = ok1;
  } else {
    a.v2 = fmax(a.v2, ov1);
  }
}

__device__ __forceinline__ void top2_warp(Top2& t) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double a = __shfl_xor_sync(0xffffffffu, t.v1, o);
    const int b = __shfl_xor_sync(0xffffffffu, t.j1, o);
    const unsigned long long c = __shfl_xor_sync(0xffffffffu, t.k1, o);
    const double d = __shfl_xor_sync(0xffffffffu, t.v2, o);
    top2_merge(t, a, b, c, d);
  }
}

constexpr int kAucMaxThreads = 1024;
constexpr int kAucUnroll = 8;  // independent loads in flight per thread

// One auction bid of row i, block-uniform result: 1 if it won a column (the
// row it displaced, or -1, in *displaced), 0 if it lost the race for it
// (retry), 2 if the auction must stop (no finite value, price range
// exhausted, time limit passed, or another CTA stopped it).
__device__ int auction_bid(const double* __restrict__ row, int i, int n, LapWs& w, double dq,
                           long long eps_q, uint64_t t0, uint64_t limit_ns, int* displaced) {
  __shared__ Top2 s_t[kAucMaxThreads / 32];
  __shared__ int s_res, s_disp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
  Top2 t{-INFINITY, -INFINITY, 0x7fffffff, 0ull};
  for (int base = tid; base < n; base += kAucUnroll * nt) {
    unsigned long long kv[kAucUnroll];
    double wv[kAucUnroll];
#pragma unroll
    for (int u = 0; u < kAucUnroll; ++u) {
      const int j = base + u * nt;
      if (j < n) {
        kv[u] = __ldcg(w.key + j);
        wv[u] = row[j];
      }
    }
#pragma unroll
    for (int u = 0; u < kAucUnroll; ++u) {
      const int j = base + u * nt;
      if (j < n) top2_merge(t, wv[u] - (double)(kv[u] >> kOwnerBits) * dq, j, kv[u], -INFINITY);
    }
  }
  top2_warp(t);
  if (lane == 0) s_t[warp] = t;
  __syncthreads();
  if (tid == 0) {
    for (int q = 1; q < nt >> 5; ++q) top2_merge(t, s_t[q].v1, s_t[q].j1, s_t[q].k1, s_t[q].v2);
    // Bid: the row's value for j1 drops to (second best - eps).
    double d = (t.v1 - t.v2) / dq;  // >= 0; +inf when n == 1
    if (!(d < 0x1p43)) d = 0x1p43;
    const long long qn = (long long)(t.k1 >> kOwnerBits) + (long long)ceil(d) + eps_q;
    int res = 0, disp = -1;
    if (t.j1 >= n || !(t.v1 > -INFINITY) || qn >= (1ll << kPriceBits) ||
        ld_volatile_s32(&w.ctl->bar.abort)) {
      res = 2;  // no finite value, price range exhausted, or stopped elsewhere
    } else {
      const unsigned long long nk = ((unsigned long long)qn << kOwnerBits) | (unsigned)i;
      const unsigned long long old = atomicMax(w.key + t.j1, nk);
      if (old < nk) {
        res = 1;
        const unsigned long long prev = old & kNoOwner;
        disp = prev == kNoOwner ? -1 : (int)prev;
      }
    }
    if (res == 0 && globaltimer_ns() - t0 > limit_ns) res = 2;
    if (res == 2) atomicExch(&w.ctl->bar.abort, 1);
    s_res = res;
    s_disp = disp;
  }
  __syncthreads();
  const int r = s_res;
  *displaced = s_disp;
  __syncthreads();
  return r;
}

// All epsilon-scaling phases in one cooperative launch.  A phase ends when
// every CTA has placed its rows and every row they displaced; then every row
// owns one column.  Stops early (leaving the rest to the exact completion)
// on a wait, time or price limit.
__global__ void __launch_bounds__(kAucMaxThreads) lap_auction_kernel(
    const double* __restrict__ W, int ldw, int n, LapWs w, uint64_t limit_ns) {
  if (!auction_on(w.ctl)) return;  // grid-uniform: set by earlier kernels
  __shared__ int s_flag;
  const int tid = threadIdx.x;
  const double dq = w.ctl->dq;
  unsigned gen = 0;
  const uint64_t t0 = globaltimer_ns();
  for (int phase = 1; phase <= kPhases; ++phase) {
    const long long eps_q = 1ll << (kQuantBits - 2 * phase);
    // Keep the prices, release every column.
    for (int j = blockIdx.x * blockDim.x + tid; j < n; j += gridDim.x * blockDim.x)
      w.key[j] = phase == 1 ? kNoOwner : (__ldcg(w.key + j) | kNoOwner);  // L2: atomics
    if (!grid_sync(&w.ctl->bar, gridDim.x, gen, limit_ns, &w.ctl->status, &s_flag)) return;
    for (int i0 = blockIdx.x; i0 < n; i0 += gridDim.x) {
      int i = i0;
      while (i >= 0) {
        int disp;
        const int r = auction_bid(W + (size_t)i * ldw, i, n, w, dq, eps_q, t0, limit_ns, &disp);
        if (r == 2) return;  // abort raised: CTAs at a barrier leave too
        if (r == 1) i = disp;
      }
    }
    if (!grid_sync(&w.ctl->bar, gridDim.x, gen, limit_ns, &w.ctl->status, &s_flag)) return;
    if (blockIdx.x == 0 && tid == 0) w.ctl->phases = phase;
  }
}

// Candidate pairs and column potentials.  Pass 0: the conflict-free argmaxes
// with v = 0.  Pass 1 (only after the budget ran out): the auction's pairs
// and v = -p if it ran, else the argmaxes again.
__global__ void lap_candidates_kernel(LapWs w, int n, int pass) {
  if (pass == 1 && !ld_volatile_s32(&w.ctl->need_auction)) return;
  const bool auction = pass == 1 && auction_on(w.ctl);
  const double dq = w.ctl->dq;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    w.colrow[j] = -1;
    w.cseq[j] = 0u;
    if (auction) {
      const unsigned long long k = w.key[j];
      w.v[j] = -(double)(k >> kOwnerBits) * dq;
      const unsigned long long r = k & kNoOwner;
      if (r != kNoOwner) w.cand[r] = j;
    } else {
      const unsigned long long k = w.tkey[j];
      w.v[j] = k != ~0ull ? from_ordered_key(k) : 0.0;
      const int r = w.owner[j];
      if (r != 0x7fffffff) w.cand[r] = j;
    }
  }
}

// u_i = -max_j (W_ij + v_j); keep the candidate pair of row i if it is
// tight, and clear the candidate for the next pass.
__global__ void lap_duals_kernel(const double* __restrict__ W, int ldw, int n, LapWs w,
                                 int pass) {
  if (pass == 1 && !ld_volatile_s32(&w.ctl->need_auction)) return;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const double* row = W + (size_t)i * ldw;
    double best = -INFINITY;
#pragma unroll 8
    for (int j = lane; j < n; j += 32) best = fmax(best, row[j] + w.v[j]);
    best = warp_max(best);
    if (lane == 0) {
      const int j = w.cand[i];
      w.cand[i] = -1;
      w.u[i] = -best;
      if (j >= 0 && row[j] + w.v[j] == best) {
        w.rowcol[i] = j;
        w.colrow[j] = i;
        w.wmat[j] = row[j];  // the concurrent completion reads W[colrow[j]][j] here
      } else {
        w.rowcol[i] = -1;
      }
    }
  }
}

// Shared memory for the completion state: label keys, test keys and
// potentials (8 bytes each) and colrow (4 bytes) per column.
constexpr size_t kSolveSmemCap = 225 * 1024;

__host__ __device__ inline size_t solve_smem_bytes(int n) {
  return al256((size_t)n * 8) * 4 + al256((size_t)n * 4);
}

// Order-preserving map of a double onto uint64 with integer operations only
// (FP64 instructions are scarce on this GPU; compares run on the ALU).
__device__ __forceinline__ unsigned long long okey(double x) {
  const long long b = __double_as_longlong(x);
  return (unsigned long long)(b ^ ((b >> 63) | (long long)0x8000000000000000ull));
}
__device__ __forceinline__ double okey_value(unsigned long long k) {
  const long long b = (long long)k;
  return __longlong_as_double(b ^ ((~b >> 63) | (long long)0x8000000000000000ull));
}

constexpr unsigned long long kVisited = ~0ull;  // label key of a popped column

// Block-wide argmin over (key, k) pairs, lexicographic, integer compares.
// The result is in *s_key / *s_k for every thread after the call.
template <int NT>
__device__ __forceinline__ void block_argmin_key(unsigned long long key, int k,
                                                 unsigned long long* rk, int* rkk,
                                                 unsigned long long* s_key, int* s_k) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o);
    const int ok2 = __shfl_xor_sync(0xffffffffu, k, o);
    if (ok < key || (ok == key && ok2 < k)) {
      key = ok;
      k = ok2;
    }
  }
  if (lane == 0) {
    rk[warp] = key;
    rkk[warp] = k;
  }
  __syncthreads();
  if (warp == 0) {
    key = lane < (NT / 32) ? rk[lane] : kVisited;
    k = lane < (NT / 32) ? rkk[lane] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o);
      const int ok2 = __shfl_xor_sync(0xffffffffu, k, o);
      if (ok < key || (ok == key && ok2 < k)) {
        key = ok;
        k = ok2;
      }
    }
    if (lane == 0) {
      *s_key = key;
      *s_k = k;
    }
  }
  __syncthreads();
}

// Exact completion in the Jonker-Volgenant form of the shortest augmenting
// path (cost c = -W, column potentials v only; an assigned row i satisfies
// c_i,col(i) - v_col(i) = min_j (c_ij - v_j)).  For a free row f the
// Dijkstra labels start at d_j = c_fj - v_j; popping column j1 at distance
// mu reaches row i = colrow[j1], whose relaxation is
//   d_j = min(d_j, c_ij - v_j - h),   h = c_i,j1 - v_j1 - mu.
// Each column also keeps t_j = -(v_j + d_j), so the test d_j > c_ij - v_j - h
// reads W_ij + h > t_j: one FP64 add per column and step, the comparison on
// order-preserving integer keys.  Among equal labels a free column is popped
// first.  At a free column every popped column gets v_j += d_j - mu (its
// label at the pop is kept in place of t_j) and the path is flipped.
// Column j's state belongs to thread j % 1024, so a step is one fused
// relax-and-argmin pass whose row loads are issued together.  The state
// sits in shared memory when it fits, else in the workspace.  Pass 0 stops
// after `budget` steps (0 = no limit) and asks for the auction; pass 1 runs
// only then.
constexpr int kSolveUnroll = 8;

__global__ void __launch_bounds__(kLapThreads, 1) lap_solve_kernel(const double* __restrict__ W,
                                                                   int ldw, int n, LapWs w,
                                                                   int pass, long long budget,
                                                                   int use_smem,
                                                                   int32_t* __restrict__ perm,
                                                                   LapStats* st) {
  if (pass == 1 && !ld_volatile_s32(&w.ctl->need_auction)) return;
  extern __shared__ __align__(16) unsigned char lap_sm[];
  __shared__ unsigned long long rk[kLapThreads / 32];
  __shared__ int rkk[kLapThreads / 32];
  __shared__ unsigned long long s_key;
  __shared__ int s_k;
  __shared__ double s_h;
  __shared__ int s_aug;
  __shared__ int s_next;
  const int tid = threadIdx.x;
  unsigned long long *dkey, *tkey;
  double *v, *wmat;
  int* colrow;
  if (use_smem) {
    unsigned char* p = lap_sm;
    dkey = reinterpret_cast<unsigned long long*>(p);
    p += al256((size_t)n * 8);
    tkey = reinterpret_cast<unsigned long long*>(p);
    p += al256((size_t)n * 8);
    v = reinterpret_cast<double*>(p);
    p += al256((size_t)n * 8);
    wmat = reinterpret_cast<double*>(p);
    p += al256((size_t)n * 8);
    colrow = reinterpret_cast<int*>(p);
    for (int j = tid; j < n; j += kLapThreads) {
      v[j] = w.v[j];
      colrow[j] = w.colrow[j];
    }
  } else {
    dkey = w.key;
    tkey = w.tkey;
    v = w.v;
    wmat = w.wmat;
    colrow = w.colrow;
  }
  // W of each column's assigned row (what h needs), kept in step with colrow.
  for (int j = tid; j < n; j += kLapThreads) {
    const int r = colrow[j];
    wmat[j] = r >= 0 ? W[(size_t)r * ldw + j] : 0.0;
  }
  int* pred = w.way;
  if (tid == 0) {
    s_aug = 0;
    st->status = 0;
    st->repeats = 0;
    st->auction_phases = pass == 1 && auction_on(w.ctl) ? w.ctl->phases : -1;
  }
  __syncthreads();

  long long total = 0;  // Dijkstra steps of this pass (the same in every thread)
  for (int f = -1;;) {
    // The next free row after f, kLapThreads rows per step.  A free row is
    // placed only by its own search, so this takes the free rows in the
    // order of a row-by-row scan, without a dependent read per row.
    int nf = n;
    for (int base = f + 1; base < n; base += kLapThreads) {
      if (tid == 0) s_next = n;
      __syncthreads();
      const int r = base + tid;
      if (r < n && w.rowcol[r] == -1) atomicMin(&s_next, r);
      __syncthreads();
      nf = s_next;
      __syncthreads();  // every thread has read s_next before it is reset
      if (nf < n) break;
    }
    if (nf >= n) break;
    f = nf;
    const double* rowf = W + (size_t)f * ldw;
    unsigned long long best = kVisited;
    int bk = 0x7fffffff;  // argmin tie key: j, plus n if column j is assigned
    for (int base = tid; base < n; base += kSolveUnroll * kLapThreads) {
      double wv[kSolveUnroll];
#pragma unroll
      for (int u = 0; u < kSolveUnroll; ++u) {
        const int j = base + u * kLapThreads;
        if (j < n) wv[u] = rowf[j];
      }
#pragma unroll
      for (int u = 0; u < kSolveUnroll; ++u) {
        const int j = base + u * kLapThreads;
        if (j >= n) continue;
        const unsigned long long dk = okey(-(wv[u] + v[j]));
        dkey[j] = dk;
        tkey[j] = okey(wv[u]);
        pred[j] = f;
        const int k = colrow[j] == -1 ? j : j + n;
        if (dk < best || (dk == best && k < bk)) {
          best = dk;
          bk = k;
        }
      }
    }
    block_argmin_key<kLapThreads>(best, bk, rk, rkk, &s_key, &s_k);
    double mu = okey_value(s_key);
    int key = s_k;
    int steps = 0;
    int j1;
    while (true) {
      if (key < 0 || key >= 2 * n || s_key == kVisited) {  // no finite label left
        if (tid == 0) st->status = 1;
        return;
      }
      j1 = key >= n ? key - n : key;
      if (j1 % kLapThreads == tid) {  // pop: keep the label where t_j was
        tkey[j1] = (unsigned long long)__double_as_longlong(mu);
        dkey[j1] = kVisited;
      }
      const int i = colrow[j1];
      if (i == -1) break;
      const double* rowi = W + (size_t)i * ldw;
      double wv[kSolveUnroll];
      // Issue this thread's row loads before h is known.
      const bool pre = n <= kSolveUnroll * kLapThreads;
      if (pre) {
#pragma unroll
        for (int u = 0; u < kSolveUnroll; ++u) {
          const int j = tid + u * kLapThreads;
          if (j < n) wv[u] = rowi[j];
        }
      }
      if (tid == 0) s_h = -(wmat[j1] + v[j1]) - mu;
      __syncthreads();
      const double h = s_h;
      best = kVisited;
      bk = 0x7fffffff;
      for (int base = tid; base < n; base += kSolveUnroll * kLapThreads) {
        if (!pre || base != tid) {
#pragma unroll
          for (int u = 0; u < kSolveUnroll; ++u) {
            const int j = base + u * kLapThreads;
            if (j < n) wv[u] = rowi[j];
          }
        }
#pragma unroll
        for (int u = 0; u < kSolveUnroll; ++u) {
          const int j = base + u * kLapThreads;
          if (j >= n) continue;
          unsigned long long dk = dkey[j];
          if (dk == kVisited) continue;
          const double x = wv[u] + h;
          const unsigned long long xk = okey(x);
          if (xk > tkey[j]) {  // W_ij + h > t_j: a shorter path to column j
            tkey[j] = xk;
            const unsigned long long nk = okey(-(x + v[j]));
            if (nk < dk) {
              dk = nk;
              dkey[j] = nk;
              pred[j] = i;
            }
          }
          const int k = colrow[j] == -1 ? j : j + n;
          if (dk < best || (dk == best && k < bk)) {
            best = dk;
            bk = k;
          }
        }
      }
      block_argmin_key<kLapThreads>(best, bk, rk, rkk, &s_key, &s_k);
      mu = okey_value(s_key);
      key = s_k;
      ++total;
      if (++steps > n) {
        if (tid == 0) st->status = 1;
        return;
      }
      if (budget > 0 && total > budget) {
        if (tid == 0) atomicExch(&w.ctl->need_auction, 1);
        return;
      }
    }
    // Potentials of the popped columns (label at the pop is in tkey), then
    // flip the path (j1 is free).
    for (int j = tid; j < n; j += kLapThreads)
      if (dkey[j] == kVisited) v[j] += __longlong_as_double((long long)tkey[j]) - mu;
    __syncthreads();
    if (tid == 0) {
      int j = j1;
      while (true) {
        const int r = pred[j];
        const int prev = w.rowcol[r];
        colrow[j] = r;
        wmat[j] = W[(size_t)r * ldw + j];
        w.rowcol[r] = j;
        if (r == f) break;
        j = prev;
      }
      ++s_aug;
    }
    __syncthreads();
  }
  if (tid == 0) st->steps = total;

  double val = 0.0;
  for (int i = tid; i < n; i += kLapThreads) {
    const int j = w.rowcol[i];
    perm[i] = j;
    val += W[(size_t)i * ldw + j];
  }
  val = warp_sum(val);
  __shared__ double rsum[kLapThreads / 32];
  const int lane = tid & 31, warp = tid >> 5;
  if (lane == 0) rsum[warp] = val;
  __syncthreads();
  if (warp == 0) {
    double t = rsum[lane];
    t = warp_sum(t);
    if (lane == 0) {
      st->value = t;
      st->augmented = s_aug;
    }
  }
}

// The same completion spread over a cluster of kLapCluster CTAs: CTA r of
// the cluster owns the columns [r S, (r+1) S) and keeps their labels, test
// keys, potentials and colrow in its own shared memory.  Each Dijkstra step
// every warp relaxes its columns, takes its best (key, index) by shuffles
// and writes it, with the row that column leads to and the next step's h,
// into its slot in its own CTA.  After one cluster barrier warp 0 of every
// CTA reads all kLapCluster x 8 slots through distributed shared memory (two
// per lane) and reduces them to the same winner by the same integer
// comparison, so every branch, return and barrier below is taken by all
// CTAs alike.  The slots are double-buffered by step parity: a slot is
// written again only two cluster barriers after the last remote read of it.
// The choices are those of lap_solve_kernel, so the results are
// bit-identical.
constexpr int kLapCluster = 8;
constexpr int kClusterThreads = 256;  // per CTA: a cheaper CTA and cluster barrier
constexpr int kClusterWarps = kClusterThreads / 32;
static_assert(kLapCluster * kClusterWarps == 64, "warp 0 reads two slots per lane");

struct CandSlot {
  unsigned long long key;
  int k;     // argmin tie key of the candidate (j, or j + n if assigned)
  int i;     // colrow of the candidate column
  double h;  // -(W[i][j] + v_j) - label of the candidate: the next step's h
};

// Column state of one CTA of a cluster completion, in its shared memory.
struct ColState {
  unsigned long long* dkey;  // label keys (kVisited once popped)
  unsigned long long* tkey;  // test keys; the label bits once popped
  double* v;                 // potentials
  double* wmat;              // W[colrow[j]][j], kept in step with colrow
  int* colrow;
};

__device__ __forceinline__ ColState col_state(unsigned char* sm, int S) {
  ColState c;
  c.dkey = reinterpret_cast<unsigned long long*>(sm);
  c.tkey = c.dkey + S;
  c.v = reinterpret_cast<double*>(c.tkey + S);
  c.wmat = c.v + S;
  c.colrow = reinterpret_cast<int*>(c.wmat + S);
  return c;
}

// First relaxation from the free row f: labels -(W_fj + v_j) for this CTA's
// columns [jb, jb + ns) and this thread's best (label key, tie key).  predl
// holds the predecessor rows of this CTA's columns (local index).
__device__ __forceinline__ void relax_first(const double* __restrict__ rowf, int f, int n, int jb,
                                            int ns, const ColState& c, int* predl,
                                            unsigned long long& best, int& bk) {
  best = kVisited;
  bk = 0x7fffffff;
  for (int jl = threadIdx.x; jl < ns; jl += kClusterThreads) {
    const int j = jb + jl;
    const double x = rowf[j];
    const unsigned long long dk = okey(-(x + c.v[jl]));
    c.dkey[jl] = dk;
    c.tkey[jl] = okey(x);
    predl[jl] = f;
    const int kk = c.colrow[jl] == -1 ? j : j + n;
    if (dk < best || (dk == best && kk < bk)) {
      best = dk;
      bk = kk;
    }
  }
}

// One Dijkstra step's relaxation with row i (shift h) over this CTA's
// unvisited columns, and this thread's best candidate afterwards.
__device__ __forceinline__ void relax_row(const double* __restrict__ rowi, double h, int i, int n,
                                          int jb, int ns, const ColState& c, int* predl,
                                          unsigned long long& best, int& bk) {
  const int tid = threadIdx.x;
  double wv[kSolveUnroll];
  const bool pre = ns <= kSolveUnroll * kClusterThreads;
  if (pre) {
#pragma unroll
    for (int u = 0; u < kSolveUnroll; ++u) {
      const int jl = tid + u * kClusterThreads;
      if (jl < ns) wv[u] = rowi[jb + jl];
    }
  }
  best = kVisited;
  bk = 0x7fffffff;
  for (int base = tid; base < ns; base += kSolveUnroll * kClusterThreads) {
    if (!pre || base != tid) {
#pragma unroll
      for (int u = 0; u < kSolveUnroll; ++u) {
        const int jl = base + u * kClusterThreads;
        if (jl < ns) wv[u] = rowi[jb + jl];
      }
    }
#pragma unroll
    for (int u = 0; u < kSolveUnroll; ++u) {
      const int jl = base + u * kClusterThreads;
      if (jl >= ns) continue;
      unsigned long long dk = c.dkey[jl];
      if (dk == kVisited) continue;
      const double x = wv[u] + h;
      const unsigned long long xk = okey(x);
      if (xk > c.tkey[jl]) {  // W_ij + h > t_j: a shorter path to column j
        c.tkey[jl] = xk;
        const unsigned long long nk = okey(-(x + c.v[jl]));
        if (nk < dk) {
          dk = nk;
          c.dkey[jl] = nk;
          predl[jl] = i;
        }
      }
      const int kk = c.colrow[jl] == -1 ? jb + jl : jb + jl + n;
      if (dk < best || (dk == best && kk < bk)) {
        best = dk;
        bk = kk;
      }
    }
  }
}

// The cluster-wide winner: each warp's best candidate into its slot; after
// the cluster barrier warp 0 of every CTA reads all kLapCluster x 8 slots
// through distributed shared memory (two per lane), reduces them by the
// same integer comparison and broadcasts through *s_win.  Slots are double-
// buffered by exchange parity (`par`): a slot is written again only two
// cluster barriers after the last remote read of it.
__device__ __forceinline__ CandSlot cluster_exchange(cg::cluster_group& cl, int cr, int n, int jb,
                                                     const ColState& c,
                                                     CandSlot (*slots)[kClusterWarps],
                                                     CandSlot* s_win, int& par,
                                                     unsigned long long best, int bk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ok = __shfl_xor_sync(0xffffffffu, best, o);
    const int ok2 = __shfl_xor_sync(0xffffffffu, bk, o);
    if (ok < best || (ok == best && ok2 < bk)) {
      best = ok;
      bk = ok2;
    }
  }
  if (lane == 0) {
    CandSlot cs{best, bk, -2, 0.0};
    if (best != kVisited && bk < 2 * n) {  // a column of this warp: stable during the step
      const int jl = (bk >= n ? bk - n : bk) - jb;
      cs.i = c.colrow[jl];
      cs.h = -(c.wmat[jl] + c.v[jl]) - okey_value(best);
    }
    slots[par][warp] = cs;
  }
  cl.sync();
  if (warp == 0) {
    // Lane l: slot l % 8 of CTAs l / 8 and l / 8 + 4.
    const CandSlot c0 = *cl.map_shared_rank(&slots[par][lane & 7], lane >> 3);
    const CandSlot c1 = *cl.map_shared_rank(&slots[par][lane & 7], (lane >> 3) + 4);
    CandSlot r = c0;
    if (c1.key < r.key || (c1.key == r.key && c1.k < r.k)) r = c1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ok = __shfl_xor_sync(0xffffffffu, r.key, o);
      const int ok2 = __shfl_xor_sync(0xffffffffu, r.k, o);
      const int oi = __shfl_xor_sync(0xffffffffu, r.i, o);
      const double oh = __shfl_xor_sync(0xffffffffu, r.h, o);
      if (ok < r.key || (ok == r.key && ok2 < r.k)) {
        r.key = ok;
        r.k = ok2;
        r.i = oi;
        r.h = oh;
      }
    }
    if (lane == 0) *s_win = r;
  }
  __syncthreads();
  par ^= 1;
  return *s_win;
}

__global__ void __launch_bounds__(kClusterThreads, 1) lap_solve_cluster_kernel(
    const double* __restrict__ W, int ldw, int n, LapWs w, int pass, long long budget,
    int32_t* __restrict__ perm, LapStats* st) {
  if (pass == 1 && !ld_volatile_s32(&w.ctl->need_auction)) return;  // uniform (earlier kernel)
  cg::cluster_group cl = cg::this_cluster();
  const int cr = (int)cl.block_rank();
  const int S = (n + kLapCluster - 1) / kLapCluster;
  const int jb = min(n, cr * S), ns = min(n, jb + S) - jb;
  extern __shared__ __align__(16) unsigned char lap_sm[];
  const ColState c = col_state(lap_sm, S);
  __shared__ CandSlot slots[2][kClusterWarps];
  __shared__ CandSlot s_win;
  __shared__ int s_aug;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int* pred = w.way;
  for (int jl = tid; jl < ns; jl += kClusterThreads) {
    c.v[jl] = w.v[jb + jl];
    const int r = w.colrow[jb + jl];
    c.colrow[jl] = r;
    c.wmat[jl] = r >= 0 ? W[(size_t)r * ldw + jb + jl] : 0.0;
  }
  if (tid == 0) {
    s_aug = 0;
    if (cr == 0) {
      st->status = 0;
      st->repeats = 0;
      st->auction_phases = pass == 1 && auction_on(w.ctl) ? w.ctl->phases : -1;
    }
  }
  int par = 0;
  cl.sync();

  long long total = 0;
  for (int f = 0; f < n; ++f) {
    if (w.rowcol[f] != -1) continue;  // uniform: written before the last cluster barrier
    unsigned long long best;
    int bk;
    relax_first(W + (size_t)f * ldw, f, n, jb, ns, c, pred + jb, best, bk);
    CandSlot win = cluster_exchange(cl, cr, n, jb, c, slots, &s_win, par, best, bk);
    double mu = okey_value(win.key);
    int steps = 0, j1;
    while (true) {
      if (win.k < 0 || win.k >= 2 * n || win.key == kVisited) {  // no finite label left (all CTAs)
        if (cr == 0 && tid == 0) st->status = 1;
        cl.sync();  // no CTA leaves while another may still read its slot
        return;
      }
      j1 = win.k >= n ? win.k - n : win.k;
      if (j1 >= jb && j1 < jb + ns && (j1 - jb) % kClusterThreads == tid) {
        c.tkey[j1 - jb] = (unsigned long long)__double_as_longlong(mu);
        c.dkey[j1 - jb] = kVisited;
      }
      if (win.i == -1) break;  // j1 is free: augment
      relax_row(W + (size_t)win.i * ldw, win.h, win.i, n, jb, ns, c, pred + jb, best, bk);
      win = cluster_exchange(cl, cr, n, jb, c, slots, &s_win, par, best, bk);
      mu = okey_value(win.key);
      ++total;
      if (++steps > n) {
        if (cr == 0 && tid == 0) st->status = 1;
        cl.sync();
        return;
      }
      if (budget > 0 && total > budget) {
        if (cr == 0 && tid == 0) atomicExch(&w.ctl->need_auction, 1);
        cl.sync();
        return;
      }
    }
    // Potentials of the popped columns, then (CTA 0) flip the path.
    for (int jl = tid; jl < ns; jl += kClusterThreads)
      if (c.dkey[jl] == kVisited) c.v[jl] += __longlong_as_double((long long)c.tkey[jl]) - mu;
    cl.sync();  // every CTA's pred writes and potentials are done
    if (cr == 0 && tid == 0) {
      int j = j1;
      while (true) {
        const int r = pred[j];
        const int prev = w.rowcol[r];
        const int owner = j / S;
        int* rc = cl.map_shared_rank(c.colrow, owner);
        double* rw = cl.map_shared_rank(c.wmat, owner);
        rc[j - owner * S] = r;
        rw[j - owner * S] = W[(size_t)r * ldw + j];
        w.rowcol[r] = j;
        if (r == f) break;
        j = prev;
      }
      ++s_aug;
    }
    cl.sync();
  }

  if (cr != 0) return;
  if (tid == 0) st->steps = total;
  double val = 0.0;
  for (int r = tid; r < n; r += kClusterThreads) {
    const int j = w.rowcol[r];
    perm[r] = j;
    val += W[(size_t)r * ldw + j];
  }
  val = warp_sum(val);
  __shared__ double rsum[kClusterWarps];
  if (lane == 0) rsum[warp] = val;
  __syncthreads();
  if (warp == 0) {
    double t = lane < kClusterWarps ? rsum[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) {
      st->value = t;
      st->augmented = s_aug;
    }
  }
}

// Concurrent completion: K clusters of kLapCluster CTAs, each running the
// search above from its own free row, with optimistic commits.
//
// A search reads the shared state (v, colrow and W[colrow[j]][j] in L2)
// into its shared memory at its start, after reading the number of
// published commits s0 with acquire semantics.  When it reaches a free
// column it takes a lock and checks every column it popped: if a commit
// numbered above s0 changed that column, the search is repeated from the
// same row on fresh state; otherwise it applies its potentials and its path
// flip, stamps every popped column with its own commit number and publishes
// that number with a release store.  Commits change only the columns their
// own search popped: they lower v_j there (v_j += d_j - mu with d_j <= mu),
// which can only raise the labels another search sees for those columns,
// and reassign the rows of the path, which are the rows of popped columns.
// A search none of whose popped columns was changed since s0 therefore pops
// the same columns in the same order on the current state as on its
// snapshot (stale or torn reads touch only columns it did not pop, or are
// caught by the check).  The applied searches are a sequence of exact
// shortest augmenting paths from feasible duals, the Hungarian method run in
// another order, so the assignment is optimal; between tied optima the
// choice may differ from run to run.
//
// Every branch and barrier is uniform inside a cluster: the row, s0, the
// stop flag and the lock outcome come from CTA 0's shared memory, the
// validation result from every CTA's flag, the pops from the exchange.
// Clusters never wait on one another except for the lock, whose holder is
// running its (wait-free) commit; the wait on it is bounded by limit_ns.
constexpr int kMaxSearches = 16;
constexpr int kDefaultSearches = 8;

__device__ __forceinline__ unsigned ld_acquire_gpu_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_gpu_s32(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct ConcJob {
  int f;        // free row of this search
  unsigned s0;  // commits published when it started
  int stop;     // leave: no row left, an error, or (pass 0) the budget is spent
  int ok;       // the lock was taken
  unsigned seq; // commits published when the lock was taken
};

__global__ void __launch_bounds__(kClusterThreads, 1) lap_solve_conc_kernel(
    const double* __restrict__ W, int ldw, int n, LapWs w, int pass, long long budget,
    uint64_t limit_ns) {
  if (pass == 1 && !ld_volatile_s32(&w.ctl->need_auction)) return;  // uniform (earlier kernel)
  cg::cluster_group cl = cg::this_cluster();
  const int cr = (int)cl.block_rank();
  const int S = (n + kLapCluster - 1) / kLapCluster;
  const int jb = min(n, cr * S), ns = min(n, jb + S) - jb;
  extern __shared__ __align__(16) unsigned char lap_sm[];
  const ColState c = col_state(lap_sm, S);
  int* predl = c.colrow + S;
  __shared__ CandSlot slots[2][kClusterWarps];
  __shared__ CandSlot s_win;
  __shared__ ConcJob s_job;
  __shared__ int s_conf;
  __shared__ int s_rows[32];   // CTA 0: free rows taken from the queue, not yet searched
  __shared__ int s_nrows, s_rpos;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) s_nrows = s_rpos = 0;
  ConcCtl* cc = &w.ctl->cc[pass];
  const ConcJob* job0 = cl.map_shared_rank(&s_job, 0);
  int par = 0;
  int f = -1;
  bool retry = false;
  while (true) {
    // Next row (or the same one again), and s0.  Warp 0 of CTA 0 takes 32
    // rows of the queue per atomic and keeps the free ones (rows are only
    // ever assigned by their own search, so "free" cannot go stale).
    if (cr == 0 && tid < 32) {
      int stop = 0;
      if (lane == 0)
        stop = ld_volatile_s32(&cc->err) != 0 ||
               (pass == 0 && ld_volatile_s32(&w.ctl->need_auction) != 0);
      stop = __shfl_sync(0xffffffffu, stop, 0);
      int row = f;
      if (!stop && !retry) {
        row = n;
        for (int chunk = 0; chunk < n / 32 + 3; ++chunk) {  // ceil(n / 32) refills at most
          __syncwarp();
          if (s_rpos < s_nrows) {
            row = s_rows[s_rpos];
            break;
          }
          int base = 0;
          if (lane == 0) base = atomicAdd(&cc->next_row, 32);
          base = __shfl_sync(0xffffffffu, base, 0);
          if (base >= n) break;
          const int r = base + lane;
          const bool fr = r < n && __ldcg(&w.rowcol[r]) == -1;
          const unsigned m = __ballot_sync(0xffffffffu, fr);
          if (fr) s_rows[__popc(m & ((1u << lane) - 1u))] = r;
          __syncwarp();
          if (lane == 0) {
            s_nrows = __popc(m);
            s_rpos = 0;
          }
        }
        __syncwarp();
        if (lane == 0 && row < n) ++s_rpos;
      }
      if (lane == 0) {
        ConcJob j{};
        j.stop = stop || row >= n;
        j.f = row;
        j.s0 = ld_acquire_gpu_u32(&cc->seq);
        s_job = j;
      }
    }
    cl.sync();
    const int stop = job0->stop;
    f = job0->f;
    const unsigned s0 = job0->s0;
    if (stop) {
      cl.sync();  // no CTA leaves while another may still read its shared memory
      return;
    }
    // Snapshot of this CTA's columns, then the first relaxation from f.
    for (int jl = tid; jl < ns; jl += kClusterThreads) {
      c.v[jl] = __ldcg(&w.v[jb + jl]);
      c.colrow[jl] = __ldcg(&w.colrow[jb + jl]);
      c.wmat[jl] = __ldcg(&w.wmat[jb + jl]);
    }
    __syncthreads();  // the exchange reads other threads' snapshot entries
    unsigned long long best;
    int bk;
    relax_first(W + (size_t)f * ldw, f, n, jb, ns, c, predl, best, bk);
    CandSlot win = cluster_exchange(cl, cr, n, jb, c, slots, &s_win, par, best, bk);
    double mu = okey_value(win.key);
    int steps = 0, j1;
    bool failed = false;
    while (true) {
      if (win.k < 0 || win.k >= 2 * n || win.key == kVisited) {  // no finite label left
        failed = true;
        break;
      }
      j1 = win.k >= n ? win.k - n : win.k;
      if (j1 >= jb && j1 < jb + ns && (j1 - jb) % kClusterThreads == tid) {
        c.tkey[j1 - jb] = (unsigned long long)__double_as_longlong(mu);
        c.dkey[j1 - jb] = kVisited;
      }
      if (win.i == -1) break;  // j1 is free: commit
      relax_row(W + (size_t)win.i * ldw, win.h, win.i, n, jb, ns, c, predl, best, bk);
      win = cluster_exchange(cl, cr, n, jb, c, slots, &s_win, par, best, bk);
      mu = okey_value(win.key);
      if (++steps > n) {
        failed = true;
        break;
      }
    }
    if (failed) {
      if (cr == 0 && tid == 0) atomicExch(&cc->err, 1);
      cl.sync();
      return;
    }
    // Lock (bounded wait), then every CTA checks its popped columns.
    if (cr == 0 && tid == 0) {
      const uint64_t t0 = globaltimer_ns();
      int ok = 1;
      while (atomicCAS(&cc->lock, 0, 1) != 0) {
        if (globaltimer_ns() - t0 > limit_ns) {
          ok = 0;
          atomicExch(&cc->err, 1);
          break;
        }
        __nanosleep(64);
      }
      __threadfence();  // acquire: the holders' writes before their release
      s_job.ok = ok;
      s_job.seq = ok ? ld_acquire_gpu_u32(&cc->seq) : 0u;
    }
    cl.sync();
    if (!job0->ok) {
      cl.sync();
      return;
    }
    const unsigned seq = job0->seq;
    int conf = 0;
    for (int jl = tid; jl < ns; jl += kClusterThreads)
      if (c.dkey[jl] == kVisited && __ldcg(&w.cseq[jb + jl]) > s0) conf = 1;
    conf = __syncthreads_or(conf);
    if (tid == 0) s_conf = conf;
    cl.sync();
    int any = tid < kLapCluster ? *cl.map_shared_rank(&s_conf, tid) : 0;
    any = __syncthreads_or(any);
    if (any) {
      if (cr == 0 && tid == 0) {
        atomicAdd(&cc->aborts, 1);
        atomicAdd((unsigned long long*)&cc->steps, (unsigned long long)steps);
        st_release_gpu_s32(&cc->lock, 0);
      }
      retry = true;
      continue;  // the next cl.sync orders the flag reads before s_conf is written again
    }
    // Apply: potentials and stamps of the popped columns, then (CTA 0) the
    // path flip, the publication of commit seq + 1 and the unlock.
    const unsigned mine = seq + 1;
    for (int jl = tid; jl < ns; jl += kClusterThreads)
      if (c.dkey[jl] == kVisited) {
        w.v[jb + jl] = c.v[jl] + __longlong_as_double((long long)c.tkey[jl]) - mu;
        w.cseq[jb + jl] = mine;
      }
    __threadfence();
    cl.sync();  // every CTA's writes are done; pred is final
    if (cr == 0 && tid == 0) {
      int j = j1;
      for (int hop = 0; hop <= n; ++hop) {
        const int owner = j / S;
        const int r = *cl.map_shared_rank(predl + (j - owner * S), owner);
        const int prev = r >= 0 && r < n ? __ldcg(&w.rowcol[r]) : -1;
        if (r < 0 || r >= n || (r != f && (prev < 0 || prev >= n))) {  // never on valid state
          atomicExch(&cc->err, 1);
          break;
        }
        w.colrow[j] = r;
        w.wmat[j] = W[(size_t)r * ldw + j];
        w.rowcol[r] = j;
        w.cseq[j] = mine;
        if (r == f) break;
        j = prev;
      }
      __threadfence();
      st_release_gpu_u32(&cc->seq, mine);
      atomicAdd(&cc->commits, 1);
      atomicAdd((unsigned long long*)&cc->steps, (unsigned long long)steps);
      // The budget counts the applied searches only: they are the work one
      // search at a time would do (repeated searches are the price of
      // concurrency, not a sign of a hard instance).
      const long long tot = atomicAdd((unsigned long long*)&cc->applied_steps,
                                      (unsigned long long)steps) + steps;
      if (pass == 0 && budget > 0 && tot > budget) atomicExch(&w.ctl->need_auction, 1);
      st_release_gpu_s32(&cc->lock, 0);
    }
    retry = false;
    cl.sync();  // the flip has read every CTA's pred before the next search writes it
  }
}

// Result of the concurrent completion: perm, the assignment value and the
// statistics of the pass that ran last.
__global__ void lap_conc_finish_kernel(const double* __restrict__ W, int ldw, int n, LapWs w,
                                       int32_t* __restrict__ perm, LapStats* st) {
  const int pass = ld_volatile_s32(&w.ctl->need_auction) ? 1 : 0;
  const ConcCtl& cc = w.ctl->cc[pass];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double val = 0.0;
  int unplaced = 0;
  for (int r = tid; r < n; r += blockDim.x) {
    const int j = w.rowcol[r];
    perm[r] = j;
    if (j >= 0)
      val += W[(size_t)r * ldw + j];
    else
      unplaced = 1;
  }
  val = warp_sum(val);
  __shared__ double rsum[32];
  if (lane == 0) rsum[warp] = val;
  unplaced = __syncthreads_or(unplaced);
  if (warp == 0) {
    double t = lane < (int)(blockDim.x >> 5) ? rsum[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) {
      st->value = t;
      st->augmented = cc.commits;
      st->status = (cc.err != 0 || unplaced) ? 1 : 0;
      st->auction_phases = pass == 1 && auction_on(w.ctl) ? w.ctl->phases : -1;
      st->repeats = cc.aborts;
      st->steps = cc.steps;
    }
  }
}

// Auction CTA size: about 8 columns per thread, 32..1024 threads.
int auction_threads(int n) {
  int t = 32;
  while (t < kAucMaxThreads && t * kAucUnroll < n) t *= 2;
  return t;
}

int launch_auction(const double* W, int ldw, int n, LapWs w, int num_sms, uint64_t limit_ns,
                   cudaStream_t s) {
  static DeviceCache per_sm[11];  // by log2(threads)
  const int t = auction_threads(n);
  const int lg = 31 - __builtin_clz((unsigned)t);
  const int occ = device_cached(per_sm[lg], [t] {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, lap_auction_kernel, t, 0) != cudaSuccess)
      return -1;
    return v > 0 ? v : -1;
  });
  if (occ < 0 || num_sms < 1) return -1;
  int blocks = occ * num_sms;
  if (blocks > n) blocks = n;
  void* args[] = {(void*)&W, (void*)&ldw, (void*)&n, (void*)&w, (void*)&limit_ns};
  if (cudaLaunchCooperativeKernel((const void*)lap_auction_kernel, dim3(blocks), dim3(t), args,
                                  0, s) != cudaSuccess)
    return -1;
  return 1;
}

}  // namespace

namespace {

// Can a cluster of kLapCluster CTAs with `smem` bytes each be resident?
bool cluster_ok(size_t smem) {
  static DeviceCache attr;
  if (device_cached(attr, [] {
        if (cudaFuncSetAttribute(lap_solve_cluster_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSolveSmemCap) != cudaSuccess) {
          cudaGetLastError();
          return -1;
        }
        return 1;
      }) < 0)
    return false;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(kLapCluster);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kLapCluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, lap_solve_cluster_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return clusters >= 1;
}

// Concurrent completion: how many clusters of kLapCluster CTAs with `smem`
// bytes each can be resident together, capped at `want`.
int conc_clusters(size_t smem, int want) {
  static DeviceCache attr;
  if (device_cached(attr, [] {
        if (cudaFuncSetAttribute(lap_solve_conc_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSolveSmemCap) != cudaSuccess) {
          cudaGetLastError();
          return -1;
        }
        return 1;
      }) < 0)
    return 0;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(kLapCluster * want);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kLapCluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, lap_solve_conc_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return clusters < want ? clusters : want;
}

}  // namespace

size_t lap_workspace_bytes(int n) {
  return 7 * al256((size_t)n * sizeof(int)) + 6 * al256((size_t)n * sizeof(double)) +
         al256(sizeof(LapCtl));
}

int launch_lap(const double* W, int ldw, int n, int32_t* perm, LapStats* st, void* ws,
               int num_sms, uint64_t limit_ns, cudaStream_t s, int searches) {
  LapWs w = carve(ws, n);
  // The auction key holds a 20-bit row index; beyond that the first
  // completion runs without a budget.
  const bool can_auction = n < (int)kNoOwner;
  const long long budget = can_auction ? 64ll * n : 0;
  int blocks = (n + 255) / 256;
  if (blocks > 1184) blocks = 1184;
  int rblocks = (n * 32 + 255) / 256;
  if (rblocks > 2368) rblocks = 2368;
  const size_t sm = solve_smem_bytes(n);
  const int use_smem = sm <= kSolveSmemCap;
  static DeviceCache attr;
  if (use_smem && device_cached(attr, [] {
                    return cudaFuncSetAttribute(lap_solve_kernel,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)kSolveSmemCap) == cudaSuccess
                               ? 1
                               : -1;
                  }) < 0)
    return -1;
  const size_t dsm = use_smem ? sm : 0;
  // The cluster completion for large n (its column state fits on chip up to
  // n = 8 x 7,800); the one-CTA kernel below that.
  const int S = (n + kLapCluster - 1) / kLapCluster;
  const size_t csm = (size_t)S * (4 * sizeof(double) + sizeof(int));
  const bool use_cluster = n >= 1024 && csm <= kSolveSmemCap && cluster_ok(csm);
  // Concurrent searches (K clusters) unless one is asked for; they add pred
  // (4 bytes per column) to the per-CTA state.
  const size_t qsm = csm + (size_t)S * sizeof(int);
  int K = searches > 0 ? searches : kDefaultSearches;
  if (K > kMaxSearches) K = kMaxSearches;
  if (use_cluster && K > 1 && qsm <= kSolveSmemCap) K = conc_clusters(qsm, K);
  const bool use_conc = use_cluster && K > 1 && qsm <= kSolveSmemCap;
  auto solve = [&](int pass, long long bud) -> bool {
    if (use_conc) {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(kLapCluster * K);
      cfg.blockDim = dim3(kClusterThreads);
      cfg.dynamicSmemBytes = qsm;
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = kLapCluster;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, lap_solve_conc_kernel, W, ldw, n, w, pass, bud,
                                limit_ns) == cudaSuccess;
    }
    if (use_cluster) {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(kLapCluster);
      cfg.blockDim = dim3(kClusterThreads);
      cfg.dynamicSmemBytes = csm;
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = kLapCluster;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, lap_solve_cluster_kernel, W, ldw, n, w, pass, bud, perm,
                                st) == cudaSuccess;
    }
    lap_solve_kernel<<<1, kLapThreads, dsm, s>>>(W, ldw, n, w, pass, bud, use_smem, perm, st);
    return cudaPeekAtLastError() == cudaSuccess;
  };
  lap_init_kernel<<<blocks, 256, 0, s>>>(w, n);
  lap_rowmax_kernel<<<rblocks, 256, 0, s>>>(W, ldw, n, w);
  {
    const int rows_per = 64;
    dim3 g((n + 255) / 256, (n + rows_per - 1) / rows_per);
    lap_colpot_kernel<<<g, 256, 0, s>>>(W, ldw, n, w, rows_per);
  }
  lap_conflicts_kernel<<<blocks, 256, 0, s>>>(w, n);
  lap_candidates_kernel<<<blocks, 256, 0, s>>>(w, n, 0);
  lap_duals_kernel<<<rblocks, 256, 0, s>>>(W, ldw, n, w, 0);
  if (!solve(0, budget)) return -1;
  int launches = 7;
  if (can_auction) {
    // Each of these returns at once unless the first completion ran out.
    if (launch_auction(W, ldw, n, w, num_sms, limit_ns, s) < 0) return -1;
    lap_candidates_kernel<<<blocks, 256, 0, s>>>(w, n, 1);
    lap_duals_kernel<<<rblocks, 256, 0, s>>>(W, ldw, n, w, 1);
    if (!solve(1, 0)) return -1;
    launches += 4;
  }
  if (use_conc) {
    lap_conc_finish_kernel<<<1, 256, 0, s>>>(W, ldw, n, w, perm, st);
    launches += 1;
  }
  return cudaPeekAtLastError() == cudaSuccess ? launches : -1;
}

}  // namespace fram
