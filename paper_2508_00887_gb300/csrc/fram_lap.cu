// Discretisation (eq. 2 / Alg. 1 step 10 of arXiv 2508.00887):
//   perm = argmax_{P in Pi_n} <P, W>   (= argmin ||P - W||_F over permutations)
//
// Two kernels.
//  1. Row argmax, one warp per row (ties -> lowest column).  If the row
//     argmaxes already form a permutation it is optimal: the sum of row
//     maxima bounds every assignment from above.  This is the common case
//     once FRAM has converged, because N is then close to a permutation.
//  2. One CTA completes the assignment exactly with the Hungarian method in
//     its shortest-augmenting-path form (Kuhn 1955 with row/column
//     potentials), warm-started from the conflict-free part of step 1:
//     u_i = -max_j W_ij, v_j = 0 is dual feasible for cost -W and tight on
//     every argmax edge.  Each Dijkstra step scans all columns in parallel
//     and picks the closest unvisited column with a block-wide argmin.
#include <math.h>

#include "fram_internal.cuh"

namespace fram {

namespace {

constexpr int kLapThreads = 1024;

struct LapWs {
  int* argc;       // [n] row argmax column
  int* owner;      // [n] lowest row claiming column j (INT_MAX if none)
  int* colrow;     // [n] row matched to column j, -1 if free
  int* rowcol;     // [n] column matched to row i, -1 if free
  int* way;        // [n] predecessor column on the search tree, -1 = root
  int* used;       // [n]
  double* rowmax;  // [n]
  double* u;       // [n]
  double* v;       // [n]
  double* minv;    // [n]
};

__host__ __device__ inline size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

__host__ __device__ inline LapWs carve(void* base, int n) {
  LapWs w;
  char* p = static_cast<char*>(base);
  const size_t ib = al256((size_t)n * sizeof(int)), db = al256((size_t)n * sizeof(double));
  w.argc = reinterpret_cast<int*>(p); p += ib;
  w.owner = reinterpret_cast<int*>(p); p += ib;
  w.colrow = reinterpret_cast<int*>(p); p += ib;
  w.rowcol = reinterpret_cast<int*>(p); p += ib;
  w.way = reinterpret_cast<int*>(p); p += ib;
  w.used = reinterpret_cast<int*>(p); p += ib;
  w.rowmax = reinterpret_cast<double*>(p); p += db;
  w.u = reinterpret_cast<double*>(p); p += db;
  w.v = reinterpret_cast<double*>(p); p += db;
  w.minv = reinterpret_cast<double*>(p); p += db;
  return w;
}

__global__ void lap_init_owner_kernel(LapWs w, int n) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    w.owner[j] = 0x7fffffff;
}

__global__ void lap_rowmax_kernel(const double* __restrict__ W, int ldw, int n, LapWs w) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const double* row = W + (size_t)i * ldw;
    double best = -INFINITY;
    int bj = 0x7fffffff;
    for (int j = lane; j < n; j += 32) {
      const double x = row[j];
      if (x > best) {
        best = x;
        bj = j;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      if (ob > best || (ob == best && oj < bj)) {
        best = ob;
        bj = oj;
      }
    }
    if (lane == 0) {
      if (bj == 0x7fffffff) bj = 0;
      w.argc[i] = bj;
      w.rowmax[i] = best;
      atomicMin(&w.owner[bj], i);
    }
  }
}

// Block-wide argmin over (value, index), ties -> lowest index.  Result in
// s_val/s_idx for every thread after the call.
__device__ __forceinline__ void block_argmin(double v, int j, double* rv, int* rj, double* s_val,
                                             int* s_idx) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oj = __shfl_xor_sync(0xffffffffu, j, o);
    if (ov < v || (ov == v && oj < j)) {
      v = ov;
      j = oj;
    }
  }
  if (lane == 0) {
    rv[warp] = v;
    rj[warp] = j;
  }
  __syncthreads();
  if (warp == 0) {
    v = lane < (kLapThreads / 32) ? rv[lane] : INFINITY;
    j = lane < (kLapThreads / 32) ? rj[lane] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oj = __shfl_xor_sync(0xffffffffu, j, o);
      if (ov < v || (ov == v && oj < j)) {
        v = ov;
        j = oj;
      }
    }
    if (lane == 0) {
      *s_val = v;
      *s_idx = j;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kLapThreads, 1) lap_solve_kernel(const double* __restrict__ W,
                                                                   int ldw, int n, LapWs w,
                                                                   int32_t* __restrict__ perm,
                                                                   LapStats* st) {
  __shared__ double rv[kLapThreads / 32];
  __shared__ int rj[kLapThreads / 32];
  __shared__ double s_val;
  __shared__ int s_idx;
  __shared__ int s_aug;
  const int tid = threadIdx.x;
  for (int j = tid; j < n; j += kLapThreads) {
    w.colrow[j] = -1;
    w.v[j] = 0.0;
  }
  for (int i = tid; i < n; i += kLapThreads) w.rowcol[i] = -1;
  __syncthreads();
  for (int i = tid; i < n; i += kLapThreads) {
    const int j = w.argc[i];
    w.u[i] = -w.rowmax[i];
    if (w.owner[j] == i) {
      w.colrow[j] = i;
      w.rowcol[i] = j;
    }
  }
  if (tid == 0) {
    s_aug = 0;
    st->status = 0;
  }
  __syncthreads();

  for (int root = 0; root < n; ++root) {
    if (w.rowcol[root] != -1) continue;  // uniform: read after a barrier
    for (int j = tid; j < n; j += kLapThreads) {
      w.minv[j] = INFINITY;
      w.used[j] = 0;
      w.way[j] = -1;
    }
    __syncthreads();
    int i0 = root, j0 = -1, steps = 0;
    while (true) {
      double best = INFINITY;
      int bj = 0x7fffffff;
      const double ui = w.u[i0];
      const double* row = W + (size_t)i0 * ldw;
      for (int j = tid; j < n; j += kLapThreads) {
        if (w.used[j]) continue;
        const double cur = -row[j] - ui - w.v[j];
        double mv = w.minv[j];
        if (cur < mv) {
          mv = cur;
          w.minv[j] = cur;
          w.way[j] = j0;
        }
        if (mv < best) {
          best = mv;
          bj = j;
        }
      }
      block_argmin(best, bj, rv, rj, &s_val, &s_idx);
      const double delta = s_val;
      const int j1 = s_idx;
      if (j1 < 0 || j1 >= n) {  // cannot happen for finite W; stop safely
        if (tid == 0) st->status = 1;
        return;
      }
      for (int j = tid; j < n; j += kLapThreads) {
        if (w.used[j]) {
          w.v[j] -= delta;
          w.u[w.colrow[j]] += delta;
        } else {
          w.minv[j] -= delta;
        }
      }
      if (tid == 0) {
        w.u[root] += delta;
        w.used[j1] = 1;
      }
      __syncthreads();
      j0 = j1;
      const int nxt = w.colrow[j1];
      if (nxt == -1) break;
      i0 = nxt;
      if (++steps > n) {
        if (tid == 0) st->status = 1;
        return;
      }
    }
    if (tid == 0) {
      int j = j0;
      while (j != -1) {
        const int jp = w.way[j];
        const int r = (jp == -1) ? root : w.colrow[jp];
        w.colrow[j] = r;
        w.rowcol[r] = j;
        j = jp;
      }
      ++s_aug;
    }
    __syncthreads();
  }

  double val = 0.0;
  for (int i = tid; i < n; i += kLapThreads) {
    const int j = w.rowcol[i];
    perm[i] = j;
    val += W[(size_t)i * ldw + j];
  }
  val = warp_sum(val);
  const int lane = tid & 31, warp = tid >> 5;
  if (lane == 0) rv[warp] = val;
  __syncthreads();
  if (warp == 0) {
    double t = rv[lane];
    t = warp_sum(t);
    if (lane == 0) {
      st->value = t;
      st->augmented = s_aug;
    }
  }
}

}  // namespace

size_t lap_workspace_bytes(int n) {
  return 6 * al256((size_t)n * sizeof(int)) + 4 * al256((size_t)n * sizeof(double));
}

int launch_lap(const double* W, int ldw, int n, int32_t* perm, LapStats* st, void* ws,
               cudaStream_t s) {
  LapWs w = carve(ws, n);
  int blocks = (n + 255) / 256;
  if (blocks > 1184) blocks = 1184;
  lap_init_owner_kernel<<<blocks, 256, 0, s>>>(w, n);
  int rblocks = (n * 32 + 255) / 256;
  if (rblocks > 2368) rblocks = 2368;
  lap_rowmax_kernel<<<rblocks, 256, 0, s>>>(W, ldw, n, w);
  lap_solve_kernel<<<1, kLapThreads, 0, s>>>(W, ldw, n, w, perm, st);
  return cudaPeekAtLastError() == cudaSuccess ? 3 : -1;
}

}  // namespace fram
