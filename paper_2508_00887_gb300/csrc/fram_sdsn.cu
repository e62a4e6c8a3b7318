// SDSN -- Scaling Doubly Stochastic Normalization (Alg. 2 of arXiv
// 2508.00887) as one persistent, cooperatively launched kernel.
//
//   step 1   Y = (theta/2) X / max(X)
//   sweep    Y_ij <- max(0, Y_ij + 1/n + S/n^2 - r_i/n - c_j/n)      (eq. 7)
//            with S = sum Y, r = row sums, c = column sums of the current Y
//   stop     gamma = sum(Y)/n - 1 <= gamma_tol, or max_sweeps sweeps
//            (gamma of Sec. 5.2, taken on each sweep's clamped result)
//
// Layout: the n x n matrix is cut into a P x Q grid of tiles, one CTA per
// tile.  Each sweep reads the tile once and writes it once; the same pass
// accumulates the new tile's row sums (warp shuffles), column sums (per-lane
// registers, combined across warps in shared memory) and total, which the
// CTA publishes as partials, double-buffered by sweep parity.  After one
// grid barrier every CTA loads the Q row partials of its rows, the P column
// partials of its columns and all P*Q totals with independent loads (a
// single L2 round trip), and combines them in a fixed order, so every CTA
// agrees bit for bit on S, on gamma and therefore on when to stop.  When the
// tile fits in shared memory it stays there for all sweeps, and global
// memory is touched only to load X and to store the result.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "fram_internal.cuh"

namespace fram {

namespace {

constexpr int kSdsnThreads = 512;
constexpr int kSdsnWarps = kSdsnThreads / 32;
constexpr size_t kSmemCap = 200 * 1024;
constexpr int kMaxGrid = 16;  // P, Q <= 16 (gather unrolled to this bound)

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

template <typename T, typename TIn>
struct SdsnK {
  int n, P, Q, tr, tc, resident;
  int block0;  // grouped launches: first CTA of this problem
  int vec_x, vec_y;  // X / Y rows can be accessed with 16-byte (8-byte) vectors
  int mode;  // 0: Y0 = (theta/2) X / max(X) (Alg. 2 step 1); 1: Y0 = X (continue a run)
  const TIn* X;
  int ldx;
  T* Y;
  int ldy;
  double theta, gamma_tol;
  int max_sweeps;
  const unsigned long long* xmax_key;
  const SdsnStats* gate;  // optional: run no sweep if gate->gamma <= gate_tol
  double gate_tol;
  SdsnStats* stats;
  T* rpart;       // [2][Q][n] row partials (sweep arithmetic type)
  T* cpart;       // [2][P][n] column partials
  double* tpart;  // [2][P*Q] tile totals (S and gamma are always FP64)
  GridBarrier* bar;
  uint64_t limit_ns;
  double one;  // 1.0, read at run time (see addx)
};

template <typename T>
__host__ __device__ inline size_t sdsn_smem_bytes(int tr, int tc, bool resident) {
  size_t b = 0;
  if (resident) b += align16((size_t)tr * tc * sizeof(T));
  b += align16((size_t)kSdsnWarps * tc * sizeof(T));  // per-warp column sums
  b += align16((size_t)tr * sizeof(T));                // row sums of the tile
  b += align16((size_t)tr * sizeof(T));                // a_i = 1/n + S/n^2 - r_i/n
  b += align16((size_t)tc * sizeof(T));                // b_j = c_j/n
  return b;
}

// max(0, y) without a floating-point instruction: clear y if its sign bit
// is set (IEEE: every value with the sign bit set is <= 0, NaN excluded).
__device__ __forceinline__ double relu(double y) {
  const long long b = __double_as_longlong(y);
  return __longlong_as_double(b & ~(b >> 63));
}
__device__ __forceinline__ float relu(float y) {
  const int b = __float_as_int(y);
  return __int_as_float(b & ~(b >> 31));
}

// Sweep additions: FP64 ones as fma with a run-time 1.0 (add64, exact and
// faster on this GPU's FP64 pipe), FP32 ones plain.
__device__ __forceinline__ double addx(double a, double b, double one) { return add64(a, b, one); }
__device__ __forceinline__ double subx(double a, double b, double one) { return sub64(a, b, one); }
__device__ __forceinline__ float addx(float a, float b, double) { return a + b; }
__device__ __forceinline__ float subx(float a, float b, double) { return a - b; }

// Sum of v[0..7] over the 32 lanes of a warp, transposed: afterwards lane l
// holds the total of entry ((l >> 4) & 1) * 4 + ((l >> 3) & 1) * 2 +
// ((l >> 2) & 1) (lanes l..l^3 agree).  9 additions per warp for 8 row sums
// instead of 40 -- FP64 additions are scarce on this GPU.  Fixed order.
template <typename T>
__device__ __forceinline__ T transpose_reduce8(T (&v)[8], int lane) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const bool hi = lane & 16;
    const T send = hi ? v[m] : v[m + 4];
    const T keep = hi ? v[m + 4] : v[m];
    v[m] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const bool hi = lane & 8;
    const T send = hi ? v[m] : v[m + 2];
    const T keep = hi ? v[m + 2] : v[m];
    v[m] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  {
    const bool hi = lane & 4;
    const T send = hi ? v[0] : v[1];
    const T keep = hi ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  T r = v[0] + __shfl_xor_sync(0xffffffffu, v[0], 2);
  return r + __shfl_xor_sync(0xffffffffu, r, 1);
}

__device__ __forceinline__ int transpose_index8(int lane) {
  return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}

// VEC consecutive elements of U at p: one 16/8/4-byte access when `vec`
// (the address is then VEC*sizeof(U)-aligned), element by element otherwise
// or when the vector would cross `lim` (elements valid: p[0 .. lim-1]).
template <typename U, int V>
__device__ __forceinline__ void vec_load(const U* p, bool vec, int lim, U (&out)[V]) {
  if (vec && lim >= V) {
    if constexpr (V * sizeof(U) == 16) {
      const uint4 r = *reinterpret_cast<const uint4*>(p);
      memcpy(out, &r, 16);
      return;
    } else if constexpr (V * sizeof(U) == 8) {
      const uint2 r = *reinterpret_cast<const uint2*>(p);
      memcpy(out, &r, 8);
      return;
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v) out[v] = v < lim ? p[v] : U(0);
}

template <typename U, int V>
__device__ __forceinline__ void vec_store(U* p, bool vec, int lim, const U (&in)[V]) {
  if (vec && lim >= V) {
    if constexpr (V * sizeof(U) == 16) {
      uint4 r;
      memcpy(&r, in, 16);
      *reinterpret_cast<uint4*>(p) = r;
      return;
    } else if constexpr (V * sizeof(U) == 8) {
      uint2 r;
      memcpy(&r, in, 8);
      *reinterpret_cast<uint2*>(p) = r;
      return;
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v)
    if (v < lim) p[v] = in[v];
}

// One pass over the tile.  FIRST: Y = (theta/2) X / m (mode 0) or Y = X
// (mode 1).  Otherwise the fused P1+P2 sweep.  Both accumulate the new
// tile's sums and publish them into partial buffer `wb`.
// MAXC > 0: lane l owns the 16-byte column groups l + 32 s (s < MAXC) of
// VEC elements, moves them with vector accesses and keeps their column sums
// in registers; for FP32 the next row's groups are loaded before the current
// row is computed, so each warp keeps two rows of loads in flight.
// MAXC == 0 (very wide tiles): one element per lane step, per-warp column
// sums in shared memory.
template <typename T, typename TIn, int MAXC, bool FIRST>
__device__ __forceinline__ void sdsn_pass(const SdsnK<T, TIn>& p, T* tile, int ldt, T* colacc,
                                          T* rowsum, T* arow, T* bcol, int nr,
                                          int nc, int r0, int c0, int bi, int bj, T scale, int wb,
                                          int blk, int nblk, T cS, T inv_n_t, double* s_total) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double one = p.one;
  T* wacc = colacc + warp * p.tc;
  if constexpr (MAXC == 0) {
    for (int j = lane; j < nc; j += 32) wacc[j] = T(0);
    for (int i = warp; i < nr; i += kSdsnWarps) {
      T* row = tile + (size_t)i * ldt;
      const TIn* xrow = FIRST ? p.X + (size_t)(r0 + i) * p.ldx + c0 : nullptr;
      const T ai = FIRST ? T(0) : addx(arow[i], cS, one);
      T racc = T(0);
      for (int j = lane; j < nc; j += 32) {
        T y;
        if (FIRST)
          y = p.mode == 0 ? (T)xrow[j] * scale : (T)xrow[j];
        else
          y = relu(subx(addx(row[j], ai, one), bcol[j], one));
        row[j] = y;
        racc = addx(racc, y, one);
        wacc[j] = addx(wacc[j], y, one);
      }
      racc = warp_sum(racc);
      if (lane == 0) rowsum[i] = racc;
    }
  } else {
    constexpr int VEC = 16 / (int)sizeof(T);
    constexpr bool PREF = sizeof(T) == 4 && MAXC <= 6;
    // Can the row source / tile be accessed with vectors?
    const bool vsrc = FIRST ? p.vec_x != 0 : (p.resident != 0 || p.vec_y != 0);
    const bool vdst = p.resident != 0 || p.vec_y != 0;
    T cacc[MAXC][VEC];
#pragma unroll
    for (int s = 0; s < MAXC; ++s)
#pragma unroll
      for (int v = 0; v < VEC; ++v) cacc[s][v] = T(0);
    T cur[MAXC][VEC], nxt[MAXC][VEC];
    auto load_row = [&](int i, T (&dst)[MAXC][VEC]) {
#pragma unroll
      for (int s = 0; s < MAXC; ++s) {
        const int j0 = (lane + 32 * s) * VEC;
        if (j0 < nc) {
          if (FIRST) {
            TIn xv[VEC];
            vec_load<TIn, VEC>(p.X + (size_t)(r0 + i) * p.ldx + c0 + j0, vsrc, nc - j0, xv);
#pragma unroll
            for (int v = 0; v < VEC; ++v) dst[s][v] = (T)xv[v];
          } else {
            vec_load<T, VEC>(tile + (size_t)i * ldt + j0, vsrc, nc - j0, dst[s]);
          }
        }
      }
    };
    // One row: the pass of eq. 7 (or step 1) on its groups; returns this
    // lane's part of the row sum.
    auto do_row = [&](int i, T (&src)[MAXC][VEC]) {
      T* row = tile + (size_t)i * ldt;
      const T ai = FIRST ? T(0) : addx(arow[i], cS, one);
      T racc = T(0);
#pragma unroll
      for (int s = 0; s < MAXC; ++s) {
        const int j0 = (lane + 32 * s) * VEC;
        if (j0 < nc) {
          T bv[VEC];
          if (!FIRST) vec_load<T, VEC>(bcol + j0, true, nc - j0, bv);
          T y[VEC];
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            if (FIRST)
              y[v] = p.mode == 0 ? src[s][v] * scale : src[s][v];
            else
              y[v] = relu(subx(addx(src[s][v], ai, one), bv[v], one));
            if (j0 + v >= nc) y[v] = T(0);
            racc = addx(racc, y[v], one);
            cacc[s][v] = addx(cacc[s][v], y[v], one);
          }
          vec_store<T, VEC>(row + j0, vdst, nc - j0, y);
        }
      }
      return racc;
    };
    if constexpr (sizeof(T) == 8 && MAXC <= 6) {
      // FP64: row sums of 8 rows at a time with one transposed reduction
      // (the 12-group variant keeps the per-row reduction: its registers are
      // already taken by the groups).
      for (int ib = warp; ib < nr; ib += 8 * kSdsnWarps) {
        T rb[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int iu = ib + u * kSdsnWarps;
          rb[u] = T(0);
          if (iu < nr) {
            load_row(iu, cur);
            rb[u] = do_row(iu, cur);
          }
        }
        const T rs = transpose_reduce8(rb, lane);
        const int ir = ib + transpose_index8(lane) * kSdsnWarps;
        if ((lane & 3) == 0 && ir < nr) rowsum[ir] = rs;
      }
    } else {
    int i = warp;
    if (i < nr) load_row(i, cur);
    for (; i < nr; i += kSdsnWarps) {
      const int inext = i + kSdsnWarps;
      if (PREF && inext < nr) load_row(inext, nxt);
      T* row = tile + (size_t)i * ldt;
      const T ai = FIRST ? T(0) : addx(arow[i], cS, one);
      T racc = T(0);
#pragma unroll
      for (int s = 0; s < MAXC; ++s) {
        const int j0 = (lane + 32 * s) * VEC;
        if (j0 < nc) {
          T bv[VEC];
          if (!FIRST) vec_load<T, VEC>(bcol + j0, true, nc - j0, bv);
          T y[VEC];
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            if (FIRST)
              y[v] = p.mode == 0 ? cur[s][v] * scale : cur[s][v];
            else
              y[v] = relu(subx(addx(cur[s][v], ai, one), bv[v], one));
            if (j0 + v >= nc) y[v] = T(0);
            racc = addx(racc, y[v], one);
            cacc[s][v] = addx(cacc[s][v], y[v], one);
          }
          vec_store<T, VEC>(row + j0, vdst, nc - j0, y);
        }
      }
      racc = warp_sum(racc);
      if (lane == 0) rowsum[i] = racc;
      if (PREF) {
#pragma unroll
        for (int s = 0; s < MAXC; ++s)
#pragma unroll
          for (int v = 0; v < VEC; ++v) cur[s][v] = nxt[s][v];
      } else if (inext < nr) {
        load_row(inext, cur);
      }
    }
    }
#pragma unroll
    for (int s = 0; s < MAXC; ++s) {
      const int j0 = (lane + 32 * s) * VEC;
#pragma unroll
      for (int v = 0; v < VEC; ++v)
        if (j0 + v < nc) wacc[j0 + v] = cacc[s][v];  // zeros for warps that had no row
    }
  }
  __syncthreads();
  // A problem on one CTA keeps its sums on chip: the next sweep's row and
  // column terms and the total go straight to shared memory (the same values
  // the gather below would produce).  Otherwise they are published as
  // partials for the other CTAs.
  const bool local = nblk == 1;
  T* rp = p.rpart + ((size_t)wb * p.Q + bj) * p.n + r0;
  for (int i = tid; i < nr; i += kSdsnThreads) {
    if (local)
      arow[i] = inv_n_t - rowsum[i] * inv_n_t;
    else
      rp[i] = rowsum[i];
  }
  // Column sums: four threads per column add four warps' values each, then
  // combine with two shuffles (a fixed order).
  T* cp = p.cpart + ((size_t)wb * p.P + bi) * p.n + c0;
  for (int base = 0; base < nc; base += kSdsnThreads / 4) {
    const int j = base + (tid >> 2), part = tid & 3;
    T c = T(0);
    if (j < nc) {
#pragma unroll
      for (int w = part; w < kSdsnWarps; w += 4) c += colacc[w * p.tc + j];
    }
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    if (part == 0 && j < nc) {
      if (local)
        bcol[j] = c * inv_n_t;
      else
        cp[j] = c;
    }
  }
  if (warp == 0) {
    // Tile total for S: FP64 in the FP64 kernel; from the FP32 row sums in
    // one FP32 warp reduction (one conversion) in the FP32 kernel.
    if (sizeof(T) == 8) {
      double t = 0.0;
      for (int i = lane; i < nr; i += 32) t += (double)rowsum[i];
      t = warp_sum(t);
      if (lane == 0) {
        if (local)
          *s_total = t;
        else
          p.tpart[(size_t)wb * nblk + blk] = t;
      }
    } else {
      T t = T(0);
      for (int i = lane; i < nr; i += 32) t += rowsum[i];
      t = warp_sum(t);
      if (lane == 0) {
        if (local)
          *s_total = (double)t;
        else
          p.tpart[(size_t)wb * nblk + blk] = (double)t;
      }
    }
  }
}

// The whole SDSN of one problem on CTAs blk = 0 .. nblk-1 of its (sub)grid.
template <typename T, typename TIn, int MAXC>
__device__ __forceinline__ void sdsn_body(const SdsnK<T, TIn>& p, int blk, int nblk,
                                          unsigned char* smem) {
  __shared__ int s_flag, s_stop;
  __shared__ double s_g, s_total;
  __shared__ T s_cS;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bi = blk / p.Q, bj = blk % p.Q;
  const int r0 = bi * p.tr, c0 = bj * p.tc;
  const int nr = max(0, min(p.tr, p.n - r0)), nc = max(0, min(p.tc, p.n - c0));
  const unsigned nblocks = (unsigned)nblk;

  size_t off = 0;
  T* tile;
  int ldt;
  if (p.resident) {
    tile = reinterpret_cast<T*>(smem);
    ldt = p.tc;
    off += align16((size_t)p.tr * p.tc * sizeof(T));
  } else {
    tile = p.Y + (size_t)r0 * p.ldy + c0;
    ldt = p.ldy;
  }
  T* colacc = reinterpret_cast<T*>(smem + off);
  off += align16((size_t)kSdsnWarps * p.tc * sizeof(T));
  T* rowsum = reinterpret_cast<T*>(smem + off);
  off += align16((size_t)p.tr * sizeof(T));
  T* arow = reinterpret_cast<T*>(smem + off);
  off += align16((size_t)p.tr * sizeof(T));
  T* bcol = reinterpret_cast<T*>(smem + off);

  // Alg. 2 step 1.  Every block reads the same max, so a degenerate input
  // makes every block return before the first barrier.
  const double m = p.mode == 0 ? from_ordered_key(*p.xmax_key) : 1.0;
  const int max_sweeps = (p.gate != nullptr && p.gate->gamma <= p.gate_tol) ? 0 : p.max_sweeps;
  if (!(m > 0.0)) {
    if (blk == 0 && tid == 0) {
      p.stats->status = DEV_DEGENERATE;
      p.stats->sweeps = 0;
      p.stats->converged = 0;
      p.stats->gamma = INFINITY;
      p.stats->xmax = m;
    }
    return;
  }
  const double n_d = (double)p.n;
  const double inv_n = 1.0 / n_d;
  const double inv_n2 = inv_n * inv_n;
  const T inv_n_t = (T)inv_n;
  int* status = &p.stats->status;
  const T scale = (T)((p.theta / 2.0) / m);

  sdsn_pass<T, TIn, MAXC, true>(p, tile, ldt, colacc, rowsum, arow, bcol, nr, nc, r0, c0, bi, bj,
                                scale, 0, blk, nblk, T(0), inv_n_t, &s_total);
  unsigned epoch = 1;
  if (nblocks > 1) {
    if (!grid_sync_epoch(p.bar, epoch * nblocks, p.limit_ns, status, &s_flag)) return;
  } else {
    __syncthreads();
  }

  double g = INFINITY;
  int k = 0;
  while (true) {
    const int rb = k & 1;
    // One round trip: totals (warp 0), row partials, column partials.  The
    // scalars S, gamma, the stop test and S/n^2 are formed once, by lane 0 of
    // warp 0 (FP64 instructions are scarce on this GPU).
    if (warp == 0) {
      double s = 0.0;
      if (nblocks > 1) {
        for (unsigned t = lane; t < nblocks; t += 32) s += __ldcg(&p.tpart[(size_t)rb * nblocks + t]);
        s = warp_sum(s);
      } else {
        s = s_total;
      }
      if (lane == 0) {
        const double gk = s * inv_n - 1.0;
        s_g = gk;
        s_stop = (k > 0 || p.mode == 1) && gk <= p.gamma_tol;
        s_cS = (T)(s * inv_n2);
      }
    }
    for (int e = tid; e < (nblocks > 1 ? nr + nc : 0); e += kSdsnThreads) {
      const bool is_row = e < nr;
      const int idx = is_row ? e : e - nr;
      const int cnt = is_row ? p.Q : p.P;
      const T* src = is_row ? p.rpart + (size_t)rb * p.Q * p.n + r0 + idx
                            : p.cpart + (size_t)rb * p.P * p.n + c0 + idx;
      T v[kMaxGrid];
#pragma unroll
      for (int q = 0; q < kMaxGrid; ++q) v[q] = q < cnt ? __ldcg(src + (size_t)q * p.n) : T(0);
      T acc = T(0);
#pragma unroll
      for (int q = 0; q < kMaxGrid; ++q) acc += v[q];
      // a_i = 1/n + S/n^2 - r_i/n: the S term is added in the pass, once S
      // is known, so that no extra barrier is needed here.
      if (is_row)
        arow[idx] = inv_n_t - acc * inv_n_t;
      else
        bcol[idx] = acc * inv_n_t;
    }
    __syncthreads();
    if (k > 0 || p.mode == 1) g = s_g;
    if (s_stop) break;
    if (k >= max_sweeps) break;
    sdsn_pass<T, TIn, MAXC, false>(p, tile, ldt, colacc, rowsum, arow, bcol, nr, nc, r0, c0, bi,
                                   bj, scale, rb ^ 1, blk, nblk, s_cS, inv_n_t, &s_total);
    ++k;
    ++epoch;
    if (nblocks > 1) {
      if (!grid_sync_epoch(p.bar, epoch * nblocks, p.limit_ns, status, &s_flag)) return;
    } else {
      __syncthreads();
    }
  }

  if (p.resident) {
    constexpr int VEC = 16 / (int)sizeof(T);
    for (int i = warp; i < nr; i += kSdsnWarps) {
      T* dst = p.Y + (size_t)(r0 + i) * p.ldy + c0;
      const T* src = tile + (size_t)i * ldt;
      for (int j0 = lane * VEC; j0 < nc; j0 += 32 * VEC) {
        T v[VEC];
        vec_load<T, VEC>(src + j0, true, nc - j0, v);
        vec_store<T, VEC>(dst + j0, p.vec_y != 0, nc - j0, v);
      }
    }
  }
  if (blk == 0 && tid == 0) {
    p.stats->sweeps = k;
    p.stats->gamma = g;
    p.stats->converged = (g <= p.gamma_tol) ? 1 : 0;
    p.stats->xmax = m;
  }
}

template <typename T, typename TIn, int MAXC>
__global__ void __launch_bounds__(kSdsnThreads, 1) sdsn_kernel(SdsnK<T, TIn> p) {
  extern __shared__ __align__(16) unsigned char smem[];
  sdsn_body<T, TIn, MAXC>(p, blockIdx.x, gridDim.x, smem);
}

// Several independent SDSN problems in one cooperative launch: problem j owns
// CTAs [block0_j, block0_j + P_j Q_j) and its own partials and barrier, so
// each problem advances at its own pace and stops on its own gamma.
template <typename T, typename TIn, int MAXC>
__global__ void __launch_bounds__(kSdsnThreads, 1) sdsn_group_kernel(const SdsnK<T, TIn>* probs,
                                                                     int nprobs) {
  extern __shared__ __align__(16) unsigned char smem[];
  int lo = 0, hi = nprobs - 1;  // last problem with block0 <= blockIdx.x
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].block0 <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const SdsnK<T, TIn> p = probs[lo];
  const int nblk = p.P * p.Q;
  if ((int)blockIdx.x - p.block0 >= nblk) return;  // spare CTA (not part of any sub-grid)
  sdsn_body<T, TIn, MAXC>(p, (int)blockIdx.x - p.block0, nblk, smem);
}

// Grid shape: square P x Q with P*Q co-resident CTAs; a single CTA for small
// n (its barrier is then only the block's own).
void choose_grid(int n, int max_blocks, int& P, int& Q) {
  if (n <= 96) {
    P = Q = 1;
    return;
  }
  int g = 1;
  while ((g + 1) * (g + 1) <= max_blocks && g + 1 <= kMaxGrid) ++g;
  const int lim = (n + 47) / 48;  // tiles of at least ~48 x 48
  P = Q = g < lim ? g : lim;
}

// Tile width: ceil(n / Q) rounded up to whole 16-byte groups, so every
// tile starts on a group boundary.
template <typename T>
int tile_cols(int n, int Q) {
  constexpr int VEC = 16 / (int)sizeof(T);
  const int tc = (n + Q - 1) / Q;
  return (tc + VEC - 1) / VEC * VEC;
}

// 16-byte groups per lane for a tile width: 0 selects the scalar path.
template <typename T>
int vec_slots(int tc) {
  constexpr int VEC = 16 / (int)sizeof(T);
  const int sl = (tc + 32 * VEC - 1) / (32 * VEC);
  return sl <= 2 ? 2 : sl <= 6 ? 6 : sl <= 12 ? 12 : 0;
}

template <typename T, typename TIn>
void set_vec_flags(SdsnK<T, TIn>& k) {
  constexpr int VEC = 16 / (int)sizeof(T);
  k.vec_x = (reinterpret_cast<uintptr_t>(k.X) % (VEC * sizeof(TIn)) == 0) && (k.ldx % VEC == 0);
  k.vec_y = (reinterpret_cast<uintptr_t>(k.Y) % 16 == 0) && (k.ldy % VEC == 0);
}

template <typename T, typename TIn, int MAXC>
int launch_k(SdsnK<T, TIn>& k, int nblocks, size_t smem, int num_sms, cudaStream_t s) {
  // Occupancy does not depend on the (capped) smem size here.
  static DeviceCache cache;
  const int per_sm = device_cached(cache, [] {
    if (cudaFuncSetAttribute(sdsn_kernel<T, TIn, MAXC>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap) !=
        cudaSuccess)
      return -1;
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, sdsn_kernel<T, TIn, MAXC>, kSdsnThreads,
                                                      kSmemCap) != cudaSuccess)
      return -1;
    return v > 0 ? v : -1;
  });
  if (per_sm < 1 || nblocks > per_sm * num_sms) return -1;
  void* args[] = {&k};
  if (cudaLaunchCooperativeKernel((const void*)sdsn_kernel<T, TIn, MAXC>, dim3(nblocks),
                                  dim3(kSdsnThreads), args, smem, s) != cudaSuccess)
    return -1;
  return 1;
}

template <typename T, typename TIn>
int launch_sdsn_t(const SdsnLaunch& L, int num_sms, cudaStream_t s) {
  SdsnK<T, TIn> k{};
  int P, Q;
  choose_grid(L.n, num_sms, P, Q);
  const int tr = (L.n + P - 1) / P, tc = tile_cols<T>(L.n, Q);
  const bool resident = sdsn_smem_bytes<T>(tr, tc, true) <= kSmemCap;
  const size_t smem = sdsn_smem_bytes<T>(tr, tc, resident);
  if (smem > kSmemCap) return -1;  // tile rows too long even for streaming
  k.n = L.n;
  k.P = P;
  k.Q = Q;
  k.tr = tr;
  k.tc = tc;
  k.resident = resident ? 1 : 0;
  k.mode = L.mode;
  k.one = 1.0;
  k.X = static_cast<const TIn*>(L.X);
  k.ldx = L.ldx;
  k.Y = static_cast<T*>(L.Y);
  k.ldy = L.ldy;
  k.theta = L.theta;
  k.gamma_tol = L.gamma_tol;
  k.max_sweeps = L.max_sweeps;
  k.xmax_key = L.xmax_key;
  k.gate = L.gate;
  k.gate_tol = L.gate_tol;
  k.stats = L.stats;
  k.rpart = reinterpret_cast<T*>(L.partials);
  k.cpart = k.rpart + (size_t)2 * Q * L.n;
  k.tpart = L.partials + (size_t)2 * (P + Q) * L.n;  // past both partial arrays (<= 8-byte T)
  k.bar = L.barrier;
  k.limit_ns = L.limit_ns;
  if (cudaMemsetAsync(L.barrier, 0, sizeof(GridBarrier), s) != cudaSuccess) return -1;
  set_vec_flags(k);
  switch (vec_slots<T>(tc)) {
    case 2: return launch_k<T, TIn, 2>(k, P * Q, smem, num_sms, s);
    case 6: return launch_k<T, TIn, 6>(k, P * Q, smem, num_sms, s);
    case 12: return launch_k<T, TIn, 12>(k, P * Q, smem, num_sms, s);
    default: return launch_k<T, TIn, 0>(k, P * Q, smem, num_sms, s);
  }
}

static_assert(sizeof(SdsnK<double, double>) <= 256, "group descriptor slot");

template <typename T, typename TIn, int MAXC>
int launch_group_k(const SdsnK<T, TIn>* dprobs, int nprobs, int nblocks, size_t smem,
                   int num_sms, cudaStream_t s) {
  static DeviceCache cache;
  const int per_sm = device_cached(cache, [] {
    if (cudaFuncSetAttribute(sdsn_group_kernel<T, TIn, MAXC>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap) !=
        cudaSuccess)
      return -1;
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, sdsn_group_kernel<T, TIn, MAXC>,
                                                      kSdsnThreads, kSmemCap) != cudaSuccess)
      return -1;
    return v > 0 ? v : -1;
  });
  if (per_sm < 1 || nblocks > per_sm * num_sms) return -1;
  void* args[] = {(void*)&dprobs, &nprobs};
  if (cudaLaunchCooperativeKernel((const void*)sdsn_group_kernel<T, TIn, MAXC>, dim3(nblocks),
                                  dim3(kSdsnThreads), args, smem, s) != cudaSuccess)
    return -1;
  return 1;
}

template <typename T, typename TIn>
int launch_sdsn_group_t(const SdsnLaunch* L, int count, int max_blocks, void* ddesc,
                        size_t ddesc_bytes, int num_sms, cudaStream_t s) {
  if (count < 1 || count > max_blocks) return -1;
  // Sub-grid sides: each problem's preferred square grid, shrunk (largest
  // first) until all sub-grids fit in one co-resident wave.
  std::vector<int> g(count);
  int total = 0;
  for (int i = 0; i < count; ++i) {
    int P, Q;
    choose_grid(L[i].n, max_blocks, P, Q);
    g[i] = P;
    total += P * P;
  }
  while (total > max_blocks) {
    int w = 0;
    for (int i = 1; i < count; ++i)
      if (g[i] > g[w]) w = i;
    if (g[w] <= 1) return -1;
    total -= g[w] * g[w];
    --g[w];
    total += g[w] * g[w];
  }
  std::vector<SdsnK<T, TIn>> ks(count);
  size_t smem = 0;
  int slots = 0, block0 = 0;
  for (int i = 0; i < count; ++i) {
    SdsnK<T, TIn>& k = ks[i];
    const int P = g[i], Q = g[i];
    const int tr = (L[i].n + P - 1) / P, tc = tile_cols<T>(L[i].n, Q);
    const bool resident = sdsn_smem_bytes<T>(tr, tc, true) <= kSmemCap;
    const size_t sm = sdsn_smem_bytes<T>(tr, tc, resident);
    if (sm > kSmemCap) return -1;
    smem = sm > smem ? sm : smem;
    const int sl = vec_slots<T>(tc);
    slots = (sl == 0 || slots == 0 && i > 0) ? 0 : (sl > slots ? sl : slots);
    k.n = L[i].n;
    k.P = P;
    k.Q = Q;
    k.tr = tr;
    k.tc = tc;
    k.resident = resident ? 1 : 0;
    k.block0 = block0;
    block0 += P * Q;
    k.mode = L[i].mode;
    k.one = 1.0;
    k.X = static_cast<const TIn*>(L[i].X);
    k.ldx = L[i].ldx;
    k.Y = static_cast<T*>(L[i].Y);
    k.ldy = L[i].ldy;
    k.theta = L[i].theta;
    k.gamma_tol = L[i].gamma_tol;
    k.max_sweeps = L[i].max_sweeps;
    k.xmax_key = L[i].xmax_key;
    k.gate = L[i].gate;
    k.gate_tol = L[i].gate_tol;
    k.stats = L[i].stats;
    k.rpart = reinterpret_cast<T*>(L[i].partials);
    k.cpart = k.rpart + (size_t)2 * Q * L[i].n;
    k.tpart = L[i].partials + (size_t)2 * (P + Q) * L[i].n;
    k.bar = L[i].barrier;
    k.limit_ns = L[i].limit_ns;
    set_vec_flags(k);
    if (!L[i].barrier_zeroed &&
        cudaMemsetAsync(L[i].barrier, 0, sizeof(GridBarrier), s) != cudaSuccess)
      return -1;
  }
  if (count * sizeof(SdsnK<T, TIn>) > ddesc_bytes) return -1;
  if (cudaMemcpyAsync(ddesc, ks.data(), count * sizeof(SdsnK<T, TIn>), cudaMemcpyHostToDevice,
                      s) != cudaSuccess)
    return -1;
  const SdsnK<T, TIn>* dk = static_cast<const SdsnK<T, TIn>*>(ddesc);
  switch (slots) {
    case 2: return launch_group_k<T, TIn, 2>(dk, count, block0, smem, num_sms, s);
    case 6: return launch_group_k<T, TIn, 6>(dk, count, block0, smem, num_sms, s);
    case 12: return launch_group_k<T, TIn, 12>(dk, count, block0, smem, num_sms, s);
    default: return launch_group_k<T, TIn, 0>(dk, count, block0, smem, num_sms, s);
  }
}

}  // namespace

int launch_sdsn_group(const SdsnLaunch* L, int count, int max_blocks, void* ddesc,
                      size_t ddesc_bytes, int num_sms, cudaStream_t s) {
  if (count < 1) return 0;
  const bool in32 = L[0].in_fp32, out32 = L[0].out_fp32;
  for (int i = 1; i < count; ++i)
    if (L[i].in_fp32 != in32 || L[i].out_fp32 != out32) return -1;
  if (!in32 && !out32)
    return launch_sdsn_group_t<double, double>(L, count, max_blocks, ddesc, ddesc_bytes, num_sms, s);
  if (in32 && out32)
    return launch_sdsn_group_t<float, float>(L, count, max_blocks, ddesc, ddesc_bytes, num_sms, s);
  if (in32 && !out32)
    return launch_sdsn_group_t<double, float>(L, count, max_blocks, ddesc, ddesc_bytes, num_sms, s);
  return -1;
}

size_t sdsn_group_desc_bytes(int count) { return (size_t)count * 256; }

int sdsn_grid_blocks(int n, int num_sms) {
  int P, Q;
  choose_grid(n, num_sms, P, Q);
  return P * Q;
}

size_t sdsn_partials_elems(int n, int max_blocks) {
  int g = 1;
  while ((g + 1) * (g + 1) <= max_blocks && g + 1 <= kMaxGrid) ++g;
  return (size_t)4 * g * (size_t)n + 2 * (size_t)g * g + 64;
}

int launch_sdsn_fp64(const SdsnLaunch& L, int num_sms, cudaStream_t s) {
  return launch_sdsn_t<double, double>(L, num_sms, s);
}

int launch_sdsn(const SdsnLaunch& L, int num_sms, cudaStream_t s) {
  if (!L.in_fp32 && !L.out_fp32) return launch_sdsn_t<double, double>(L, num_sms, s);
  if (L.in_fp32 && L.out_fp32) {
    // 2 <= n <= 1024: the whole FP32 iterate in one cluster (no grid barrier).
    const int k = launch_sdsn_cluster(L, s);
    if (k != 0) return k;
    return launch_sdsn_t<float, float>(L, num_sms, s);
  }
  if (L.in_fp32 && !L.out_fp32) {
    // The mixed paths' FP64 polish of a small problem: one CTA of warps.
    const int k = launch_sdsn_polish_small(L, s);
    if (k != 0) return k;
    return launch_sdsn_t<double, float>(L, num_sms, s);
  }
  return -1;
}

}  // namespace fram
