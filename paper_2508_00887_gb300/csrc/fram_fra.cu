// Exact FRA projection: a variant of Alg. 1 step 6 that computes the FRA
// solution of eq. 4 / Thm. 1 of arXiv 2508.00887 itself,
//
//   D = argmin over D_n of || D - Y0 ||_F,   Y0 = (theta/2) X / max(X),
//
// where the paper's SDSN (Alg. 2) runs alternating projections towards it.
// The KKT conditions give D = max(0, Y0 - a 1^T - 1 b^T) with multipliers
// a, b that make every row and column sum 1.  Block coordinate ascent on the
// concave dual alternates: with b fixed, each a_i solves
//
//   f_i(a) = sum_j max(0, Y0_ij - b_j - a) - 1 = 0,
//
// a convex, decreasing, piecewise-linear equation in a; then each b_j the
// same way on the columns with a fixed.
//
// GPU layout: one cooperative launch; CTA k owns the index block
// [k R, (k+1) R) of rows AND of columns (a transposed copy of Y0 makes a
// column a contiguous row), so every equation is solved by one warp without
// global communication.  Per sweep: row step, grid barrier, every CTA loads
// the new a; column step, barrier, loads the new b.
//
// One equation (a warp): Newton's method on f from the previous sweep's
// value (the first sweep starts from (sum z - 1)/n, left of the root).  For
// this convex decreasing f, a step from either side lands left of the root
// and later steps climb monotonically; the active set {z > a} then only
// shrinks, and when its size repeats the root is exact (Michelot's rule).
// The first evaluation, f_i at the previous value, is row i's residual at
// the current point, so the stop test costs nothing extra.  Comparisons use
// order-preserving integer keys.  FP64 is scarce on this GPU, so for n up to
// 2048 a warp forms z_j = Y0_ij - v_j once per equation and keeps only the
// keys of z in registers (the key is a bijection, so z comes back exactly);
// a Newton pass then costs integer compares plus one FP64 add per active
// element.  Larger n streams z again on every pass (one add per element).
//
// Over-relaxation: both steps move omega = 1.6 of the way to the solved
// value while the row residual keeps falling, 1 otherwise; once the residual
// is within tol the method switches to plain steps for good, and it stops at
// the first point whose row residual is within tol and whose b came from a
// plain column step (so the column sums are exact up to rounding).
#include <math.h>

#include "fram_internal.cuh"

namespace fram {

namespace {

constexpr int kFraThreads = 256;
constexpr int kFraWarps = kFraThreads / 32;
constexpr int kMaxNewton = 64;
constexpr double kOmega = 1.6;

struct FraK {
  int n;
  double* Y;    // in: X (ld-strided); then Y0 in place; out: D
  int ldy;
  double* Yt;   // scratch: Y0 transposed (ldt-strided)
  int ldt;
  const unsigned long long* xmax_key;
  double theta, tol;
  int max_sweeps;
  double* av;    // [2][n] row multipliers, double-buffered by sweep parity
  double* bv;    // [n] column multipliers
  double* rres;  // [2][grid] per-CTA row residuals
  GridBarrier* bar;
  SdsnStats* stats;
  uint64_t limit_ns;
};

// Root of sum_j max(0, y[j] - v[j] - a) = 1 over j < n, by one warp.  Cold
// start: a0 = (sum z - 1)/n.  Warm start from w0; then *res = |f(w0)|.
__device__ double warp_threshold(const double* __restrict__ y, const double* v, int n, bool cold,
                                 double w0, double* res) {
  const int lane = threadIdx.x & 31;
  double a;
  if (cold) {
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s += y[j] - v[j];
    s = warp_sum(s);
    a = (s - 1.0) / n;
  } else {
    a = w0;
  }
  int kprev = -1;
  for (int it = 0; it < kMaxNewton; ++it) {
    const unsigned long long ak = ordered_key(a);
    double S = 0.0;
    int k = 0;
    unsigned long long zmax = 0;
    for (int j = lane; j < n; j += 32) {
      const double z = y[j] - v[j];
      const unsigned long long zk = ordered_key(z);
      zmax = zk > zmax ? zk : zmax;
      if (zk > ak) {
        S += z;
        ++k;
      }
    }
    S = warp_sum(S);
    k = warp_sum(k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long oz = __shfl_xor_sync(0xffffffffu, zmax, o);
      zmax = oz > zmax ? oz : zmax;
    }
    if (it == 0 && !cold) *res = fabs(S - k * a - 1.0);
    if (k == kprev) break;  // the active set repeated: a is the root
    kprev = k;
    if (k == 0) {
      // every z <= a (a right of the root with no slope): restart left of it
      a = from_ordered_key(zmax) - 1.0;
      kprev = -1;
      continue;
    }
    a = (S - 1.0) / k;
  }
  return a;
}

// warp_threshold with the keys of z held in registers: C chunks of 32 per
// lane, n <= 32 C.  A pass over the registers also compacts the keys above
// the current a into the warp's list (ballot and popcount, integer work
// only); while a stays at or above the point the list was built at, the
// next passes read only the list, so a pass costs about (active / 32) FP64
// adds per lane instead of one per chunk.  A list that would overflow is
// not kept and the pass sums from the registers.
constexpr int kListCap = 256;

template <int C>
__device__ double warp_threshold_reg(const double* __restrict__ y, const double* v, int n,
                                     bool cold, double w0, double* res,
                                     unsigned long long* __restrict__ list,
                                     const double* __restrict__ rinv) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long zk[C];
  unsigned long long zmax = 0;  // below the key of every finite value
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int j = lane + 32 * c;
    zk[c] = 0;
    if (j < n) {
      const double z = y[j] - v[j];
      zk[c] = ordered_key(z);
      if (cold) s += z;
    }
    zmax = zk[c] > zmax ? zk[c] : zmax;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long oz = __shfl_xor_sync(0xffffffffu, zmax, o);
    zmax = oz > zmax ? oz : zmax;
  }
  double a = w0;
  if (cold) a = (warp_sum(s) - 1.0) * rinv[n];
  int m = -1;                   // list length (-1: no list)
  unsigned long long lkey = 0;  // key of the a the list was built at
  int kprev = -1;
  for (int it = 0; it < kMaxNewton; ++it) {
    const unsigned long long ak = ordered_key(a);
    double S = 0.0;
    int k = 0;
    if (m < 0 || ak < lkey) {
      // Pass over the registers, compacting {z > a} into the list.
      __syncwarp();  // every lane is done reading the old list
      int base = 0;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const bool act = zk[c] > ak;
        const unsigned msk = __ballot_sync(0xffffffffu, act);
        const int pos = base + __popc(msk & lt);
        if (act && pos < kListCap) list[pos] = zk[c];
        base += __popc(msk);
      }
      __syncwarp();
      lkey = ak;
      m = base <= kListCap ? base : -1;
      if (m < 0) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          if (zk[c] > ak) {
            S += from_ordered_key(zk[c]);
            ++k;
          }
        }
      } else {
        for (int t = lane; t < m; t += 32) {
          S += from_ordered_key(list[t]);
          ++k;
        }
      }
    } else {
      for (int t = lane; t < m; t += 32) {
        const unsigned long long q = list[t];
        if (q > ak) {
          S += from_ordered_key(q);
          ++k;
        }
      }
    }
    S = warp_sum(S);
    k = __reduce_add_sync(0xffffffffu, k);
    if (it == 0 && !cold) *res = fabs(S - k * a - 1.0);
    if (k == kprev) break;
    kprev = k;
    if (k == 0) {
      a = from_ordered_key(zmax) - 1.0;
      kprev = -1;
      continue;
    }
    a = (S - 1.0) * rinv[k];  // within an ulp of the quotient; no FP64 divide
  }
  return a;
}

// C = 0: stream z on every pass; C > 0: warp_threshold_reg<C>.
template <int C>
__device__ __forceinline__ double threshold(const double* __restrict__ y, const double* v, int n,
                                            bool cold, double w0, double* res,
                                            unsigned long long* list, const double* rinv) {
  if constexpr (C == 0)
    return warp_threshold(y, v, n, cold, w0, res);
  else
    return warp_threshold_reg<C>(y, v, n, cold, w0, res, list, rinv);
}

// Dynamic shared memory: a and b (n doubles each), then with C > 0 one
// key list per warp and the reciprocals 1/k, k = 0..n (FP64 division is a
// long instruction sequence on this GPU; each Newton step needs one).
template <int C>
size_t fra_smem_bytes(int n) {
  return 2 * (size_t)n * sizeof(double) +
         (C > 0 ? (size_t)kFraWarps * kListCap * sizeof(unsigned long long) +
                      (size_t)(n + 1) * sizeof(double)
                : 0);
}

template <int C>
__global__ void __launch_bounds__(kFraThreads) fra_kernel(FraK p) {
  extern __shared__ double fra_sm[];  // a_s[n], b_s[n], lists
  __shared__ double s_res[kFraWarps];
  __shared__ int s_flag;
  const int n = p.n;
  double* a_s = fra_sm;
  double* b_s = fra_sm + n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned long long* lists = reinterpret_cast<unsigned long long*>(fra_sm + 2 * (size_t)n);
  unsigned long long* list = lists + (size_t)warp * kListCap;
  double* rinv = reinterpret_cast<double*>(lists + (size_t)kFraWarps * kListCap);  // C > 0 only
  const int G = gridDim.x, blk = blockIdx.x;
  const int R = (n + G - 1) / G;
  const int i0 = min(n, blk * R), i1 = min(n, i0 + R);
  int* status = &p.stats->status;

  const double m = from_ordered_key(*p.xmax_key);
  if (!(m > 0.0)) {  // every block sees the same max: all return together
    if (blk == 0 && tid == 0) {
      p.stats->status = DEV_DEGENERATE;
      p.stats->sweeps = 0;
      p.stats->converged = 0;
      p.stats->gamma = INFINITY;
      p.stats->xmax = m;
    }
    return;
  }
  const double scale = (p.theta / 2.0) / m;
  unsigned epoch = 0;

  // Y0 in place (own rows), then its transpose (own columns).
  for (int i = i0 + warp; i < i1; i += kFraWarps) {
    double* row = p.Y + (size_t)i * p.ldy;
    for (int j = lane; j < n; j += 32) row[j] *= scale;
  }
  if (!grid_sync_epoch(p.bar, ++epoch * G, p.limit_ns, status, &s_flag)) return;
  for (int j = i0 + warp; j < i1; j += kFraWarps) {
    double* trow = p.Yt + (size_t)j * p.ldt;
    for (int i = lane; i < n; i += 32) trow[i] = __ldcg(p.Y + (size_t)i * p.ldy + j);
  }
  for (int j = tid; j < n; j += kFraThreads) b_s[j] = 0.0;
  if (C > 0)
    for (int q = tid; q <= n; q += kFraThreads) rinv[q] = q > 0 ? 1.0 / q : 0.0;
  __syncthreads();

  double omega = 1.0, prev_res = INFINITY, rowres = INFINITY;
  bool plain = false, col_plain = true;
  int k = 0;
  for (;; ++k) {
    // Row step: a_i from Y0 row i and b.
    double lres = 0.0;
    const double* a_cur = p.av + (size_t)((k + 1) & 1) * n;
    double* a_new = p.av + (size_t)(k & 1) * n;
    for (int i = i0 + warp; i < i1; i += kFraWarps) {
      double r = 0.0;
      const double w0 = k > 0 ? a_cur[i] : 0.0;
      const double t = threshold<C>(p.Y + (size_t)i * p.ldy, b_s, n, k == 0, w0, &r, list, rinv);
      if (lane == 0) a_new[i] = k > 0 ? w0 + omega * (t - w0) : t;
      lres = fmax(lres, r);
    }
    if (lane == 0) s_res[warp] = lres;
    __syncthreads();
    if (tid == 0) {
      double r = 0.0;
      for (int w = 0; w < kFraWarps; ++w) r = fmax(r, s_res[w]);
      p.rres[(size_t)(k & 1) * G + blk] = r;
    }
    if (!grid_sync_epoch(p.bar, ++epoch * G, p.limit_ns, status, &s_flag)) return;
    for (int j = tid; j < n; j += kFraThreads) a_s[j] = __ldcg(a_new + j);
    if (warp == 0) {
      double r = 0.0;
      for (int b = lane; b < G; b += 32) r = fmax(r, __ldcg(p.rres + (size_t)(k & 1) * G + b));
      r = warp_max(r);
      if (lane == 0) s_res[0] = r;
    }
    __syncthreads();
    rowres = k > 0 ? s_res[0] : INFINITY;  // residual at the previous point (a_{k-1}, b_{k-1})
    if (k > 0 && rowres <= p.tol && col_plain) break;  // that point is the answer
    if (k >= p.max_sweeps) break;
    if (rowres <= p.tol) plain = true;
    const double w_col = plain ? 1.0 : omega;
    __syncthreads();  // s_res is reused below

    // Column step: b_j from Y0 column j (a row of Yt) and the new a.
    for (int j = i0 + warp; j < i1; j += kFraWarps) {
      double r = 0.0;
      const double w0 = b_s[j];
      const double t = threshold<C>(p.Yt + (size_t)j * p.ldt, a_s, n, k == 0, w0, &r, list, rinv);
      if (lane == 0) p.bv[j] = k > 0 ? w0 + w_col * (t - w0) : t;
    }
    col_plain = k == 0 || w_col == 1.0;
    if (!grid_sync_epoch(p.bar, ++epoch * G, p.limit_ns, status, &s_flag)) return;
    for (int j = tid; j < n; j += kFraThreads) b_s[j] = __ldcg(p.bv + j);
    __syncthreads();
    omega = (!plain && rowres < prev_res) ? kOmega : 1.0;
    prev_res = rowres;
  }

  // Output at (a_{k-1}, b_{k-1}), the point whose row residual is rowres:
  // D = max(0, Y0 - a - b) for own rows.  (k == 0 cannot reach here.)
  const double* a_fin = p.av + (size_t)((k + 1) & 1) * n;
  for (int i = i0 + warp; i < i1; i += kFraWarps) {
    double* row = p.Y + (size_t)i * p.ldy;
    const double ai = a_fin[i];
    for (int j = lane; j < n; j += 32) row[j] = fmax(row[j] - ai - b_s[j], 0.0);
  }
  if (blk == 0 && tid == 0) {
    p.stats->sweeps = k;
    p.stats->converged = rowres <= p.tol ? 1 : 0;
    p.stats->gamma = rowres;
    p.stats->xmax = m;
  }
}

}  // namespace

size_t fra_workspace_elems(int n, int num_sms) { return 3 * (size_t)n + 2 * (size_t)num_sms; }

namespace {

template <int C>
int launch_fra_c(const FraK& k, int n, int num_sms, cudaStream_t s) {
  const size_t smem = fra_smem_bytes<C>(n);
  static DeviceCache attr;
  if (device_cached(attr, [] {
        return cudaFuncSetAttribute(fra_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    216 * 1024) == cudaSuccess
                   ? 1
                   : -1;
      }) < 0)
    return -1;
  // Occupancy depends on smem (n); query it for each launch size.
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fra_kernel<C>, kFraThreads, smem) !=
          cudaSuccess ||
      occ < 1)
    return -1;
  // About one warp per row of the owned block; no more CTAs than rows.
  int grid = occ * num_sms;
  const int want = (n + kFraWarps - 1) / kFraWarps;
  if (grid > want) grid = want > num_sms ? want : (n < num_sms ? n : num_sms);
  if (grid < 1) grid = 1;
  if (cudaMemsetAsync(k.bar, 0, sizeof(GridBarrier), s) != cudaSuccess) return -1;
  FraK kk = k;
  void* args[] = {&kk};
  if (cudaLaunchCooperativeKernel((const void*)fra_kernel<C>, dim3(grid), dim3(kFraThreads), args,
                                  smem, s) != cudaSuccess)
    return -1;
  return 1;
}

}  // namespace

int launch_fra(double* Y, int ldy, double* Yt, int ldt, int n, const unsigned long long* xmax_key,
               double theta, double tol, int max_sweeps, double* ws, GridBarrier* bar,
               SdsnStats* stats, uint64_t limit_ns, int num_sms, cudaStream_t s) {
  if (2 * (size_t)n * sizeof(double) > 200 * 1024) return -1;  // a and b live in shared memory
  FraK k{};
  k.n = n;
  k.Y = Y;
  k.ldy = ldy;
  k.Yt = Yt;
  k.ldt = ldt;
  k.xmax_key = xmax_key;
  k.theta = theta;
  k.tol = tol;
  k.max_sweeps = max_sweeps < 1 ? 1 : max_sweeps;
  k.av = ws;
  k.bv = ws + 2 * (size_t)n;
  k.rres = ws + 3 * (size_t)n;
  k.bar = bar;
  k.stats = stats;
  k.limit_ns = limit_ns;
  if (n <= 256) return launch_fra_c<8>(k, n, num_sms, s);
  if (n <= 512) return launch_fra_c<16>(k, n, num_sms, s);
  if (n <= 1024) return launch_fra_c<32>(k, n, num_sms, s);
  if (n <= 2048) return launch_fra_c<64>(k, n, num_sms, s);
  return launch_fra_c<0>(k, n, num_sms, s);
}

}  // namespace fram
