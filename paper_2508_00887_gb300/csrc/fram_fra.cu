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
// order-preserving integer keys and each pass costs one FP64 add per
// element (plus one per active element): FP64 is scarce on this GPU.
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

__global__ void __launch_bounds__(kFraThreads) fra_kernel(FraK p) {
  extern __shared__ double fra_sm[];  // a_s[n], b_s[n]
  __shared__ double s_res[kFraWarps];
  __shared__ int s_flag;
  const int n = p.n;
  double* a_s = fra_sm;
  double* b_s = fra_sm + n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
      const double t = warp_threshold(p.Y + (size_t)i * p.ldy, b_s, n, k == 0, w0, &r);
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
      const double t = warp_threshold(p.Yt + (size_t)j * p.ldt, a_s, n, k == 0, w0, &r);
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

int launch_fra(double* Y, int ldy, double* Yt, int ldt, int n, const unsigned long long* xmax_key,
               double theta, double tol, int max_sweeps, double* ws, GridBarrier* bar,
               SdsnStats* stats, uint64_t limit_ns, int num_sms, cudaStream_t s) {
  const size_t smem = 2 * (size_t)n * sizeof(double);
  if (smem > 200 * 1024) return -1;  // the two multiplier vectors live in shared memory
  static int per_sm = 0;
  static size_t attr_smem = 0;
  if (attr_smem < smem) {
    if (cudaFuncSetAttribute(fra_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024) != cudaSuccess)
      return -1;
    attr_smem = 200 * 1024;
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fra_kernel, kFraThreads, smem) !=
          cudaSuccess ||
      occ < 1)
    return -1;
  per_sm = occ;
  // About one warp per row of the owned block; no more CTAs than rows.
  int grid = per_sm * num_sms;
  const int want = (n + kFraWarps - 1) / kFraWarps;
  if (grid > want) grid = want > num_sms ? want : (n < num_sms ? n : num_sms);
  if (grid < 1) grid = 1;
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
  if (cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s) != cudaSuccess) return -1;
  void* args[] = {&k};
  if (cudaLaunchCooperativeKernel((const void*)fra_kernel, dim3(grid), dim3(kFraThreads), args,
                                  smem, s) != cudaSuccess)
    return -1;
  return 1;
}

}  // namespace fram
