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
// accumulates the new tile's row sums, column sums and total, which the CTA
// publishes as partials (double-buffered by sweep parity).  After one grid
// barrier every CTA combines the Q row partials of its rows, the P column
// partials of its columns and the P*Q totals, always in the same order, so
// all CTAs agree bit for bit on S, on gamma and therefore on when to stop.
// When the tile fits in shared memory it stays there for all sweeps and
// global memory is touched only to load X and to store the result.
#include <math.h>

#include "fram_internal.cuh"

namespace fram {

namespace {

constexpr int kSdsnThreads = 512;
constexpr int kSdsnWarps = kSdsnThreads / 32;
constexpr size_t kSmemCap = 200 * 1024;

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

template <typename T>
struct SdsnK {
  int n, P, Q, tr, tc, resident;
  const T* X;
  int ldx;
  T* Y;
  int ldy;
  double theta, gamma_tol;
  int max_sweeps;
  const unsigned long long* xmax_key;
  SdsnStats* stats;
  double* rpart;  // [2][Q][n]
  double* cpart;  // [2][P][n]
  double* tpart;  // [2][P*Q]
  GridBarrier* bar;
  uint64_t limit_ns;
};

template <typename T>
__host__ __device__ inline size_t sdsn_smem_bytes(int tr, int tc, bool resident) {
  size_t b = 0;
  if (resident) b += align16((size_t)tr * tc * sizeof(T));
  b += align16((size_t)kSdsnWarps * tc * sizeof(T));  // column accumulators
  b += align16((size_t)tr * sizeof(double));           // row sums of the tile
  b += align16((size_t)tr * sizeof(T));                // a_i = 1/n + S/n^2 - r_i/n
  b += align16((size_t)tc * sizeof(T));                // b_j = c_j/n
  return b;
}

// One pass over the tile.  FIRST: Y = (theta/2) X / m.  Otherwise the fused
// P1+P2 sweep.  Both accumulate the new tile's sums and publish them into
// partial buffer `wb`.
template <typename T, bool FIRST>
__device__ __forceinline__ void sdsn_pass(const SdsnK<T>& p, T* tile, int ldt, T* colacc,
                                          double* rowsum, const T* arow, const T* bcol, int nr,
                                          int nc, int r0, int c0, int bi, int bj, double half_theta,
                                          double m, int wb) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < kSdsnWarps * p.tc; e += kSdsnThreads) colacc[e] = T(0);
  __syncthreads();
  T* cacc = colacc + warp * p.tc;
  for (int i = warp; i < nr; i += kSdsnWarps) {
    T* row = tile + (size_t)i * ldt;
    T racc = T(0);
    if (FIRST) {
      const T* xrow = p.X + (size_t)(r0 + i) * p.ldx + c0;
      for (int j = lane; j < nc; j += 32) {
        const T y = (T)(half_theta * ((double)xrow[j] / m));
        row[j] = y;
        racc += y;
        cacc[j] += y;
      }
    } else {
      const T ai = arow[i];
      for (int j = lane; j < nc; j += 32) {
        T y = (row[j] + ai) - bcol[j];
        y = y > T(0) ? y : T(0);
        row[j] = y;
        racc += y;
        cacc[j] += y;
      }
    }
    racc = warp_sum(racc);
    if (lane == 0) rowsum[i] = (double)racc;
  }
  __syncthreads();
  double* rp = p.rpart + ((size_t)wb * p.Q + bj) * p.n + r0;
  for (int i = tid; i < nr; i += kSdsnThreads) rp[i] = rowsum[i];
  double* cp = p.cpart + ((size_t)wb * p.P + bi) * p.n + c0;
  for (int j = tid; j < nc; j += kSdsnThreads) {
    double c = 0.0;
#pragma unroll 4
    for (int w = 0; w < kSdsnWarps; ++w) c += (double)colacc[w * p.tc + j];
    cp[j] = c;
  }
  if (warp == 0) {
    double t = 0.0;
    for (int i = lane; i < nr; i += 32) t += rowsum[i];
    t = warp_sum(t);
    if (lane == 0) p.tpart[(size_t)wb * gridDim.x + blockIdx.x] = t;
  }
}

template <typename T>
__global__ void __launch_bounds__(kSdsnThreads, 1) sdsn_kernel(SdsnK<T> p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag;
  __shared__ double s_S;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bi = blockIdx.x / p.Q, bj = blockIdx.x % p.Q;
  const int r0 = bi * p.tr, c0 = bj * p.tc;
  const int nr = max(0, min(p.tr, p.n - r0)), nc = max(0, min(p.tc, p.n - c0));
  const unsigned nblocks = gridDim.x;

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
  double* rowsum = reinterpret_cast<double*>(smem + off);
  off += align16((size_t)p.tr * sizeof(double));
  T* arow = reinterpret_cast<T*>(smem + off);
  off += align16((size_t)p.tr * sizeof(T));
  T* bcol = reinterpret_cast<T*>(smem + off);

  // Alg. 2 step 1.  Every block reads the same max, so a degenerate input
  // makes every block return before the first barrier.
  const double m = from_ordered_key(*p.xmax_key);
  if (!(m > 0.0)) {
    if (blockIdx.x == 0 && tid == 0) {
      p.stats->status = DEV_DEGENERATE;
      p.stats->sweeps = 0;
      p.stats->converged = 0;
      p.stats->gamma = INFINITY;
      p.stats->xmax = m;
    }
    return;
  }
  const double half_theta = p.theta / 2.0;
  const double n_d = (double)p.n;
  const double inv_n = 1.0 / n_d;
  const double n_sq = n_d * n_d;
  unsigned gen = 0;
  int* status = &p.stats->status;

  sdsn_pass<T, true>(p, tile, ldt, colacc, rowsum, arow, bcol, nr, nc, r0, c0, bi, bj, half_theta,
                     m, 0);
  if (!grid_sync(p.bar, nblocks, gen, p.limit_ns, status, &s_flag)) return;

  auto total = [&](int buf) {
    if (warp == 0) {
      double s = 0.0;
      for (unsigned t = lane; t < nblocks; t += 32) s += __ldcg(&p.tpart[(size_t)buf * nblocks + t]);
      s = warp_sum(s);
      if (lane == 0) s_S = s;
    }
    __syncthreads();
    return s_S;
  };

  double S = total(0);
  double g = INFINITY;
  int k = 0;
  while (k < p.max_sweeps) {
    const int rb = k & 1, wb = rb ^ 1;
    const double c1 = inv_n + S / n_sq;
    // Row sums of my rows (Q partials each) -> a_i; column sums -> b_j.
    for (int i = tid; i < nr; i += kSdsnThreads) {
      const double* rp = p.rpart + (size_t)rb * p.Q * p.n + r0 + i;
      double r = 0.0;
      for (int q = 0; q < p.Q; ++q) r += __ldcg(rp + (size_t)q * p.n);
      arow[i] = (T)(c1 - r / n_d);
    }
    for (int j = tid; j < nc; j += kSdsnThreads) {
      const double* cp = p.cpart + (size_t)rb * p.P * p.n + c0 + j;
      double c = 0.0;
      for (int q = 0; q < p.P; ++q) c += __ldcg(cp + (size_t)q * p.n);
      bcol[j] = (T)(c / n_d);
    }
    __syncthreads();
    sdsn_pass<T, false>(p, tile, ldt, colacc, rowsum, arow, bcol, nr, nc, r0, c0, bi, bj,
                        half_theta, m, wb);
    ++k;
    if (!grid_sync(p.bar, nblocks, gen, p.limit_ns, status, &s_flag)) return;
    S = total(wb);
    g = S / n_d - 1.0;
    if (g <= p.gamma_tol) break;
  }

  if (p.resident) {
    for (int i = warp; i < nr; i += kSdsnWarps) {
      T* dst = p.Y + (size_t)(r0 + i) * p.ldy + c0;
      const T* src = tile + (size_t)i * ldt;
      for (int j = lane; j < nc; j += 32) dst[j] = src[j];
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    p.stats->sweeps = k;
    p.stats->gamma = g;
    p.stats->converged = (g <= p.gamma_tol) ? 1 : 0;
    p.stats->xmax = m;
  }
}

// Grid shape: square-ish P x Q with P*Q co-resident CTAs; a single CTA for
// small n (no grid barrier traffic beyond its own block).
void choose_grid(int n, int max_blocks, int& P, int& Q) {
  if (n <= 96) {
    P = Q = 1;
    return;
  }
  int g = 1;
  while ((g + 1) * (g + 1) <= max_blocks) ++g;
  const int lim = (n + 47) / 48;  // tiles of at least ~48 x 48
  P = Q = g < lim ? g : lim;
}

template <typename T>
int launch_sdsn_t(const SdsnLaunch& L, int num_sms, cudaStream_t s) {
  SdsnK<T> k{};
  k.n = L.n;
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = 0;
  int P, Q;
  // Occupancy with the largest footprint we may request is at least 1/SM.
  choose_grid(L.n, num_sms, P, Q);
  int tr = (L.n + P - 1) / P, tc = (L.n + Q - 1) / Q;
  bool resident = sdsn_smem_bytes<T>(tr, tc, true) <= kSmemCap;
  size_t smem = sdsn_smem_bytes<T>(tr, tc, resident);
  if (smem > kSmemCap) return -1;  // tile rows too long even for streaming
  if (cudaFuncSetAttribute(sdsn_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sdsn_kernel<T>, kSdsnThreads, smem) !=
          cudaSuccess ||
      per_sm < 1)
    return -1;
  if (P * Q > per_sm * num_sms) return -1;
  k.P = P;
  k.Q = Q;
  k.tr = tr;
  k.tc = tc;
  k.resident = resident ? 1 : 0;
  k.X = static_cast<const T*>(L.X);
  k.ldx = L.ldx;
  k.Y = static_cast<T*>(L.Y);
  k.ldy = L.ldy;
  k.theta = L.theta;
  k.gamma_tol = L.gamma_tol;
  k.max_sweeps = L.max_sweeps;
  k.xmax_key = L.xmax_key;
  k.stats = L.stats;
  k.rpart = L.partials;
  k.cpart = k.rpart + (size_t)2 * Q * L.n;
  k.tpart = k.cpart + (size_t)2 * P * L.n;
  k.bar = L.barrier;
  k.limit_ns = L.limit_ns;
  if (cudaMemsetAsync(L.barrier, 0, sizeof(GridBarrier), s) != cudaSuccess) return -1;
  void* args[] = {&k};
  if (cudaLaunchCooperativeKernel((const void*)sdsn_kernel<T>, dim3(P * Q), dim3(kSdsnThreads),
                                  args, smem, s) != cudaSuccess)
    return -1;
  (void)dev;
  return 1;
}

}  // namespace

size_t sdsn_partials_elems(int n, int max_blocks) {
  int g = 1;
  while ((g + 1) * (g + 1) <= max_blocks) ++g;
  return (size_t)4 * g * (size_t)n + 2 * (size_t)g * g + 64;
}

int launch_sdsn_fp64(const SdsnLaunch& L, int num_sms, cudaStream_t s) {
  return launch_sdsn_t<double>(L, num_sms, s);
}

}  // namespace fram
