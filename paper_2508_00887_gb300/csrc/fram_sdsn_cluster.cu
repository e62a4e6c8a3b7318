// SDSN (Alg. 2 of arXiv 2508.00887) in FP32 for 2 <= n <= 1024, held
// entirely on chip: for n <= 64 in the registers of one or two warps (the
// warp form, further down), above that by ONE thread-block cluster of s x s
// CTAs (s = 1, 2 or 4; 16 CTAs is a non-portable cluster size).  The mixed
// paths' FP64 polish of n <= 64 also runs here, in a warp form of its own.
//
//   step 1   Y = (theta/2) X / max(X)
//   sweep    Y_ij <- max(0, Y_ij + 1/n + S/n^2 - r_i/n - c_j/n)      (eq. 7)
//   stop     gamma = sum(Y)/n - 1 <= gamma_tol, or max_sweeps sweeps
//
// Why a cluster: one sweep needs the row sums, column sums and total of the
// previous sweep, a global all-reduce.  Among co-resident CTAs of a grid that
// reduction goes through L2 -- a store becomes visible to another SM after
// about 0.37 us, and among 144 CTAs the exchange costs about 3 us per sweep,
// more than the sweep's arithmetic.  Within a cluster each CTA writes its
// partial sums straight into the shared memory of the CTAs that need them
// (st.async into distributed shared memory), and each CTA waits on its own
// mbarrier until every byte it expects has landed, so no sweep touches
// global memory and no sweep needs a cluster-wide barrier.
//
// Layout: CTA (bi, bj) of the s x s cluster owns the tr x tc tile at rows
// bi*tr, columns bj*tc (tc a multiple of 4).  16 warps; warp w owns tile
// rows w, w+16, w+32, ...; lane l owns the 16-byte column groups l and l+32
// (G = 2, tc <= 256) or l (G = 1).  The first RR rows of each warp are held
// in registers, the remaining ones in shared memory.  Padding columns carry
// b_j = +inf, so every sweep leaves them at 0 without a test per element.
//
// Per sweep: the pass updates the tile and accumulates per-lane row and
// column sums; row sums are reduced across each warp by a transposing
// shuffle tree, column sums across warps through shared memory, the tile
// total from the warps' row sums.  Each CTA then pushes its row partials to
// the s CTAs of its tile row, its column partials to the s CTAs of its tile
// column and its total to all s*s, into slots indexed by the sender and
// double-buffered by sweep parity, and waits on that parity's mbarrier for
// the bytes of all its peers.  It sums the slots in a fixed order: every CTA
// forms the same S and gamma, so all of them stop at the same sweep.
//
// Why two buffers suffice: every CTA sends its tile total to every other
// CTA, so a CTA that has received all totals of sweep t knows that every
// CTA has finished sweep t, and with it the reads of the sweep t - 1 slots
// and the wait on the sweep t - 1 phase of the mbarrier those slots share.
// Only then does it send its sweep t + 1 partials into them.
#include <math.h>
#include <stdint.h>

#include <vector>

#include "fram_internal.cuh"

namespace fram {

namespace {

constexpr int kCT = 512;           // threads per CTA
constexpr int kCW = kCT / 32;      // warps per CTA
constexpr int kMaxTile = 256;      // tr, tc <= 256
constexpr int kMaxRowsPerWarp = kMaxTile / kCW;  // 16

struct ClusterK {
  int n, s, tr, tc;
  int vec_x, vec_y;
  const float* X;
  int ldx;
  float* Y;
  int ldy;
  double theta, gamma_tol;
  int max_sweeps;
  const unsigned long long* xmax_key;
  SdsnStats* stats;
  uint64_t limit_ns;  // limit of each wait for the peers' partial sums
};

// Shared-memory layout (floats unless noted), fixed for a kernel variant.
// Tiles are padded to TCP = 128 G columns and kMaxTile rows: every lane owns
// G whole 16-byte groups and every warp 16 rows, so the sweep loop has no
// bounds tests.  Padding rows carry a_i = -inf and padding columns b_j =
// +inf; their entries therefore stay 0 and add nothing to any sum.
//   ts      [kCW * RS][TCP]     tile rows held in shared memory (RS = 16 - RR)
//   colacc  [kCW][TCP]          per-warp column sums
//   arow    [kMaxTile]          1/n - r_i/n (-inf on padding rows)
//   bcol    [TCP]               c_j/n (+inf on padding columns)
//   rrecv   [2][4][kMaxTile]    row partials by sweep parity and sender bj
//   crecv   [2][4][TCP]         column partials by parity and sender bi
//   wtot    [kCW]               per-warp totals
//   trecv   [2][16]             tile totals by parity and sender rank
template <int G, int RR>
struct SmemLayout {
  static constexpr int TCP = 128 * G;
  static constexpr int RS = kMaxRowsPerWarp - RR;
  static constexpr size_t ts = 0;
  static constexpr size_t colacc = ts + (size_t)kCW * RS * TCP * 4;
  static constexpr size_t arow = colacc + (size_t)kCW * TCP * 4;
  static constexpr size_t bcol = arow + (size_t)kMaxTile * 4;
  static constexpr size_t rrecv = bcol + (size_t)TCP * 4;
  static constexpr size_t crecv = rrecv + (size_t)2 * 4 * kMaxTile * 4;
  static constexpr size_t wtot = crecv + (size_t)2 * 4 * TCP * 4;
  static constexpr size_t trecv = wtot + (size_t)kCW * 4;
  static constexpr size_t bytes = trecv + 2 * 16 * 4;
};

// Two FP32 values in one 64-bit register (low word = lower address), and the
// packed FP32x2 arithmetic of sm_100+ (each lane of the pair rounded to
// nearest, exactly as two scalar operations): half the instructions per
// element, which bounds a sweep on the 16 SMs of one cluster.
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t pack2(float lo, float hi) {
  f2_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void unpack2(f2_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2_t add2(f2_t a, f2_t b) {
  f2_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t sub2(f2_t a, f2_t b) {
  f2_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t mul2(f2_t a, f2_t b) {
  f2_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// max(0, .) of both halves (P2 of eq. 7).
__device__ __forceinline__ f2_t relu2(f2_t v) {
  float lo, hi;
  unpack2(v, lo, hi);
  return pack2(fmaxf(lo, 0.f), fmaxf(hi, 0.f));
}
// The sweep of eq. 7 on one pair: max(0, (y + a) - b), then both sums.
__device__ __forceinline__ f2_t sweep2(f2_t y, f2_t aa, f2_t bb, f2_t& racc, f2_t& cacc) {
  const f2_t t = relu2(sub2(add2(y, aa), bb));
  racc = add2(racc, t);
  cacc = add2(cacc, t);
  return t;
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::
          : "memory");
}

// Address of the same shared-memory word in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t remote(const void* local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r)
               : "r"((uint32_t)__cvta_generic_to_shared(local)), "r"(rank));
  return r;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// The exchange's mbarriers: one arrival (the owner's, with the byte count it
// expects) plus the bytes of the peers' st.async stores.  A store may land
// before the owner arms the phase: the transaction count then runs negative
// until the owner's expect_tx brings it back.
__device__ __forceinline__ void mbar_init(uint64_t* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void mbar_arm(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
               "r"(bytes)
               : "memory");
}
// Acquire at cluster scope: the peers' st.async stores of the completed
// phase are visible to the waiting thread afterwards.
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of `parity` to complete, at most limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, uint64_t limit_ns) {
  const uint32_t bar = smem_addr(b);
  if (mbar_test(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (unsigned polls = 1;; ++polls) {
    if (mbar_test(bar, parity)) return true;
    if ((polls & 63u) == 0 && globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// Stores into CTA `rank`'s shared memory that complete on that CTA's
// mbarrier `bar` (both arguments are local addresses, mapped here).
__device__ __forceinline__ void push_f32x4(const void* local, float4 v, uint64_t* bar,
                                           uint32_t rank) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::
          "r"(remote(local, rank)),
      "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
      "r"(__float_as_uint(v.w)), "r"(remote(bar, rank))
      : "memory");
}
__device__ __forceinline__ void push_f32(const void* local, float v, uint64_t* bar, uint32_t rank) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(
                   remote(local, rank)),
               "r"(__float_as_uint(v)), "r"(remote(bar, rank))
               : "memory");
}

// Error-free sum of two floats (Knuth's TwoSum): a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Sum of v[0..15] over the 32 lanes of a warp, transposed: afterwards lane l
// holds the total of entry ((l >> 4) & 1) * 8 + ((l >> 3) & 1) * 4 +
// ((l >> 2) & 1) * 2 + ((l >> 1) & 1), and lanes l, l ^ 1 hold the same one.
// 16 shuffles instead of 80; the addition order is fixed.
template <typename T>
__device__ __forceinline__ T transpose_reduce16(T (&v)[16], int lane) {
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const bool hi = lane & 16;
    const T send = hi ? v[m] : v[m + 8];
    const T keep = hi ? v[m + 8] : v[m];
    v[m] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const bool hi = lane & 8;
    const T send = hi ? v[m] : v[m + 4];
    const T keep = hi ? v[m + 4] : v[m];
    v[m] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const bool hi = lane & 4;
    const T send = hi ? v[m] : v[m + 2];
    const T keep = hi ? v[m + 2] : v[m];
    v[m] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const bool hi = lane & 2;
    const T send = hi ? v[0] : v[1];
    const T keep = hi ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__device__ __forceinline__ int transpose_index16(int lane) {
  return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

template <int G, int RR>
__device__ __forceinline__ void sdsn_cluster_body(const ClusterK& p, unsigned char* smem) {
  using Lay = SmemLayout<G, RR>;
  constexpr int TCP = Lay::TCP;
  constexpr int RS = Lay::RS;
  __shared__ float s_S[2];  // S of the last gathered sweep as hi + lo (double-float)
  __shared__ float s_cS;    // S / n^2 for the next sweep
  __shared__ int s_stop;
  __shared__ int s_fail;    // a wait for the peers' partials ran out of time
  __shared__ uint64_t s_bar[2];  // exchange mbarriers, by sweep parity
  float* ts = reinterpret_cast<float*>(smem + Lay::ts);
  float* colacc = reinterpret_cast<float*>(smem + Lay::colacc);
  float* arow = reinterpret_cast<float*>(smem + Lay::arow);
  float* bcol = reinterpret_cast<float*>(smem + Lay::bcol);
  float* rrecv = reinterpret_cast<float*>(smem + Lay::rrecv);
  float* crecv = reinterpret_cast<float*>(smem + Lay::crecv);
  float* wtot = reinterpret_cast<float*>(smem + Lay::wtot);
  float* trecv = reinterpret_cast<float*>(smem + Lay::trecv);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int s = p.s;
  const uint32_t rank = s > 1 ? cluster_rank() : 0u;
  const int bi = (int)rank / s, bj = (int)rank % s;
  const int r0 = bi * p.tr, c0 = bj * p.tc;
  const int nr = max(0, min(p.tr, p.n - r0)), nc = max(0, min(p.tc, p.n - c0));
  // Partials travel in whole 16-byte groups; a tile row's CTAs share nr and
  // a tile column's share nc, so sender and receiver count the same groups.
  const int rg = (nr + 3) >> 2, cg = (nc + 3) >> 2;
  const uint32_t expect_bytes = (uint32_t)((s - 1) * 16 * (rg + cg) + 4 * (s * s - 1));

  // Alg. 2 step 1.  Every CTA reads the same max, so a degenerate input makes
  // all of them return before the first cluster barrier.
  const double m = from_ordered_key(*p.xmax_key);
  if (!(m > 0.0)) {
    if (rank == 0 && tid == 0) {
      p.stats->status = DEV_DEGENERATE;
      p.stats->sweeps = 0;
      p.stats->converged = 0;
      p.stats->gamma = INFINITY;
      p.stats->xmax = m;
    }
    return;
  }
  const double n_d = (double)p.n;
  const double inv_n = 1.0 / n_d, inv_n2 = inv_n * inv_n;
  const float inv_n_f = (float)inv_n, inv_n2_f = (float)inv_n2;
  const float scale = (float)((p.theta / 2.0) / m);
  // The stop test gamma = S/n - 1 <= gamma_tol, as S <= n (1 + gamma_tol),
  // with the threshold as a double-float; FP64 work stays out of the sweep
  // loop (FP64 instructions are scarce on this GPU).
  const double thr = n_d * (1.0 + p.gamma_tol);
  const float thr_hi = (float)thr, thr_lo = (float)(thr - (double)thr_hi);
  const f2_t zero2 = pack2(0.f, 0.f);
  const f2_t scale2 = pack2(scale, scale);

  // Padding terms, written once: gathers only ever write valid rows/columns.
  for (int i = nr + tid; i < kMaxTile; i += kCT) arow[i] = -INFINITY;
  for (int j = nc + tid; j < TCP; j += kCT) bcol[j] = INFINITY;

  f2_t y[RR][G][2];  // register rows: column pairs (j0, j0 + 1), (j0 + 2, j0 + 3)
  float racc[16];    // per-lane row sums
  f2_t cacc2[G][2];  // per-lane column sums
  float cS = 0.f;

  // Alg. 2 step 1 for one 16-byte group: (theta/2) X / max X, 0 outside the tile.
  auto load_x = [&](int i, int j0, f2_t& a, f2_t& b) {
    if (i >= nr) {
      a = b = zero2;
      return;
    }
    const float* xr = p.X + (size_t)(r0 + i) * p.ldx + c0 + j0;
    if (p.vec_x && j0 + 4 <= nc) {
      const ulonglong2 x = *reinterpret_cast<const ulonglong2*>(xr);
      a = mul2(x.x, scale2);
      b = mul2(x.y, scale2);
    } else {
      float t[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) t[v] = j0 + v < nc ? xr[v] * scale : 0.f;
      a = pack2(t[0], t[1]);
      b = pack2(t[2], t[3]);
    }
  };

  auto first_pass = [&]() {
#pragma unroll
    for (int g = 0; g < G; ++g) cacc2[g][0] = cacc2[g][1] = zero2;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int i = warp + kCW * r;
      f2_t rp = zero2;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int j0 = 4 * (lane + 32 * g);
        f2_t t[2];
        load_x(i, j0, t[0], t[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          rp = add2(rp, t[h]);
          cacc2[g][h] = add2(cacc2[g][h], t[h]);
          if (r < RR) y[r < RR ? r : 0][g][h] = t[h];
        }
        if (r >= RR)
          *reinterpret_cast<ulonglong2*>(ts + (size_t)(warp + kCW * (r - RR)) * TCP + j0) =
              make_ulonglong2(t[0], t[1]);
      }
      float lo, hi;
      unpack2(rp, lo, hi);
      racc[r] = lo + hi;
    }
  };

  // The fused P1 + P2 sweep (eq. 7) over the tile; no bounds tests.
  auto sweep_pass = [&]() {
#pragma unroll
    for (int g = 0; g < G; ++g) cacc2[g][0] = cacc2[g][1] = zero2;
    f2_t bb[G][2];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const ulonglong2 b = *reinterpret_cast<const ulonglong2*>(bcol + 4 * (lane + 32 * g));
      bb[g][0] = b.x;
      bb[g][1] = b.y;
    }
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      const float ai = arow[warp + kCW * r] + cS;
      const f2_t aa = pack2(ai, ai);
      f2_t rp = zero2;
#pragma unroll
      for (int g = 0; g < G; ++g)
#pragma unroll
        for (int h = 0; h < 2; ++h) y[r][g][h] = sweep2(y[r][g][h], aa, bb[g][h], rp, cacc2[g][h]);
      float lo, hi;
      unpack2(rp, lo, hi);
      racc[r] = lo + hi;
    }
    if constexpr (RS > 0) {
      // Shared-memory rows, software-pipelined: the next row's groups are
      // loaded before the current row is stored.
      const float* base = ts + (size_t)warp * TCP + 4 * lane;
      ulonglong2 cur[G], nxt[G];
#pragma unroll
      for (int g = 0; g < G; ++g) cur[g] = *reinterpret_cast<const ulonglong2*>(base + 128 * g);
#pragma unroll
      for (int q = 0; q < RS; ++q) {
        float* row = ts + (size_t)(warp + kCW * q) * TCP + 4 * lane;
        if (q + 1 < RS) {
#pragma unroll
          for (int g = 0; g < G; ++g)
            nxt[g] = *reinterpret_cast<const ulonglong2*>(row + (size_t)kCW * TCP + 128 * g);
        }
        const float ai = arow[warp + kCW * (RR + q)] + cS;
        const f2_t aa = pack2(ai, ai);
        f2_t rp = zero2;
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const f2_t t0 = sweep2(cur[g].x, aa, bb[g][0], rp, cacc2[g][0]);
          const f2_t t1 = sweep2(cur[g].y, aa, bb[g][1], rp, cacc2[g][1]);
          *reinterpret_cast<ulonglong2*>(row + 128 * g) = make_ulonglong2(t0, t1);
        }
        float lo, hi;
        unpack2(rp, lo, hi);
        racc[RR + q] = lo + hi;
#pragma unroll
        for (int g = 0; g < G; ++g) cur[g] = nxt[g];
      }
    }
  };

  // Reduce the pass's sums, keep them in this CTA's own slots of parity
  // buffer `par` and push them into the same slots of the peers that need
  // them; then wait until the peers' partials of this sweep have landed.
  // Returns false when that wait ran out of time.
  auto publish = [&](const int par, const int t) -> bool {
    if (s > 1 && tid == 0) mbar_arm(&s_bar[par], expect_bytes);
    float* rslot = rrecv + (size_t)(par * 4 + bj) * kMaxTile;
    float* cslot = crecv + (size_t)(par * 4 + bi) * TCP;
    const float rs = transpose_reduce16(racc, lane);
    const int ri = warp + kCW * transpose_index16(lane);
    const bool holder = (lane & 1) == 0 && ri < nr;
    if (holder) rslot[ri] = rs;
    const float wt = warp_sum(holder ? rs : 0.f);
    if (lane == 0) wtot[warp] = wt;
#pragma unroll
    for (int g = 0; g < G; ++g)
      *reinterpret_cast<ulonglong2*>(colacc + warp * TCP + 4 * (lane + 32 * g)) =
          make_ulonglong2(cacc2[g][0], cacc2[g][1]);
    __syncthreads();
    if (tid < TCP) {
      // Column tid's partial; lanes 4m..4m+3 hand theirs to lane 4m, which
      // pushes the group to the other CTAs of the tile column.
      float c = 0.f;
#pragma unroll
      for (int w = 0; w < kCW; ++w) c += colacc[w * TCP + tid];
      cslot[tid] = c;
      if (s > 1) {
        const float c1 = __shfl_down_sync(0xffffffffu, c, 1);
        const float c2 = __shfl_down_sync(0xffffffffu, c, 2);
        const float c3 = __shfl_down_sync(0xffffffffu, c, 3);
        if ((lane & 3) == 0 && (tid >> 2) < cg) {
          const float4 v = make_float4(c, c1, c2, c3);
          for (int q = 0; q < s; ++q)
            if (q != bi) push_f32x4(&cslot[tid], v, &s_bar[par], (uint32_t)(q * s + bj));
        }
      }
    } else if (tid < TCP + 32) {
      // The tile total: lane 0 keeps it, lanes 1 .. s*s - 1 push it.
      float tt = 0.f;
#pragma unroll
      for (int w = 0; w < kCW; ++w) tt += wtot[w];
      float* tslot = trecv + par * 16 + rank;
      if (lane == 0)
        *tslot = tt;
      else if (lane < s * s)
        push_f32(tslot, tt, &s_bar[par], (rank + (uint32_t)lane) % (uint32_t)(s * s));
    } else if (s > 1) {
      // Row groups to the other CTAs of the tile row: one group per thread.
      const int u = tid - (TCP + 32);
      if (u < (s - 1) * rg) {
        const int qi = u / rg, e0 = 4 * (u - qi * rg);
        const int q = qi < bj ? qi : qi + 1;
        push_f32x4(&rslot[e0], *reinterpret_cast<const float4*>(&rslot[e0]), &s_bar[par],
                   (uint32_t)(bi * s + q));
      }
    }
    __syncthreads();
    if (s == 1) return true;
    return mbar_wait(&s_bar[par], (uint32_t)((t >> 1) & 1), p.limit_ns);
  };

  // After the exchange: warp 0 forms S (from the s*s tile totals), gamma,
  // S/n^2 and the stop test; the other 15 warps form the next sweep's row
  // and column terms from the partials of their rows and columns, each
  // summed over the s senders in a fixed order.
  auto gather = [&](const int par, const int k) {
    if (warp == 0) {
      // S: the s*s tile totals summed as a double-float by a pairwise tree
      // over lanes in a fixed order (TwoSum at every node: exact up to the
      // rounding of the low parts, ~2^-48 relative).  A tree, not a chain:
      // the other warps wait for S at the next barrier.
      float hi = 0.f, lo = 0.f;
      if (lane < s * s) hi = trecv[par * 16 + lane];
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        if (o >= s * s) continue;  // uniform: s*s is 1, 4 or 16
        const float ohi = __shfl_down_sync(0xffffffffu, hi, o);
        const float olo = __shfl_down_sync(0xffffffffu, lo, o);
        float e;
        two_sum(hi, ohi, hi, e);
        lo = (lo + olo) + e;
      }
      {
        float e;
        two_sum(hi, lo, hi, e);
        lo = e;
      }
      if (lane == 0) {
        s_S[0] = hi;
        s_S[1] = lo;
        s_cS = hi * inv_n2_f + lo * inv_n2_f;
        const bool below = hi < thr_hi || (hi == thr_hi && lo <= thr_lo);
        s_stop = (k > 0 && below) ? 1 : 0;
      }
      return;
    }
    // Four consecutive entries per thread (rows [0, nr), then columns
    // [0, nc)), one 16-byte load from each of the s senders' slots; each
    // entry is summed in the same fixed order as one at a time.  The slots
    // are 16-byte aligned; entries past nr or nc are summed from stale words
    // and not stored.
    const int g = tid - 32;
    if (g < rg + cg) {
      const bool isrow = g < rg;
      const int e0 = 4 * (isrow ? g : g - rg);
      float4 v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q < s)
          v[q] = *reinterpret_cast<const float4*>(
              isrow ? &rrecv[(size_t)(par * 4 + q) * kMaxTile + e0]
                    : &crecv[(size_t)(par * 4 + q) * TCP + e0]);
      }
      const float acc[4] = {((v[0].x + v[1].x) + v[2].x) + v[3].x,
                            ((v[0].y + v[1].y) + v[2].y) + v[3].y,
                            ((v[0].z + v[1].z) + v[2].z) + v[3].z,
                            ((v[0].w + v[1].w) + v[2].w) + v[3].w};
      const int lim = isrow ? nr : nc;
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int e = e0 + h;
        if (e < lim) {
          if (isrow)
            arow[e] = inv_n_f - acc[h] * inv_n_f;
          else
            bcol[e] = acc[h] * inv_n_f;
        }
      }
    }
  };

  // The mbarriers must be initialised, and the initialisation visible to
  // the peers, before the first push.
  if (tid == 0) {
    s_fail = 0;
    mbar_init(&s_bar[0]);
    mbar_init(&s_bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (s > 1) cluster_sync(); else __syncthreads();

  first_pass();
  if (!publish(0, 0)) s_fail = 1;
  gather(0, 0);
  __syncthreads();
  int k = 0;
  while (true) {
    if (s_stop || s_fail || k >= p.max_sweeps) break;
    cS = s_cS;
    sweep_pass();
    ++k;
    if (!publish(k & 1, k)) s_fail = 1;
    gather(k & 1, k);
    __syncthreads();
  }
  if (s_fail && tid == 0) atomicCAS(&p.stats->status, DEV_OK, DEV_TIMEOUT);
  // No CTA leaves while a peer may still push into its shared memory.
  if (s > 1) cluster_sync();

  // Store the tile.
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int i = warp + kCW * r;
    if (i >= nr) continue;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int j0 = 4 * (lane + 32 * g);
      if (j0 >= nc) continue;
      ulonglong2 t;
      if (r < RR) {
        t.x = y[r < RR ? r : 0][g][0];
        t.y = y[r < RR ? r : 0][g][1];
      } else {
        t = *reinterpret_cast<const ulonglong2*>(ts + (size_t)(warp + kCW * (r - RR)) * TCP + j0);
      }
      float* yr = p.Y + (size_t)(r0 + i) * p.ldy + c0 + j0;
      if (p.vec_y && j0 + 4 <= nc) {
        *reinterpret_cast<ulonglong2*>(yr) = t;
      } else {
        float f[4];
        unpack2(t.x, f[0], f[1]);
        unpack2(t.y, f[2], f[3]);
#pragma unroll
        for (int vv = 0; vv < 4; ++vv)
          if (j0 + vv < nc) yr[vv] = f[vv];
      }
    }
  }
  if (rank == 0 && tid == 0) {
    const double g = k > 0 ? ((double)s_S[0] + (double)s_S[1]) * inv_n - 1.0 : INFINITY;
    p.stats->sweeps = k;
    p.stats->gamma = g;
    p.stats->converged = (g <= p.gamma_tol) ? 1 : 0;
    p.stats->xmax = m;
  }
}

template <int G, int RR>
__global__ void __launch_bounds__(kCT, 1) sdsn_cluster_kernel(const __grid_constant__ ClusterK p) {
  extern __shared__ __align__(16) unsigned char smem[];
  sdsn_cluster_body<G, RR>(p, smem);
}

// Many independent problems of one cluster shape in one launch: cluster c
// solves problem c.  Clusters never wait on one another, so the launch needs
// no co-residency and any number of problems fit.
template <int G, int RR>
__global__ void __launch_bounds__(kCT, 1) sdsn_cluster_group_kernel(const ClusterK* probs) {
  extern __shared__ __align__(16) unsigned char smem[];
  // By reference: fields are read from the descriptor array where used
  // instead of occupying registers for the whole launch.
  const ClusterK& p = probs[blockIdx.x / (unsigned)(probs[0].s * probs[0].s)];
  sdsn_cluster_body<G, RR>(p, smem);
}

// ---------------------------------------------------------------------------
// Small problems, 2 <= n <= 64: the warp form.  NC warps of 32 threads; warp
// w owns rows 32w .. 32w + 31 and lane l owns columns l + 32c (c < NC), so
// the whole iterate stays in the lanes' registers.  A sweep forms each row's
// sum with one transposed shuffle tree over the warp's 32 rows and each
// column's sum in the lane that owns it.  With two warps the two column
// halves meet in shared memory behind one 64-thread barrier, double-buffered
// by sweep parity: that is the sweep's only barrier.  Every lane forms S (a
// double-float tree over the column sums), gamma and the stop test itself,
// with the same operations, so all lanes take the same branch.
// ---------------------------------------------------------------------------

// Sum of v[0..31] over the 32 lanes, transposed: afterwards lane l holds the
// total of entry l.  31 shuffles, in a fixed order.  (Arithmetic of the warp
// form is written with _rn intrinsics so that no two kernels built from it
// can differ by a contraction into FMA: the grouped launch must reproduce
// the solo one bit for bit.)
__device__ __forceinline__ float transpose_reduce32(float (&v)[32], int lane) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool hi = lane & h;
#pragma unroll
    for (int m = 0; m < h; ++m) {
      const float send = hi ? v[m] : v[m + h];
      const float keep = hi ? v[m + h] : v[m];
      v[m] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  return v[0];
}

template <int NC>
__device__ __forceinline__ void sdsn_warp_body(const ClusterK& p) {
  __shared__ float s_a[NC][32];               // 1/n - r_i/n of each warp's rows
  __shared__ float s_colp[2][NC][32 * NC];    // column partials by parity and warp
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = p.n, r0 = 32 * w;

  // Alg. 2 step 1 (every thread reads the same max).
  const double m = from_ordered_key(*p.xmax_key);
  if (!(m > 0.0)) {
    if (threadIdx.x == 0) {
      p.stats->status = DEV_DEGENERATE;
      p.stats->sweeps = 0;
      p.stats->converged = 0;
      p.stats->gamma = INFINITY;
      p.stats->xmax = m;
    }
    return;
  }
  const double n_d = (double)n;
  const double inv_n = 1.0 / n_d;
  const float inv_n_f = (float)inv_n, inv_n2_f = (float)(inv_n * inv_n);
  const float scale = (float)((p.theta / 2.0) / m);
  const double thr = n_d * (1.0 + p.gamma_tol);
  const float thr_hi = (float)thr, thr_lo = (float)(thr - (double)thr_hi);

  float y[32][NC];  // rows r0 + r, columns lane + 32c
  float rp[32];     // this lane's part of each row sum
  float cacc[NC];   // this lane's column sums
  float bb[NC];     // c_j/n (+inf on padding columns)
  float cS = 0.f, S_hi = 0.f, S_lo = 0.f;

#pragma unroll
  for (int c = 0; c < NC; ++c) cacc[c] = 0.f;
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const int i = r0 + r;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int j = lane + 32 * c;
      const float v = (i < n && j < n) ? __fmul_rn(p.X[(size_t)i * p.ldx + j], scale) : 0.f;
      y[r][c] = v;
      rp[r] = c == 0 ? v : __fadd_rn(rp[r], v);
      cacc[c] = __fadd_rn(cacc[c], v);
    }
  }

  // The sums of the pass just made: the next sweep's a_i (in s_a) and b_j,
  // S/n^2, and the stop test after sweep k.
  auto exchange = [&](const int par, const int k) -> bool {
    // Column totals first: the barrier's wait then overlaps nothing that
    // matters, and the row tree below is independent of the S tree, so the
    // two interleave.
    float ct[NC];
    if constexpr (NC == 1) {
      ct[0] = cacc[0];
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) s_colp[par][w][lane + 32 * c] = cacc[c];
      __syncthreads();
#pragma unroll
      for (int c = 0; c < NC; ++c)
        ct[c] = __fadd_rn(s_colp[par][0][lane + 32 * c], s_colp[par][1][lane + 32 * c]);
    }
    const float rs = transpose_reduce32(rp, lane);  // row r0 + lane
#pragma unroll
    for (int c = 0; c < NC; ++c) bb[c] = lane + 32 * c < n ? __fmul_rn(ct[c], inv_n_f) : INFINITY;
    __syncwarp();
    s_a[w][lane] = r0 + lane < n ? __fmaf_rn(-rs, inv_n_f, inv_n_f) : -INFINITY;
    __syncwarp();
    // S over all columns: a pairwise double-float butterfly.  TwoSum is
    // exact, so lanes l and l ^ o form the same pair and every lane (of
    // either warp) ends with the same S.
    float hi = ct[0], lo = 0.f;
#pragma unroll
    for (int c = 1; c < NC; ++c) {
      float e;
      two_sum(hi, ct[c], hi, e);
      lo += e;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
      const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
      float e;
      two_sum(hi, ohi, hi, e);
      lo = (lo + olo) + e;
    }
    {
      float e;
      two_sum(hi, lo, hi, e);
      lo = e;
    }
    S_hi = hi;
    S_lo = lo;
    cS = __fmaf_rn(hi, inv_n2_f, __fmul_rn(lo, inv_n2_f));
    const bool below = hi < thr_hi || (hi == thr_hi && lo <= thr_lo);
    return k > 0 && below;
  };

  bool stop = exchange(0, 0);
  int k = 0;
  while (!stop && k < p.max_sweeps) {
    // The fused P1 + P2 sweep (eq. 7).
#pragma unroll
    for (int c = 0; c < NC; ++c) cacc[c] = 0.f;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const float ai = __fadd_rn(s_a[w][r], cS);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float t = fmaxf(__fsub_rn(__fadd_rn(y[r][c], ai), bb[c]), 0.f);
        y[r][c] = t;
        rp[r] = c == 0 ? t : __fadd_rn(rp[r], t);
        cacc[c] = __fadd_rn(cacc[c], t);
      }
    }
    ++k;
    stop = exchange(k & 1, k);
  }

#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const int i = r0 + r;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int j = lane + 32 * c;
      if (i < n && j < n) p.Y[(size_t)i * p.ldy + j] = y[r][c];
    }
  }
  if (threadIdx.x == 0) {
    const double g = k > 0 ? ((double)S_hi + (double)S_lo) * inv_n - 1.0 : INFINITY;
    p.stats->sweeps = k;
    p.stats->gamma = g;
    p.stats->converged = (g <= p.gamma_tol) ? 1 : 0;
    p.stats->xmax = m;
  }
}

template <int NC>
__global__ void __launch_bounds__(32 * NC) sdsn_warp_kernel(const __grid_constant__ ClusterK p) {
  sdsn_warp_body<NC>(p);
}

// Problem b of a group in CTA b: each CTA computes exactly what the solo
// launch computes for its problem.
template <int NC>
__global__ void __launch_bounds__(32 * NC) sdsn_warp_group_kernel(const ClusterK* probs) {
  sdsn_warp_body<NC>(probs[blockIdx.x]);
}

// ---------------------------------------------------------------------------
// The FP64 polish of the mixed paths for 2 <= n <= 64, in the same form: it
// continues from the FP32 result (Y0 = X, no scaling) and runs FP64 sweeps
// until gamma <= gamma_tol or max_sweeps, or none at all when the gate says
// the FP32 phase already met its tolerance.  2 NC warps of 16 rows each, so
// that all four schedulers' FP64 units work; lane l owns columns l + 32c.
// Row sums by one transposed shuffle tree per warp, column sums through
// shared memory behind one barrier per sweep (double-buffered by parity), S
// by a butterfly over the column sums, identical in every lane.
// ---------------------------------------------------------------------------
struct PolishK {
  int n;
  const float* X;
  int ldx;
  double* Y;
  int ldy;
  double gamma_tol;
  int max_sweeps;
  const SdsnStats* gate;
  double gate_tol;
  SdsnStats* stats;
  double one;  // 1.0, read at run time (add64)
};

// max(0, y) on the integer pipe: clear y if its sign bit is set.
__device__ __forceinline__ double relu_d(double y) {
  const long long b = __double_as_longlong(y);
  return __longlong_as_double(b & ~(b >> 63));
}

template <int NC>
__device__ __forceinline__ void polish_warp_body(const PolishK& p) {
  constexpr int W = 2 * NC;
  __shared__ double s_a[W][16];
  __shared__ double s_colp[2][W][32 * NC];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = p.n, r0 = 16 * w;
  const int max_sweeps =
      (p.gate != nullptr && p.gate->gamma <= p.gate_tol) ? 0 : p.max_sweeps;
  const double inv_n = 1.0 / (double)n, inv_n2 = inv_n * inv_n;
  const double one = p.one;

  double y[16][NC], rp[16], cacc[NC], bb[NC];
  double cS = 0.0, g = INFINITY;
#pragma unroll
  for (int c = 0; c < NC; ++c) cacc[c] = 0.0;
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int i = r0 + r;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int j = lane + 32 * c;
      const double v = (i < n && j < n) ? (double)p.X[(size_t)i * p.ldx + j] : 0.0;
      y[r][c] = v;
      rp[r] = c == 0 ? v : add64(rp[r], v, one);
      cacc[c] = add64(cacc[c], v, one);
    }
  }

  // Sums of the pass just made; returns the stop test (gamma of this pass;
  // as a continuation, the input itself may already meet the tolerance).
  auto exchange = [&](const int par) -> bool {
#pragma unroll
    for (int c = 0; c < NC; ++c) s_colp[par][w][lane + 32 * c] = cacc[c];
    __syncthreads();
    double ct[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double t = s_colp[par][0][lane + 32 * c];
#pragma unroll
      for (int q = 1; q < W; ++q) t = add64(t, s_colp[par][q][lane + 32 * c], one);
      ct[c] = t;
    }
    const double rs = transpose_reduce16(rp, lane);  // row r0 + (lane >> 1)
    double S = ct[0];
#pragma unroll
    for (int c = 1; c < NC; ++c) S = add64(S, ct[c], one);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) S = add64(S, __shfl_xor_sync(0xffffffffu, S, o), one);
#pragma unroll
    for (int c = 0; c < NC; ++c) bb[c] = lane + 32 * c < n ? __dmul_rn(ct[c], inv_n) : INFINITY;
    __syncwarp();
    const int ri = lane >> 1;
    if ((lane & 1) == 0) s_a[w][ri] = r0 + ri < n ? __fma_rn(-rs, inv_n, inv_n) : -INFINITY;
    __syncwarp();
    cS = __dmul_rn(S, inv_n2);
    g = __fma_rn(S, inv_n, -1.0);
    return g <= p.gamma_tol;
  };

  bool stop = exchange(0);
  int k = 0;
  while (!stop && k < max_sweeps) {
#pragma unroll
    for (int c = 0; c < NC; ++c) cacc[c] = 0.0;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const double ai = add64(s_a[w][r], cS, one);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const double t = relu_d(sub64(add64(y[r][c], ai, one), bb[c], one));
        y[r][c] = t;
        rp[r] = c == 0 ? t : add64(rp[r], t, one);
        cacc[c] = add64(cacc[c], t, one);
      }
    }
    ++k;
    stop = exchange(k & 1);
  }

#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int i = r0 + r;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int j = lane + 32 * c;
      if (i < n && j < n) p.Y[(size_t)i * p.ldy + j] = y[r][c];
    }
  }
  if (threadIdx.x == 0) {
    p.stats->sweeps = k;
    p.stats->gamma = g;
    p.stats->converged = (g <= p.gamma_tol) ? 1 : 0;
    p.stats->xmax = 1.0;
  }
}

template <int NC>
__global__ void __launch_bounds__(64 * NC) polish_warp_kernel(const __grid_constant__ PolishK p) {
  polish_warp_body<NC>(p);
}

template <int NC>
__global__ void __launch_bounds__(64 * NC) polish_warp_group_kernel(const PolishK* probs) {
  polish_warp_body<NC>(probs[blockIdx.x]);
}

// Warps (and columns per lane) of the warp form for n, 0 above 64.
int warp_form(int n) { return n <= 32 ? 1 : n <= 64 ? 2 : 0; }

bool polish_warp_applies(const SdsnLaunch& L) {
  return L.in_fp32 && !L.out_fp32 && L.mode == 1 && L.n >= 2 && L.n <= 64;
}

PolishK make_polish(const SdsnLaunch& L) {
  PolishK k{};
  k.n = L.n;
  k.X = static_cast<const float*>(L.X);
  k.ldx = L.ldx;
  k.Y = static_cast<double*>(L.Y);
  k.ldy = L.ldy;
  k.gamma_tol = L.gamma_tol;
  k.max_sweeps = L.max_sweeps;
  k.gate = L.gate;
  k.gate_tol = L.gate_tol;
  k.stats = L.stats;
  k.one = 1.0;
  return k;
}

int launch_warp_form(const ClusterK* dk, const ClusterK* hk, int count, cudaStream_t st) {
  const int nc = warp_form(hk[0].n);
  if (dk == nullptr) {
    if (nc == 1) sdsn_warp_kernel<1><<<1, 32, 0, st>>>(hk[0]);
    else sdsn_warp_kernel<2><<<1, 64, 0, st>>>(hk[0]);
  } else {
    if (nc == 1) sdsn_warp_group_kernel<1><<<count, 32, 0, st>>>(dk);
    else sdsn_warp_group_kernel<2><<<count, 64, 0, st>>>(dk);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// Cluster side s for n: one CTA up to 256, 2 x 2 up to 512, 4 x 4 up to 1024.
int cluster_side(int n) { return n <= 256 ? 1 : n <= 512 ? 2 : 4; }

// Fill the problem descriptor; false when this form does not apply.
bool make_cluster_problem(const SdsnLaunch& L, ClusterK& k) {
  if (!L.in_fp32 || !L.out_fp32 || L.mode != 0 || L.gate != nullptr) return false;
  if (L.n < 2 || L.n > 1024) return false;
  k = ClusterK{};
  k.n = L.n;
  k.s = cluster_side(L.n);
  k.tr = (L.n + k.s - 1) / k.s;
  k.tc = (k.tr + 3) / 4 * 4;
  if (k.tr > kMaxTile || k.tc > kMaxTile) return false;
  k.X = static_cast<const float*>(L.X);
  k.ldx = L.ldx;
  k.Y = static_cast<float*>(L.Y);
  k.ldy = L.ldy;
  k.vec_x = (reinterpret_cast<uintptr_t>(k.X) % 16 == 0) && (k.ldx % 4 == 0);
  k.vec_y = (reinterpret_cast<uintptr_t>(k.Y) % 16 == 0) && (k.ldy % 4 == 0);
  k.theta = L.theta;
  k.gamma_tol = L.gamma_tol;
  k.max_sweeps = L.max_sweeps;
  k.xmax_key = L.xmax_key;
  k.stats = L.stats;
  k.limit_ns = L.limit_ns;
  return true;
}

// Kernel attributes set, and a cluster of s*s CTAs with `smem` bytes each
// schedulable on this GPU (checked once per shape and device).
template <int G, int RR>
bool cluster_ready(int s, size_t smem) {
  static DeviceCache attr;
  if (device_cached(attr, [] {
        const void* f1 = (const void*)sdsn_cluster_kernel<G, RR>;
        const void* f2 = (const void*)sdsn_cluster_group_kernel<G, RR>;
        for (const void* f : {f1, f2}) {
          if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
                  cudaSuccess ||
              cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                  cudaSuccess) {
            cudaGetLastError();
            return -1;
          }
        }
        return 1;
      }) < 0)
    return false;
  static DeviceCache fits[3];
  const int si = s == 1 ? 0 : s == 2 ? 1 : 2;
  return device_cached(fits[si], [&] {
           cudaLaunchConfig_t cfg = {};
           cfg.gridDim = dim3((unsigned)(s * s));
           cfg.blockDim = dim3(kCT);
           cfg.dynamicSmemBytes = 200 * 1024;
           cudaLaunchAttribute at[1];
           at[0].id = cudaLaunchAttributeClusterDimension;
           at[0].val.clusterDim.x = (unsigned)(s * s);
           at[0].val.clusterDim.y = 1;
           at[0].val.clusterDim.z = 1;
           cfg.attrs = at;
           cfg.numAttrs = 1;
           int ncl = 0;
           if (cudaOccupancyMaxActiveClusters(&ncl, sdsn_cluster_kernel<G, RR>, &cfg) !=
               cudaSuccess) {
             cudaGetLastError();
             return -1;
           }
           return ncl > 0 ? 1 : -1;
         }) > 0 &&
         smem <= 200 * 1024;
}

template <int G, int RR>
int launch_cluster_t(const ClusterK* dk, const ClusterK* hk, int count, size_t smem,
                     cudaStream_t st) {
  const int s = hk[0].s;
  if (!cluster_ready<G, RR>(s, smem)) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(count * s * s));
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)(s * s);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = dk == nullptr ? cudaLaunchKernelEx(&cfg, sdsn_cluster_kernel<G, RR>, hk[0])
                                : cudaLaunchKernelEx(&cfg, sdsn_cluster_group_kernel<G, RR>, dk);
  return e == cudaSuccess ? 1 : -1;
}

size_t problem_smem(const ClusterK& k) {
  return k.tc <= 128 ? SmemLayout<1, 16>::bytes : SmemLayout<2, 8>::bytes;
}

}  // namespace

// FP32 SDSN of one problem in one cluster.  Returns 1 when launched, 0 when
// this form does not apply (size, shape, or the cluster is not schedulable:
// the caller then uses the grid form), -1 on a launch error.
int launch_sdsn_cluster(const SdsnLaunch& L, cudaStream_t st) {
  ClusterK k;
  if (!make_cluster_problem(L, k)) return 0;
  if (warp_form(k.n)) return launch_warp_form(nullptr, &k, 1, st);
  const size_t smem = problem_smem(k);
  if (k.tc <= 128) return launch_cluster_t<1, 16>(nullptr, &k, 1, smem, st);
  return launch_cluster_t<2, 8>(nullptr, &k, 1, smem, st);
}

// Cluster class of a problem (problems of one class can share a grouped
// launch): 1 + 3 * (wide tile) + (side index) for the cluster forms, 6 +
// (warps) for the warp form, 0 if neither applies.
int sdsn_cluster_class(const SdsnLaunch& L) {
  ClusterK k;
  if (!make_cluster_problem(L, k)) return 0;
  if (const int nw = warp_form(k.n)) return 6 + nw;
  const int si = k.s == 1 ? 0 : k.s == 2 ? 1 : 2;
  return 1 + 3 * (k.tc > 128 ? 1 : 0) + si;
}

// `count` problems of one cluster class in one launch (cluster c = problem c,
// each computing exactly what launch_sdsn_cluster computes for it).
// ddesc: device scratch of count * sdsn_cluster_desc_bytes().
int launch_sdsn_cluster_group(const SdsnLaunch* L, int count, void* ddesc, size_t ddesc_bytes,
                              cudaStream_t st) {
  if (count < 1) return 0;
  std::vector<ClusterK> ks(count);
  size_t smem = 0;
  for (int i = 0; i < count; ++i) {
    if (!make_cluster_problem(L[i], ks[i])) return -1;
    if (ks[i].s != ks[0].s || (ks[i].tc > 128) != (ks[0].tc > 128) ||
        warp_form(ks[i].n) != warp_form(ks[0].n))
      return -1;
    const size_t b = problem_smem(ks[i]);
    smem = b > smem ? b : smem;
  }
  if (count * sizeof(ClusterK) > ddesc_bytes) return -1;
  if (cudaMemcpyAsync(ddesc, ks.data(), count * sizeof(ClusterK), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return -1;
  const ClusterK* dk = static_cast<const ClusterK*>(ddesc);
  if (warp_form(ks[0].n)) return launch_warp_form(dk, ks.data(), count, st);
  const int r = ks[0].tc <= 128 ? launch_cluster_t<1, 16>(dk, ks.data(), count, smem, st)
                                : launch_cluster_t<2, 8>(dk, ks.data(), count, smem, st);
  return r == 0 ? -1 : r;
}

size_t sdsn_cluster_desc_bytes() { return sizeof(ClusterK); }

bool sdsn_polish_small_applies(const SdsnLaunch& L) { return polish_warp_applies(L); }

// FP64 polish of one problem with 2 <= n <= 64 in the warp form: 1 launched,
// 0 not applicable (the caller uses the grid form), -1 error.
int launch_sdsn_polish_small(const SdsnLaunch& L, cudaStream_t st) {
  if (!polish_warp_applies(L)) return 0;
  const PolishK k = make_polish(L);
  if (warp_form(k.n) == 1)
    polish_warp_kernel<1><<<1, 64, 0, st>>>(k);
  else
    polish_warp_kernel<2><<<1, 128, 0, st>>>(k);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// `count` such polishes in at most two launches (one per warp form), each
// CTA computing exactly what launch_sdsn_polish_small computes for its
// problem.  ddesc: device scratch of count * sdsn_cluster_desc_bytes().
int launch_sdsn_polish_small_group(const SdsnLaunch* L, int count, void* ddesc,
                                   size_t ddesc_bytes, cudaStream_t st) {
  if (count < 1) return 0;
  std::vector<PolishK> ks;
  ks.reserve(count);
  int n1 = 0;
  for (int form = 1; form <= 2; ++form)
    for (int i = 0; i < count; ++i) {
      if (!polish_warp_applies(L[i])) return -1;
      if (warp_form(L[i].n) != form) continue;
      ks.push_back(make_polish(L[i]));
      if (form == 1) ++n1;
    }
  if (ks.size() * sizeof(PolishK) > ddesc_bytes) return -1;
  if (cudaMemcpyAsync(ddesc, ks.data(), ks.size() * sizeof(PolishK), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return -1;
  const PolishK* dk = static_cast<const PolishK*>(ddesc);
  if (n1 > 0) polish_warp_group_kernel<1><<<n1, 64, 0, st>>>(dk);
  if (count - n1 > 0) polish_warp_group_kernel<2><<<count - n1, 128, 0, st>>>(dk + n1);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace fram
