// Tensor-core gradient GEMMs of the mixed-precision path (Alg. 1 step 5,
// eq. 3 of arXiv 2508.00887; the paper runs this step in TF32):
//
//   C[i][j] = sum_k A[i][k] * Bop[j][k]      (both operands K-major)
//
// Used twice per outer iteration: T = A_s * N (Bop = N^T, written transposed
// by the update kernel) and X = T * B_s (+ lambda K) (Bop = B_s, symmetric).
// Inputs are BF16 (tcgen05.mma kind::f16) or TF32-rounded FP32 (kind::tf32);
// accumulation is FP32 in tensor memory.
//
// Persistent, warp-specialised: one CTA per SM walks its share of the
// 128 x BN output tiles (BN = 256 for large ld; 64 where 128 x 128 tiles
// would leave SMs idle, ld <= 1536; else 128) in a grouped order
// (8 row panels at a time, so concurrent CTAs share A and B strips in L2):
//   warp 0     TMA producer: 128-byte-swizzled A/B k-slices into a 4-stage
//              shared-memory ring (mbarrier full/empty pairs)
//   warp 1     allocates 2 x BN TMEM columns (two accumulators); one elected
//              thread issues the tcgen05.mma instructions (M=128, N=BN, K=16
//              or 8 each), commits each stage back to its empty barrier and
//              each finished tile to its accumulator's full barrier
//   warps 2-5  epilogue: tcgen05.ld of an accumulator (each warp reads its
//              own 32-lane quarter of TMEM), optional + lambda K, max(C), the
//              store in the output precision, then the accumulator is handed
//              back; the next tile's MMAs meanwhile fill the other one
// Every mbarrier wait is limited in time; on expiry the kernel records an
// error, drains its own TMA copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>

#include "fram_internal.cuh"
#include "fram_tc.h"

namespace fram {

namespace {

constexpr int BM = 128;
constexpr int ROW_BYTES = 128;              // one swizzle atom row per k-slice
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * ROW_BYTES;     // 16 KiB of A per stage
constexpr int GEMM_THREADS = 192;
constexpr int GROUP_M = 8;                  // row panels per rasterisation group

template <int BN>
struct Cfg {
  static constexpr int B_BYTES = BN * ROW_BYTES;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
  static constexpr int TMEM_COLS = 2 * BN;  // two accumulators
};

struct GemmArgs {
  int ld;                  // M = N = K = ld (multiple of 128)
  int n;                   // valid rows/cols for the K term and the max
  int kind;                // 0: BF16 operands, 1: TF32 operands
  int out_kind;            // 0: FP32, 1: BF16, 2: TF32-rounded FP32
  void* C;
  const double* Kmat;      // optional lambda K term (FP64, ld-strided)
  double lam;
  unsigned long long* cmax;  // optional ordered-key max over n x n
  int* err;
  uint64_t limit_ns;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of `parity` to complete, at most limit_ns.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// tcgen05 shared-memory matrix descriptor, K-major, 128-byte swizzle:
// start address >> 4 in bits [0,14), stride byte offset (8 rows x 128 B) >> 4
// in [32,46), descriptor version 1 in [46,48), layout SWIZZLE_128B (2) in [61,64).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((1024 >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor: FP32 accumulator (bits [4,6) = 1), A/B format in
// [7,10)/[10,13) (BF16 = 1, TF32 = 2), both K-major, N >> 3 in [17,23),
// M >> 4 in [24,29).
__host__ __device__ constexpr uint32_t instr_desc(int kind, int bn) {
  return (1u << 4) | ((kind == 0 ? 1u : 2u) << 7) | ((kind == 0 ? 1u : 2u) << 10) |
         ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accumulate) {
  if (KIND == 0) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Tile t of the grouped order -> (row panel, column panel).
__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int& tm, int& tn) {
  const int per_group = GROUP_M * tiles_n;
  const int g = t / per_group, r = t % per_group;
  const int first = g * GROUP_M;
  const int gm = min(GROUP_M, tiles_m - first);
  tm = first + r % gm;
  tn = r / gm;
}

template <int KIND, int BN>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   GemmArgs g) {
  using C = Cfg<BN>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ float s_max[4];
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024 - (raw & 1023)) & 1023);
  const uint32_t sbase = smem_u32(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * C::STAGE_BYTES);
  // full[STAGES], empty[STAGES], acc_full[2], acc_empty[2], drain
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * STAGES;
  const uint32_t accf0 = empty0 + 8 * STAGES, acce0 = accf0 + 16, drain = acce0 + 16;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  volatile int* s_fail = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int KELEMS = KIND == 0 ? 64 : 32;     // elements per 128-byte row
  constexpr int UMMA_K_BYTES = 32;                 // K=16 BF16 or K=8 TF32 per MMA
  const int nkb = g.ld / KELEMS;
  const int tiles_m = g.ld / BM, tiles_n = (g.ld + BN - 1) / BN;
  const int ntiles = tiles_m * tiles_n;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 4);  // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    *s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      long long issued = 0, it = 0;
      for (int t = blockIdx.x; t < ntiles && !*s_fail; t += gridDim.x) {
        int tm, tn;
        tile_coords(t, tiles_m, tiles_n, tm, tn);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          const uint32_t ph = (uint32_t)((it / STAGES) & 1);
          if (it >= STAGES && !mbar_wait(empty0 + 8 * s, ph ^ 1, g.limit_ns)) {
            *s_fail = 1;
            break;
          }
          if (*s_fail) break;
          const uint32_t fb = full0 + 8 * s;
          mbar_expect_tx(fb, C::STAGE_BYTES);
          tma_load_2d(sbase + s * C::STAGE_BYTES, &tmA, kb * KELEMS, tm * BM, fb);
          tma_load_2d(sbase + s * C::STAGE_BYTES + A_BYTES, &tmB, kb * KELEMS, tn * BN, fb);
          issued = it + 1;
        }
      }
      if (*s_fail) {
        // Drain: wait (limited) for our own copies; the last STAGES issued
        // may still be in flight whether or not they were consumed.
        for (long long k = issued > STAGES ? issued - STAGES : 0; k < issued; ++k)
          mbar_wait(full0 + 8 * (int)(k % STAGES), (uint32_t)((k / STAGES) & 1), g.limit_ns);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = instr_desc(KIND, BN);
      long long it = 0;
      int i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
        const int buf = i & 1;
        const uint32_t acc = tmem + (uint32_t)(buf * BN);
        if (i >= 2 && !mbar_wait(acce0 + 8 * buf, ((i >> 1) & 1) ^ 1, g.limit_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          if (!mbar_wait(full0 + 8 * s, (uint32_t)((it / STAGES) & 1), g.limit_ns) || *s_fail) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_addr = sbase + s * C::STAGE_BYTES;
          const uint32_t b_addr = a_addr + A_BYTES;
#pragma unroll
          for (int k = 0; k < ROW_BYTES / UMMA_K_BYTES; ++k) {
            mma<KIND>(acc, smem_desc_sw128(a_addr + k * UMMA_K_BYTES),
                      smem_desc_sw128(b_addr + k * UMMA_K_BYTES), idesc, (kb | k) != 0 ? 1u : 0u);
          }
          mma_commit(empty0 + 8 * s);
        }
        if (!ok) break;
        mma_commit(accf0 + 8 * buf);
      }
      if (!ok) {
        *s_fail = 1;
        // Let every MMA issued so far finish before TMEM is released.
        mma_commit(drain);
        mbar_wait(drain, 0, g.limit_ns);
      }
    }
  } else {
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    float lmax = -INFINITY;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int buf = i & 1;
      if (!mbar_wait(accf0 + 8 * buf, (uint32_t)((i >> 1) & 1), g.limit_ns) || *s_fail) {
        *s_fail = 1;
        break;
      }
      tc_fence_after();
      int tm, tn;
      tile_coords(t, tiles_m, tiles_n, tm, tn);
      const int row = tm * BM + q * 32 + lane;
      const uint32_t acc = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN);
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tmem_ld16(acc + c0, v);
        const int col0 = tn * BN + c0;
        if (col0 >= g.ld) break;  // past the last column (partial BN tile)
        if (g.Kmat != nullptr && row < g.n) {
          const double* kr = g.Kmat + (size_t)row * g.ld + col0;
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (col0 + e < g.n) v[e] += (float)(g.lam * kr[e]);
        }
        if (g.cmax != nullptr && row < g.n) {
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (col0 + e < g.n) lmax = fmaxf(lmax, v[e]);
        }
        if (g.out_kind == 1) {
          __nv_bfloat162 h[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) h[e] = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
          uint4* dst = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(g.C) +
                                                (size_t)row * g.ld + col0);
          dst[0] = *reinterpret_cast<uint4*>(&h[0]);
          dst[1] = *reinterpret_cast<uint4*>(&h[4]);
        } else {
          if (g.out_kind == 2) {
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] = to_tf32(v[e]);
          }
          float4* dst = reinterpret_cast<float4*>(static_cast<float*>(g.C) + (size_t)row * g.ld +
                                                  col0);
#pragma unroll
          for (int e = 0; e < 4; ++e) dst[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2],
                                                           v[4 * e + 3]);
        }
      }
      // Hand the accumulator back to the MMA warp.
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce0 + 8 * buf)
                                  : "memory");
    }
    if (g.cmax != nullptr) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
      if (lane == 0) s_max[warp - 2] = lmax;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::TMEM_COLS)
                 : "memory");
  }
  if (threadIdx.x == 0) {
    if (*s_fail) atomicExch(g.err, DEV_TIMEOUT);
    if (g.cmax != nullptr && !*s_fail) {
      const float m = fmaxf(fmaxf(s_max[0], s_max[1]), fmaxf(s_max[2], s_max[3]));
      if (m > -INFINITY) atomicMax(g.cmax, ordered_key((double)m));
    }
  }
}

// ---------------------------------------------------------------- grouped
// Many independent problems in ONE persistent launch (serving: every active
// request's gradient GEMM of a step).  Problem q has its own tensor maps, C,
// ld, n and max key; its 128 x 128 tiles occupy global tile indices
// [tile0_q, tile0_q + tiles_q), each in the grouped order a solo launch of
// that problem uses, and every tile is computed exactly as the solo launch
// computes it (same k order, same epilogue), so results do not depend on
// which other problems share the launch.
template <int KIND>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    gemm_tc_group_kernel(const GemmGroupProblem* __restrict__ probs, int nprob, int ntiles,
                         int out_kind, uint64_t limit_ns) {
  constexpr int BN = 128;
  using C = Cfg<BN>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024 - (raw & 1023)) & 1023);
  const uint32_t sbase = smem_u32(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * C::STAGE_BYTES);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * STAGES;
  const uint32_t accf0 = empty0 + 8 * STAGES, acce0 = accf0 + 16, drain = acce0 + 16;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  volatile int* s_fail = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int KELEMS = KIND == 0 ? 64 : 32;
  constexpr int UMMA_K_BYTES = 32;

  // Global tile t -> (problem, row panel, column panel, k blocks).
  auto resolve = [&](int t, int& q, int& tm, int& tn, int& nkb) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (probs[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    q = lo;
    const int tiles_m = probs[q].ld / BM;
    tile_coords(t - probs[q].tile0, tiles_m, tiles_m, tm, tn);
    nkb = probs[q].ld / KELEMS;
  };

  if (threadIdx.x == 0) {
    for (int st = 0; st < STAGES; ++st) {
      mbar_init(full0 + 8 * st, 1);
      mbar_init(empty0 + 8 * st, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 4);
    }
    mbar_init(drain, 1);
    *s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      long long issued = 0, it = 0;
      int fenced = -1;
      for (int t = blockIdx.x; t < ntiles && !*s_fail; t += gridDim.x) {
        int q, tm, tn, nkb;
        resolve(t, q, tm, tn, nkb);
        const CUtensorMap* ma = &probs[q].ma;
        const CUtensorMap* mb = &probs[q].mb;
        if (q != fenced) {
          // The descriptor array is rewritten between launches at the same
          // address: make the tensor-map proxy see the current maps.
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(ma)
                       : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mb)
                       : "memory");
          fenced = q;
        }
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int st = (int)(it % STAGES);
          const uint32_t ph = (uint32_t)((it / STAGES) & 1);
          if (it >= STAGES && !mbar_wait(empty0 + 8 * st, ph ^ 1, limit_ns)) {
            *s_fail = 1;
            break;
          }
          if (*s_fail) break;
          const uint32_t fb = full0 + 8 * st;
          mbar_expect_tx(fb, C::STAGE_BYTES);
          tma_load_2d(sbase + st * C::STAGE_BYTES, ma, kb * KELEMS, tm * BM, fb);
          tma_load_2d(sbase + st * C::STAGE_BYTES + A_BYTES, mb, kb * KELEMS, tn * BN, fb);
          issued = it + 1;
        }
      }
      if (*s_fail) {
        for (long long k = issued > STAGES ? issued - STAGES : 0; k < issued; ++k)
          mbar_wait(full0 + 8 * (int)(k % STAGES), (uint32_t)((k / STAGES) & 1), limit_ns);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = instr_desc(KIND, BN);
      long long it = 0;
      int i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
        int q, tm, tn, nkb;
        resolve(t, q, tm, tn, nkb);
        const int buf = i & 1;
        const uint32_t acc = tmem + (uint32_t)(buf * BN);
        if (i >= 2 && !mbar_wait(acce0 + 8 * buf, ((i >> 1) & 1) ^ 1, limit_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int st = (int)(it % STAGES);
          if (!mbar_wait(full0 + 8 * st, (uint32_t)((it / STAGES) & 1), limit_ns) || *s_fail) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_addr = sbase + st * C::STAGE_BYTES;
          const uint32_t b_addr = a_addr + A_BYTES;
#pragma unroll
          for (int k = 0; k < ROW_BYTES / UMMA_K_BYTES; ++k) {
            mma<KIND>(acc, smem_desc_sw128(a_addr + k * UMMA_K_BYTES),
                      smem_desc_sw128(b_addr + k * UMMA_K_BYTES), idesc, (kb | k) != 0 ? 1u : 0u);
          }
          mma_commit(empty0 + 8 * st);
        }
        if (!ok) break;
        mma_commit(accf0 + 8 * buf);
      }
      if (!ok) {
        *s_fail = 1;
        mma_commit(drain);
        mbar_wait(drain, 0, limit_ns);
      }
    }
  } else {
    const int qw = warp & 3;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int buf = i & 1;
      if (!mbar_wait(accf0 + 8 * buf, (uint32_t)((i >> 1) & 1), limit_ns) || *s_fail) {
        *s_fail = 1;
        break;
      }
      tc_fence_after();
      int q, tm, tn, nkb;
      resolve(t, q, tm, tn, nkb);
      const int ld = probs[q].ld, n = probs[q].n;
      void* Cq = probs[q].C;
      unsigned long long* cmax = probs[q].cmax;
      float lmax = -INFINITY;
      const int row = tm * BM + qw * 32 + lane;
      const uint32_t acc = tmem + ((uint32_t)(qw * 32) << 16) + (uint32_t)(buf * BN);
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tmem_ld16(acc + c0, v);
        const int col0 = tn * BN + c0;
        if (cmax != nullptr && row < n) {
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (col0 + e < n) lmax = fmaxf(lmax, v[e]);
        }
        if (out_kind == 1) {
          __nv_bfloat162 h[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) h[e] = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
          uint4* dst = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(Cq) +
                                                (size_t)row * ld + col0);
          dst[0] = *reinterpret_cast<uint4*>(&h[0]);
          dst[1] = *reinterpret_cast<uint4*>(&h[4]);
        } else {
          if (out_kind == 2) {
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] = to_tf32(v[e]);
          }
          float4* dst = reinterpret_cast<float4*>(static_cast<float*>(Cq) + (size_t)row * ld + col0);
#pragma unroll
          for (int e = 0; e < 4; ++e)
            dst[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce0 + 8 * buf)
                                  : "memory");
      if (cmax != nullptr) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        if (lane == 0 && lmax > -INFINITY) atomicMax(cmax, ordered_key((double)lmax));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::TMEM_COLS)
                 : "memory");
  }
  if (threadIdx.x == 0 && *s_fail) {
    // A wait expired: every problem of the launch is reported failed.
    for (int q = 0; q < nprob; ++q) atomicExch(probs[q].err, DEV_TIMEOUT);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (fn == nullptr) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool make_map(CUtensorMap* m, const void* ptr, int ld, int kind, int box_rows) {
  auto enc = get_encode();
  if (!enc) return false;
  const size_t es = kind == 0 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)ld};
  cuuint64_t strides[1] = {(cuuint64_t)ld * es};
  cuuint32_t box[2] = {(cuuint32_t)(ROW_BYTES / es), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                   2, const_cast<void*>(ptr), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

namespace {

int num_sms_cached() {
  static DeviceCache cache;
  return device_cached(cache, [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
      v = 1;
    return v;
  });
}

template <int KIND, int BN>
int launch_k(const CUtensorMap& ma, const CUtensorMap& mb, const GemmArgs& g, int ld,
             cudaStream_t s) {
  static DeviceCache attr;
  if (device_cached(attr, [] {
        return cudaFuncSetAttribute(gemm_tc_kernel<KIND, BN>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    Cfg<BN>::SMEM_BYTES) == cudaSuccess
                   ? 1
                   : -1;
      }) < 0)
    return -1;
  const int ntiles = (ld / BM) * ((ld + BN - 1) / BN);
  const int grid = ntiles < num_sms_cached() ? ntiles : num_sms_cached();
  gemm_tc_kernel<KIND, BN><<<grid, GEMM_THREADS, Cfg<BN>::SMEM_BYTES, s>>>(ma, mb, g);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace

bool make_group_problem(GemmGroupProblem* q, const void* A, const void* Bop, void* C, int ld,
                        int n, int kind, unsigned long long* cmax, int* err) {
  if (ld % 128 != 0 || ld <= 0) return false;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(Bop) |
       reinterpret_cast<uintptr_t>(C)) & 15)
    return false;
  if (!make_map(&q->ma, A, ld, kind, BM) || !make_map(&q->mb, Bop, ld, kind, 128)) return false;
  q->C = C;
  q->cmax = cmax;
  q->err = err;
  q->ld = ld;
  q->n = n;
  q->tile0 = 0;
  return true;
}

int launch_gemm_tc_group(GemmGroupProblem* hp, int count, int kind, int out_kind, void* dp,
                         size_t dp_bytes, uint64_t limit_ns, cudaStream_t s) {
  if (count < 1) return 0;
  if ((size_t)count * sizeof(GemmGroupProblem) > dp_bytes ||
      (reinterpret_cast<uintptr_t>(dp) & 63))
    return -1;
  int total = 0;
  for (int q = 0; q < count; ++q) {
    hp[q].tile0 = total;
    total += (hp[q].ld / BM) * (hp[q].ld / BM);
  }
  if (cudaMemcpyAsync(dp, hp, (size_t)count * sizeof(GemmGroupProblem), cudaMemcpyHostToDevice,
                      s) != cudaSuccess)
    return -1;
  static DeviceCache attr[2];
  if (device_cached(attr[kind], [kind] {
        const void* f = kind == 0 ? (const void*)gemm_tc_group_kernel<0>
                                  : (const void*)gemm_tc_group_kernel<1>;
        return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    Cfg<128>::SMEM_BYTES) == cudaSuccess
                   ? 1
                   : -1;
      }) < 0)
    return -1;
  const int grid = total < num_sms_cached() ? total : num_sms_cached();
  const GemmGroupProblem* d = static_cast<const GemmGroupProblem*>(dp);
  if (kind == 0)
    gemm_tc_group_kernel<0><<<grid, GEMM_THREADS, Cfg<128>::SMEM_BYTES, s>>>(d, count, total,
                                                                            out_kind, limit_ns);
  else
    gemm_tc_group_kernel<1><<<grid, GEMM_THREADS, Cfg<128>::SMEM_BYTES, s>>>(d, count, total,
                                                                            out_kind, limit_ns);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_gemm_tc(const void* A, const void* Bop, void* C, int ld, int n, int kind, int out_kind,
                   const double* Kmat, double lam, unsigned long long* cmax, int* err,
                   uint64_t limit_ns, cudaStream_t s) {
  if (ld % 128 != 0 || ld <= 0) return -1;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(Bop) |
       reinterpret_cast<uintptr_t>(C)) & 15)
    return -1;
  // 256-wide tiles once every CTA gets at least two of them; 64-wide ones
  // while 128-wide tiles would not give every SM one (twice the tiles, each
  // CTA streaming a narrower B strip).
  const int sms = num_sms_cached();
  const bool wide = (ld / BM) * ((ld + 255) / 256) >= 2 * sms;
  const bool narrow = !wide && (ld / BM) * ((ld + 127) / 128) < sms;
  const int bn = wide ? 256 : (narrow ? 64 : 128);
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, ld, kind, BM) || !make_map(&mb, Bop, ld, kind, bn)) return -1;
  GemmArgs g{};
  g.ld = ld;
  g.n = n;
  g.kind = kind;
  g.out_kind = out_kind;
  g.C = C;
  g.Kmat = Kmat;
  g.lam = lam;
  g.cmax = cmax;
  g.err = err;
  g.limit_ns = limit_ns;
  if (kind == 0) {
    if (wide) return launch_k<0, 256>(ma, mb, g, ld, s);
    return narrow ? launch_k<0, 64>(ma, mb, g, ld, s) : launch_k<0, 128>(ma, mb, g, ld, s);
  }
  if (wide) return launch_k<1, 256>(ma, mb, g, ld, s);
  return narrow ? launch_k<1, 64>(ma, mb, g, ld, s) : launch_k<1, 128>(ma, mb, g, ld, s);
}

}  // namespace fram
