// Serving: fram_submit / fram_poll with continuous batching.
//
// A scheduler thread owned by the context runs FRAM (Alg. 1 of arXiv
// 2508.00887) for many requests at once, at outer-iteration granularity:
//   * admission: waiting requests get a device slot (A, B, N, X and the
//     low-precision shadows stay resident until the request retires) while
//     the HBM budget has room; freed slots are cached and reused;
//   * one tick = one outer iteration of every active request, in a number
//     of launches that does not grow with the number of requests (mixed
//     precision): one kernel clears every slot's per-iteration state, one
//     grouped tensor-core launch per GEMM of step 5 and input precision
//     (each request's tiles computed exactly as its solo launch computes
//     them), the grouped FP32 SDSN (one cluster per request for n <= 1024,
//     co-resident sub-grids otherwise), the grouped FP64 polish, and one
//     grouped update per precision; FP64 requests keep per-request GEMMs
//     and updates;
//   * stats of all active requests come back in one copy per tick; requests
//     that stopped (delta, rounding floor, cap, or an error) retire: LAP and
//     objective on the device, results copied to host, slot released;
//   * requests that arrive meanwhile join at the next tick.
// Each request follows the same arithmetic as fram_solve with its params,
// so a result does not depend on which other requests share its ticks.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fram_ctx.h"
#include "fram_tc.h"

namespace fram {

namespace {

constexpr int kMaxActive = 48;       // requests iterating at once (<= SMs for the SDSN group)
constexpr size_t kMaxWaiting = 1u << 16;

struct SlotStats {
  IterStats it;
  LapStats lap;
  ObjStats obj;
  ValidateStats val;
  unsigned long long xmax;
  GridBarrier bar32;
  GridBarrier bar64;
  unsigned ticket_upd;
  unsigned ticket_obj;
  int pad[2];
};

enum ReqState { R_WAITING, R_ACTIVE, R_DONE };

struct Request {
  uint64_t ticket = 0;
  int n = 0, ld = 0, kind = 0;  // kind: 0 BF16, 1 TF32 (mixed paths)
  bool mixed = false;
  fram_params p{};
  std::vector<double> hA, hB;
  // device slot
  char* base = nullptr;
  size_t bytes = 0;
  int sid = -1;
  double *A0 = nullptr, *B0 = nullptr, *As = nullptr, *Bs = nullptr, *N = nullptr, *X64 = nullptr,
         *T64 = nullptr;
  void *Alp = nullptr, *Blp = nullptr, *Nt = nullptr, *Tlp = nullptr;
  float* X32 = nullptr;
  GemmGroupProblem g1{}, g2{};  // T = A N and X = T B as grouped-GEMM problems
  double *spart = nullptr, *upart = nullptr;
  void* lap_ws = nullptr;
  int32_t* perm = nullptr;
  // progress
  ReqState state = R_WAITING;
  bool prepped = false;
  int t = 0;
  double prev_delta = INFINITY;
  fram_status status = FRAM_OK;
  std::string err;
  fram_info info{};
  std::vector<double> Nres;
  std::vector<int32_t> permres;
  std::chrono::steady_clock::time_point t_submit;
};

struct Serve {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread th;
  bool stop = false;
  std::deque<Request*> waiting;
  std::vector<Request*> active;
  std::unordered_map<uint64_t, Request*> all;
  uint64_t next_ticket = 1;
  cudaStream_t stream = nullptr, copy_stream = nullptr;
  SlotStats* dstats = nullptr;
  SlotStats* hstats = nullptr;
  void* ddesc = nullptr;
  void* gdesc[2] = {nullptr, nullptr};  // grouped GEMM problems (64-byte aligned)
  void* udesc = nullptr;                // grouped update problems
  uint64_t ticks = 0;
  std::vector<int> free_ids;
  std::vector<std::pair<size_t, char*>> cache;  // free slot blocks
  size_t budget = 0;
};

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

size_t slot_bytes(const fram_ctx* c, int n, bool mixed) {
  const size_t ld = round_ld(n), m64 = ld * ld * 8, m32 = ld * ld * 4;
  size_t b = 2 * al256((size_t)n * n * 8);           // A0, B0
  b += 4 * al256(m64);                                // As, Bs, N, X64
  b += mixed ? 5 * al256(m32) : al256(m64);           // lp shadows | T64
  b += al256(sdsn_partials_elems(n, c->num_sms) * 8);
  b += al256(4096 * 8);
  b += al256(lap_workspace_bytes(n));
  b += al256((size_t)n * 4);
  return b;
}

void carve(Request* r, int num_sms) {
  char* p = r->base;
  const size_t n = r->n, ld = r->ld, m64 = ld * ld * 8, m32 = ld * ld * 4;
  auto take = [&](size_t b) {
    char* q = p;
    p += al256(b);
    return q;
  };
  r->A0 = (double*)take(n * n * 8);
  r->B0 = (double*)take(n * n * 8);
  r->As = (double*)take(m64);
  r->Bs = (double*)take(m64);
  r->N = (double*)take(m64);
  r->X64 = (double*)take(m64);
  if (r->mixed) {
    r->Alp = take(m32);
    r->Blp = take(m32);
    r->Nt = take(m32);
    r->Tlp = take(m32);
    r->X32 = (float*)take(m32);
  } else {
    r->T64 = (double*)take(m64);
  }
  r->spart = (double*)take(sdsn_partials_elems(r->n, num_sms) * 8);
  r->upart = (double*)take(4096 * 8);
  r->lap_ws = take(lap_workspace_bytes(r->n));
  r->perm = (int32_t*)take(n * 4);
}

// Device memory for a slot: best-fitting cached block, else a new
// allocation within the budget (evicting cached blocks if needed).
bool get_block(fram_ctx* c, Serve& S, size_t need, char** out, size_t* got) {
  int best = -1;
  for (int i = 0; i < (int)S.cache.size(); ++i)
    if (S.cache[i].first >= need && (best < 0 || S.cache[i].first < S.cache[best].first)) best = i;
  if (best >= 0) {
    *out = S.cache[best].second;
    *got = S.cache[best].first;
    S.cache.erase(S.cache.begin() + best);
    return true;
  }
  while (c->serve_bytes + need > S.budget && !S.cache.empty()) {
    cudaFree(S.cache.back().second);
    c->serve_bytes -= S.cache.back().first;
    S.cache.pop_back();
  }
  if (c->serve_bytes + need > S.budget) return false;
  void* p = nullptr;
  if (cudaMalloc(&p, need) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  c->serve_bytes += need;
  *out = static_cast<char*>(p);
  *got = need;
  return true;
}

void release_slot(Serve& S, Request* r) {
  if (r->base) S.cache.push_back({r->bytes, r->base});
  r->base = nullptr;
  if (r->sid >= 0) S.free_ids.push_back(r->sid);
  r->sid = -1;
}

void finish(Serve& S, Request* r, fram_status st, const char* msg) {
  r->status = st;
  if (msg) r->err = msg;
  auto dt = std::chrono::steady_clock::now() - r->t_submit;
  r->info.ms_total = std::chrono::duration<double, std::milli>(dt).count();
  {
    std::lock_guard<std::mutex> lk(S.mu);
    release_slot(S, r);
    r->state = R_DONE;
  }
  S.cv_done.notify_all();
}

// Count the kernels a launcher started (its return value, evaluated once).
bool sv_ok(fram_ctx* c, int launched) {
  if (launched < 0) return false;
  c->launches += (uint64_t)launched;
  return true;
}
#define SV_OK(x) sv_ok(c, (x))

// Clear the per-iteration state of every slot (IterStats, the max key and
// both SDSN barriers) in one launch, instead of three memsets per request.
__global__ void tick_prologue_kernel(SlotStats* st, int count) {
  SlotStats& s = st[blockIdx.x];
  if (blockIdx.x >= (unsigned)count) return;
  int* it = reinterpret_cast<int*>(&s.it);
  for (unsigned k = threadIdx.x; k < sizeof(IterStats) / sizeof(int); k += blockDim.x) it[k] = 0;
  if (threadIdx.x == 0) {
    s.xmax = 0ull;
    s.bar32 = GridBarrier{};
    s.bar64 = GridBarrier{};
  }
}

void serve_loop(fram_ctx* c, Serve* Sp) {
  Serve& S = *Sp;
  cudaSetDevice(c->device);
  std::vector<Request*> fresh;
  while (true) {
    fresh.clear();
    {
      std::unique_lock<std::mutex> lk(S.mu);
      S.cv_work.wait(lk, [&] { return S.stop || !S.waiting.empty() || !S.active.empty(); });
      if (S.stop) break;
      // Admission by HBM footprint.
      while (!S.waiting.empty() && !S.free_ids.empty()) {
        Request* r = S.waiting.front();
        const size_t need = slot_bytes(c, r->n, r->mixed);
        char* blk = nullptr;
        size_t got = 0;
        if (!get_block(c, S, need, &blk, &got)) {
          if (S.active.empty() && fresh.empty() && c->serve_bytes == 0) {
            // Can never fit: fail it rather than wait forever.
            S.waiting.pop_front();
            lk.unlock();
            finish(S, r, FRAM_ERR_OOM, "request does not fit the HBM budget");
            lk.lock();
            continue;
          }
          break;
        }
        S.waiting.pop_front();
        r->base = blk;
        r->bytes = got;
        r->sid = S.free_ids.back();
        S.free_ids.pop_back();
        carve(r, c->num_sms);
        r->state = R_ACTIVE;
        fresh.push_back(r);
      }
    }
    cudaStream_t s = S.stream;
    // Prepare newly admitted requests: upload, validate, prescale, init.
    if (!fresh.empty()) {
      for (Request* r : fresh) {
        const size_t nn = (size_t)r->n * r->n;
        cudaMemcpyAsync(r->A0, r->hA.data(), nn * 8, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(r->B0, r->hB.data(), nn * 8, cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(&S.dstats[r->sid], 0, sizeof(SlotStats), s);
        SV_OK(launch_validate(r->A0, r->B0, nullptr, r->n, &S.dstats[r->sid].val, s));
      }
      cudaMemcpyAsync(S.hstats, S.dstats, kMaxActive * sizeof(SlotStats), cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) cudaGetLastError();
      for (Request* r : fresh) {
        r->hA = std::vector<double>();
        r->hB = std::vector<double>();
        const ValidateStats& v = S.hstats[r->sid].val;
        double mx[2], as[2];
        memcpy(mx, v.maxbits, 16);
        memcpy(as, v.asymbits, 16);
        if (v.bad_value[0] || v.bad_value[1] || as[0] > 1e-12 * std::max(mx[0], 1.0) ||
            as[1] > 1e-12 * std::max(mx[1], 1.0)) {
          finish(S, r, FRAM_ERR_INVALID, "input outside the graph model");
          continue;
        }
        const double cc = std::max(mx[0], mx[1]);
        if (!(cc > 0.0)) {
          finish(S, r, FRAM_ERR_DEGENERATE, "all inputs are zero");
          continue;
        }
        const double inv_s = 1.0 / sqrt(cc);  // as fram_solve's prescale
        SV_OK(launch_scale(r->A0, r->n, inv_s, r->As, r->ld, s));
        SV_OK(launch_scale(r->B0, r->n, inv_s, r->Bs, r->ld, s));
        SV_OK(launch_fill_assignment(r->N, r->n, r->ld, 1.0 / r->n, s));
        if (r->mixed) {
          SV_OK(launch_convert_lp(r->As, r->Alp, r->ld, r->kind, s));
          SV_OK(launch_convert_lp(r->Bs, r->Blp, r->ld, r->kind, s));
          SV_OK(launch_transpose_lp(r->N, r->Nt, r->ld, r->kind, s));
          SlotStats* sst = &S.dstats[r->sid];
          if (!make_group_problem(&r->g1, r->Alp, r->Nt, r->Tlp, r->ld, r->n, r->kind, nullptr,
                                  &sst->it.gemm_err) ||
              !make_group_problem(&r->g2, r->Tlp, r->Blp, r->X32, r->ld, r->n, r->kind,
                                  &sst->xmax, &sst->it.gemm_err)) {
            finish(S, r, FRAM_ERR_CUDA, "tensor map encode failed");
            continue;
          }
        }
        r->prepped = true;
        std::lock_guard<std::mutex> lk(S.mu);
        S.active.push_back(r);
      }
    }
    std::vector<Request*> act;
    {
      std::lock_guard<std::mutex> lk(S.mu);
      act = S.active;
    }
    if (act.empty()) continue;
    // One outer iteration of every active request.
    ++S.ticks;
    bool ok = true;
    tick_prologue_kernel<<<kMaxActive, 64, 0, s>>>(S.dstats, kMaxActive);
    ok = SV_OK(cudaPeekAtLastError() == cudaSuccess ? 1 : -1) && ok;
    std::vector<SdsnLaunch> L64, L32, Lpol;
    std::vector<GemmGroupProblem> gp1[2], gp2[2];
    for (Request* r : act) {
      SlotStats* st = &S.dstats[r->sid];
      SdsnLaunch L{};
      L.n = r->n;
      L.ldx = L.ldy = r->ld;
      L.theta = r->p.theta;
      L.xmax_key = &st->xmax;
      L.stats = &st->it.sdsn;
      L.partials = r->spart;
      L.limit_ns = c->wait_limit_ns;
      L.barrier_zeroed = 1;
      if (!r->mixed) {
        ok = SV_OK(launch_dgemm(r->As, r->N, r->T64, r->ld, r->n, nullptr, 0.0, nullptr, s)) && ok;
        ok = SV_OK(launch_dgemm(r->T64, r->Bs, r->X64, r->ld, r->n, nullptr, 0.0, &st->xmax, s)) && ok;
        L.X = L.Y = r->X64;
        L.gamma_tol = r->p.gamma_tol;
        L.max_sweeps = r->p.max_sweeps;
        L.barrier = &st->bar64;
        L64.push_back(L);
      } else {
        gp1[r->kind].push_back(r->g1);
        gp2[r->kind].push_back(r->g2);
        const double tol32 = std::max(r->p.polish_tol, r->p.gamma_tol);
        L.X = L.Y = r->X32;
        L.in_fp32 = L.out_fp32 = 1;
        L.gamma_tol = tol32;
        L.max_sweeps = std::max(1, r->p.max_sweeps - r->p.max_polish);
        L.barrier = &st->bar32;
        L32.push_back(L);
        SdsnLaunch P = L;
        P.X = r->X32;
        P.Y = r->X64;
        P.out_fp32 = 0;
        P.mode = 1;
        P.gamma_tol = r->p.gamma_tol;
        P.max_sweeps = r->p.max_polish;
        P.gate = &st->it.sdsn;
        P.gate_tol = tol32;
        P.stats = &st->it.polish;
        P.barrier = &st->bar64;
        Lpol.push_back(P);
      }
    }
    // Step 5: one grouped launch per GEMM and input precision.
    const size_t gbytes = kMaxActive * sizeof(GemmGroupProblem);
    for (int kind = 0; kind < 2 && ok; ++kind) {
      if (gp1[kind].empty()) continue;
      ok = SV_OK(launch_gemm_tc_group(gp1[kind].data(), (int)gp1[kind].size(), kind,
                                      kind == 0 ? 1 : 2, S.gdesc[0], gbytes, c->wait_limit_ns,
                                      s)) && ok;
      ok = ok && SV_OK(launch_gemm_tc_group(gp2[kind].data(), (int)gp2[kind].size(), kind, 0,
                                            S.gdesc[1], gbytes, c->wait_limit_ns, s));
    }
    // Grouped SDSN launches.  Every request keeps the sub-grid that
    // fram_solve would give it alone (so its arithmetic, and its result, do
    // not depend on the other requests); requests are packed into waves of
    // co-resident sub-grids of at most one CTA per SM.
    const size_t dbytes = sdsn_group_desc_bytes(kMaxActive);
    auto waves = [&](std::vector<SdsnLaunch>& Ls) {
      size_t i = 0;
      while (ok && i < Ls.size()) {
        size_t j = i;
        int blocks = 0;
        while (j < Ls.size() && blocks + sdsn_grid_blocks(Ls[j].n, c->num_sms) <= c->num_sms)
          blocks += sdsn_grid_blocks(Ls[j++].n, c->num_sms);
        if (j == i) ++j;  // a single problem always fits on its own
        ok = ok && SV_OK(launch_sdsn_group(Ls.data() + i, (int)(j - i), c->num_sms, S.ddesc,
                                           dbytes, c->num_sms, s));
        i = j;
      }
    };
    waves(L64);
    // FP32 problems of 2 <= n <= 1024 run on chip, as fram_solve runs them
    // (warps up to n = 64, one cluster each above): one launch per class,
    // any number of problems.
    {
      std::vector<SdsnLaunch> grid32, cls[kSdsnClusterClasses];
      for (const SdsnLaunch& L : L32) {
        const int k = sdsn_cluster_class(L);
        (k > 0 ? cls[k] : grid32).push_back(L);
      }
      for (int k = 1; k < kSdsnClusterClasses && ok; ++k)
        if (!cls[k].empty())
          ok = SV_OK(launch_sdsn_cluster_group(cls[k].data(), (int)cls[k].size(), S.ddesc, dbytes,
                                               s)) && ok;
      waves(grid32);
    }
    // FP64 polishes: those of 2 <= n <= 64 in one CTA of warps each, as
    // fram_solve runs them; the rest in co-resident waves.
    {
      std::vector<SdsnLaunch> small, rest;
      for (const SdsnLaunch& L : Lpol) (sdsn_polish_small_applies(L) ? small : rest).push_back(L);
      if (!small.empty())
        ok = SV_OK(launch_sdsn_polish_small_group(small.data(), (int)small.size(), S.ddesc, dbytes,
                                                  s)) && ok;
      waves(rest);
    }
    // Steps 7-8: one grouped update per precision (FP64 requests alone).
    std::vector<UpdGroupProblem> up[2];
    for (Request* r : act) {
      SlotStats* st = &S.dstats[r->sid];
      if (!r->mixed) {
        ok = SV_OK(launch_update(r->N, r->ld, r->X64, r->ld, r->n, r->p.alpha, &st->it, r->upart,
                                 &st->ticket_upd, s)) && ok;
      } else {
        UpdGroupProblem u{};
        u.N = r->N;
        u.D = r->X64;
        u.Nt = r->Nt;
        u.partials = r->upart;
        u.ticket = &st->ticket_upd;
        u.st = &st->it;
        u.alpha = r->p.alpha;
        u.ld = r->ld;
        u.n = r->n;
        up[r->kind].push_back(u);
      }
    }
    for (int kind = 0; kind < 2 && ok; ++kind)
      if (!up[kind].empty())
        ok = SV_OK(launch_update_mixed_group(up[kind].data(), (int)up[kind].size(), kind,
                                             kind == 0 ? S.udesc : static_cast<char*>(S.udesc) +
                                                             kMaxActive * sizeof(UpdGroupProblem),
                                             kMaxActive * sizeof(UpdGroupProblem), s)) && ok;
    cudaMemcpyAsync(S.hstats, S.dstats, kMaxActive * sizeof(SlotStats), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (!ok || e != cudaSuccess) {
      const char* m = e != cudaSuccess ? cudaGetErrorString(e) : "launch failed";
      cudaGetLastError();
      for (Request* r : act) finish(S, r, FRAM_ERR_CUDA, m);
      std::lock_guard<std::mutex> lk(S.mu);
      S.active.clear();
      continue;
    }
    // Stop tests (Alg. 1 step 4; mixed paths also stop at the rounding floor).
    std::vector<Request*> retire, keep;
    for (Request* r : act) {
      const IterStats& it = S.hstats[r->sid].it;
      int dev_err = it.sdsn.status ? it.sdsn.status : (r->mixed ? it.polish.status : 0);
      if (it.gemm_err) dev_err = DEV_TIMEOUT;
      if (dev_err) {
        finish(S, r, dev_err == DEV_DEGENERATE ? FRAM_ERR_DEGENERATE : FRAM_ERR_TIMEOUT,
               dev_err == DEV_DEGENERATE ? "max(X) <= 0" : "a device-side wait exceeded its limit");
        continue;
      }
      r->t += 1;
      r->info.outer_iters = r->t;
      r->info.total_sweeps += it.sdsn.sweeps + (r->mixed ? it.polish.sweeps : 0);
      r->info.polish_sweeps += r->mixed ? it.polish.sweeps : 0;
      r->info.gamma = r->mixed ? it.polish.gamma : it.sdsn.gamma;
      r->info.sdsn_converged_last = r->info.gamma <= r->p.gamma_tol ? 1 : 0;
      r->info.delta = it.delta;
      bool stop = it.delta <= r->p.delta_tol || r->t >= r->p.max_outer ||
                  (r->mixed && it.delta <= r->p.mixed_delta_tol);
      if (r->mixed && r->p.stall_ratio > 0.0 && it.delta <= r->p.stall_below &&
          it.delta > r->p.stall_ratio * r->prev_delta)
        stop = true;
      r->prev_delta = it.delta;
      (stop ? retire : keep).push_back(r);
    }
    {
      std::lock_guard<std::mutex> lk(S.mu);
      S.active = keep;
    }
    if (retire.empty()) continue;
    // Retire: discretise (eq. 2) and the objective (eq. 1), then results to host.
    for (Request* r : retire) {
      SlotStats* st = &S.dstats[r->sid];
      r->Nres.resize((size_t)r->n * r->n);
      r->permres.resize(r->n);
      SV_OK(launch_lap(r->N, r->ld, r->n, r->perm, &st->lap, r->lap_ws, c->num_sms,
                       c->wait_limit_ns, s, c->lap_searches));
      SV_OK(launch_objective(r->A0, r->B0, nullptr, r->p.lambda, r->n, r->perm, &st->obj, r->upart,
                             &st->ticket_obj, s));
      cudaMemcpy2DAsync(r->Nres.data(), (size_t)r->n * 8, r->N, (size_t)r->ld * 8, (size_t)r->n * 8,
                        r->n, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(r->permres.data(), r->perm, (size_t)r->n * 4, cudaMemcpyDeviceToHost, s);
    }
    cudaMemcpyAsync(S.hstats, S.dstats, kMaxActive * sizeof(SlotStats), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    for (Request* r : retire) {
      if (e != cudaSuccess) {
        finish(S, r, FRAM_ERR_CUDA, cudaGetErrorString(e));
        continue;
      }
      const SlotStats& st = S.hstats[r->sid];
      r->info.lap_augmentations = st.lap.augmented;
      r->info.lap_auction_phases = st.lap.auction_phases;
      r->info.assignment_value = st.lap.value;
      r->info.objective = st.obj.objective;
      r->info.match_error = st.obj.match_error;
      finish(S, r, st.lap.status ? FRAM_ERR_TIMEOUT : FRAM_OK,
             st.lap.status ? "assignment search did not terminate" : nullptr);
    }
    if (e != cudaSuccess) cudaGetLastError();
  }
}

Serve* get_serve(fram_ctx* c, fram_status* st) {
  std::lock_guard<std::mutex> lk(c->serve_mu);
  if (c->serve) return static_cast<Serve*>(c->serve);
  Serve* S = new Serve();
  size_t freeb = 0, total = 0;
  cudaMemGetInfo(&freeb, &total);
  S->budget = c->budget ? c->budget : (size_t)(0.6 * (double)freeb);
  bool ok = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMalloc(&S->dstats, kMaxActive * sizeof(SlotStats)) == cudaSuccess &&
            cudaMallocHost(&S->hstats, kMaxActive * sizeof(SlotStats)) == cudaSuccess &&
            cudaMalloc(&S->ddesc, sdsn_group_desc_bytes(kMaxActive)) == cudaSuccess &&
            cudaMalloc(&S->gdesc[0], kMaxActive * sizeof(GemmGroupProblem)) == cudaSuccess &&
            cudaMalloc(&S->gdesc[1], kMaxActive * sizeof(GemmGroupProblem)) == cudaSuccess &&
            cudaMalloc(&S->udesc, 2 * kMaxActive * sizeof(UpdGroupProblem)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    *st = FRAM_ERR_OOM;
    if (S->stream) cudaStreamDestroy(S->stream);
    if (S->copy_stream) cudaStreamDestroy(S->copy_stream);
    if (S->dstats) cudaFree(S->dstats);
    if (S->hstats) cudaFreeHost(S->hstats);
    if (S->ddesc) cudaFree(S->ddesc);
    for (void* d : {S->gdesc[0], S->gdesc[1], S->udesc})
      if (d) cudaFree(d);
    delete S;
    return nullptr;
  }
  for (int i = kMaxActive - 1; i >= 0; --i) S->free_ids.push_back(i);
  c->serve = S;
  S->th = std::thread(serve_loop, c, S);
  return S;
}

}  // namespace

void serve_shutdown(fram_ctx* c) {
  Serve* S = static_cast<Serve*>(c->serve);
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->th.joinable()) S->th.join();
  cudaStreamSynchronize(S->stream);
  for (auto& kv : S->all) {
    if (kv.second->base) cudaFree(kv.second->base);
    delete kv.second;
  }
  for (auto& b : S->cache) cudaFree(b.second);
  cudaStreamDestroy(S->stream);
  cudaStreamDestroy(S->copy_stream);
  cudaFree(S->dstats);
  cudaFreeHost(S->hstats);
  cudaFree(S->ddesc);
  cudaFree(S->gdesc[0]);
  cudaFree(S->gdesc[1]);
  cudaFree(S->udesc);
  c->serve_bytes = 0;
  delete S;
  c->serve = nullptr;
}

}  // namespace fram

using namespace fram;

extern "C" uint64_t fram_serve_ticks(const fram_ctx* c) {
  if (!c || !c->serve) return 0;
  return static_cast<const Serve*>(c->serve)->ticks;
}

extern "C" fram_status fram_submit(fram_ctx* c, int n, const double* A, const double* B,
                                   const fram_params* params, uint64_t* ticket) {
  if (!c) return FRAM_ERR_INVALID;
  if (n < 1 || !A || !B || !ticket) {
    set_err(c, "fram_submit: n >= 1 and non-NULL A, B, ticket are required");
    return FRAM_ERR_INVALID;
  }
  fram_params p;
  if (params)
    p = *params;
  else
    fram_default_params(&p);
  fram_status st = check_params(c, p);
  if (st != FRAM_OK) return st;
  if (p.projection != FRAM_PROJ_SDSN) {
    set_err(c, "fram_submit: the exact projection is available through fram_solve only");
    return FRAM_ERR_INVALID;
  }
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "set device");
  st = FRAM_OK;
  Serve* S = get_serve(c, &st);
  if (!S) {
    set_err(c, "fram_submit: could not start the scheduler");
    return st;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->waiting.size() >= kMaxWaiting) {
      set_err(c, "fram_submit: the waiting queue is full");
      return FRAM_ERR_BUSY;
    }
  }
  Request* r = new Request();
  r->n = n;
  r->ld = round_ld(n);
  r->p = p;
  r->mixed = p.precision != FRAM_PREC_FP64;
  r->kind = p.precision == FRAM_PREC_MIXED_BF16 ? 0 : 1;
  r->t_submit = std::chrono::steady_clock::now();
  const size_t nn = (size_t)n * n;
  r->hA.resize(nn);
  r->hB.resize(nn);
  // Library-owned copies before returning (device inputs come back through
  // the private copy stream).
  cudaError_t e = cudaMemcpyAsync(r->hA.data(), A, nn * 8, cudaMemcpyDefault, S->copy_stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->hB.data(), B, nn * 8, cudaMemcpyDefault, S->copy_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S->copy_stream);
  if (e != cudaSuccess) {
    delete r;
    return cuda_fail(c, e, "fram_submit: input copy");
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->ticket = S->next_ticket++;
    S->all[r->ticket] = r;
    S->waiting.push_back(r);
  }
  S->cv_work.notify_all();
  *ticket = r->ticket;
  return FRAM_OK;
}

extern "C" fram_status fram_poll(fram_ctx* c, uint64_t ticket, double* X_out, int32_t* perm_out,
                                 fram_info* info, int wait_ms) {
  if (!c) return FRAM_ERR_INVALID;
  Serve* S = static_cast<Serve*>(c->serve);
  if (!S) {
    set_err(c, "fram_poll: unknown ticket");
    return FRAM_ERR_INVALID;
  }
  Request* r = nullptr;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) {
      set_err(c, "fram_poll: unknown ticket %llu", (unsigned long long)ticket);
      return FRAM_ERR_INVALID;
    }
    r = it->second;
    auto done = [&] { return r->state == R_DONE; };
    if (!done()) {
      if (wait_ms == 0) return FRAM_NOT_READY;
      if (wait_ms < 0)
        S->cv_done.wait(lk, done);
      else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), done))
        return FRAM_NOT_READY;
    }
    S->all.erase(it);
  }
  fram_status st = r->status;
  if (st == FRAM_OK) {
    cudaError_t e = cudaSuccess;
    if (X_out)
      e = cudaMemcpy(X_out, r->Nres.data(), r->Nres.size() * 8, cudaMemcpyDefault);
    if (e == cudaSuccess && perm_out)
      e = cudaMemcpy(perm_out, r->permres.data(), r->permres.size() * 4, cudaMemcpyDefault);
    if (e != cudaSuccess) st = cuda_fail(c, e, "fram_poll: output copy");
    if (info) *info = r->info;
  } else {
    set_err(c, "fram_poll: request %llu failed: %s", (unsigned long long)ticket, r->err.c_str());
  }
  delete r;
  return st;
}
