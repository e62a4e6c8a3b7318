"""Benchmark: FRAM solves/s on one GB300 (or N independent replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload medium|small|large] [--precision fp64|bf16|tf32]

A step is one complete FRAM solve (prescale, outer iterations of gradient
GEMMs + SDSN + damped update, assignment, objective) of one synthetic graph
pair.  The default workload is the n=1000 ER pair (p=0.05, U(0,1) weights,
N(0,0.05) edge noise, 5% edge flips, theta=10).  Inputs are resident in HBM
when the timed region starts; L2 is flushed (a 256 MiB write) between timed
steps and the flush is outside the timed events.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import fram_inputs as fi  # noqa: E402

METRIC = "FRAM solves/s and ms/solve, mixed vs FP64 on 1 GB300 at equal accuracy; p50/p99 latency"
UNIT = "solves/s"

BATCH_DESC = ("4096 keypoint-like Gaussian-kernel pairs, n ~ U{10..64}, 0-20% outliers per side "
              "padded with dummy nodes, N(0,0.02) jitter, theta=2; one batched call per step")

WORKLOADS = {
    "small": ("ER pair n=50, p=0.2, U(0,1), N(0,0.02) edge noise, theta=10", fi.small_er_pair),
    "medium": ("ER pair n=1000, p=0.05, U(0,1), N(0,0.05) noise, 5% edge flips, theta=10",
               fi.medium_er_pair),
    "large": ("Gaussian-kernel pair n=8192, sigma=median distance, N(0,0.01) jitter, theta=2",
              fi.large_gaussian_pair),
    "social": ("Facebook-sized power-law social pair: Chung-Lu graph, n=4039, ~88k unweighted "
               "edges, degree exponent 3.1, planted relabelling, 5% edge flips, theta=10",
               fi.facebook_like_pair),
    "attributed": ("Gaussian-kernel pair n=1000 with d=128 nonnegative unit node descriptors "
                   "(N(0,0.5/sqrt(d)) noise on the partner), K = F F~^T computed in the step, "
                   "theta=2, lambda=1", fi.attributed_medium_pair),
}
PRECISIONS = {"fp64": 0, "tf32": 1, "bf16": 2}
DTYPES = {"fp64": "f64", "tf32": "tf32+f32+f64", "bf16": "bf16+f32+f64"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(seconds, ws, device="cuda"):
    """The job's time is the slowest replica's: MAX over ranks (identity at
    ws == 1).  `device` is the tensor device of the process group's backend."""
    if ws <= 1:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, ws, seconds):
    """Whole-job throughput: units every replica processed / the job's time."""
    return ws * units_per_rank / seconds


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_node_term(g):
    import oracle as o
    return o.node_affinity(g.F, g.Ft) if g.F is not None else None


def oracle_solve(g, max_outer=100):
    import oracle as o
    return o.fram(g.A, g.B, K=oracle_node_term(g), theta=g.theta, max_outer=max_outer)


def cpu_baseline(g, budget_s=12.0):
    """The oracle timed on the host cores on the same workload: complete
    solves of the same pair, run until `budget_s` seconds have passed (at
    least one), and the measured rate."""
    solves, spent, outer = 0, 0.0, 0
    while spent < budget_s or solves == 0:
        t0 = time.perf_counter()
        r = oracle_solve(g)
        spent += time.perf_counter() - t0
        solves += 1
        outer = r.outer_iters
    return {"value": solves / spent, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"numpy FP64 oracle, {solves} complete solves of the same pair "
                      f"({outer} outer iterations each), {spent:.1f} s measured"}


def cpu_baseline_scaled(g, outer_full):
    """For pairs whose complete oracle solve takes many minutes on the host
    (n > 2048): one outer iteration timed, scaled to `outer_full`."""
    t0 = time.perf_counter()
    oracle_solve(g, max_outer=1)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / (dt * outer_full), "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"numpy FP64 oracle, first outer iteration of the same solve ({dt:.1f} s), "
                      f"scaled to the FP64 solve's {outer_full} iterations (a full solve would "
                      f"take {dt * outer_full / 60:.0f} min)"}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, as it stands, on the host
    cores.  Every warm-up and timed step is one complete solve of the
    workload's pair (measured, not extrapolated)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    desc, make = WORKLOADS.get(args.workload, WORKLOADS["medium"])
    g = make(0)
    for _ in range(args.warmup):
        oracle_solve(g)
    per, outer = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle_solve(g)
        per.append(time.perf_counter() - t0)
        outer = r.outer_iters
    value = len(per) / sum(per)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(per),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc, "n": g.n, "precision": "fp64",
                                        "l2": "n/a (CPU)"},
        "latency_ms": {"p50": 1e3 * float(np.percentile(per, 50)),
                       "p99": 1e3 * float(np.percentile(per, 99))},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                         "sample": f"numpy FP64 oracle; every step one complete solve of the "
                                   f"pair ({outer} outer iterations), {sum(per):.1f} s for "
                                   f"{len(per)} timed solves"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def solve_step(fr, ctx, n, A, B, params, X, P, node):
    """One solve; with node attributes (d, F, Ft, K) the affinity K = F Ft^T
    is formed first, inside the step."""
    K = None
    if node is not None:
        d, F, Ft, K = node
        fr.fram_node_affinity(ctx, n, d, F, Ft, K)
    return fr.fram_solve(ctx, n, A, B, K, params, X, P)


def time_solves(fr, torch, ctx, n, A, B, params, steps, warmup, flush, node=None):
    """W untimed solves, then `steps` solves each bracketed by CUDA events on
    the library's stream (L2 flushed before each, outside the events)."""
    X = torch.empty((n, n), dtype=torch.float64, device="cuda")
    P = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        solve_step(fr, ctx, n, A, B, params, X, P, node)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    launches0 = fr.fram_kernel_launches(ctx)
    infos = []
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        _, info = solve_step(fr, ctx, n, A, B, params, X, P, node)
        ev[k][1].record(stream)
        infos.append(info)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    return ms, infos, X, P, fr.fram_kernel_launches(ctx) - launches0


# FP32 CUDA-core peak of one GB300 for the batched kernel's ALU roofline:
# 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz maximum SM clock.
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def batch_roofline(ns, infos, step_s):
    """ALU roofline of the batched kernel (one launch per call; the gather and
    scatter kernels around it take under 0.3% of the call).  Algorithmic FP32
    flops per pair: per outer iteration the two n^3 products (4 n^3) and the
    update with its delta (6 n^2); per SDSN sweep 7 n^2 (row and column sums,
    the three-term affine map of eq. 7, the gamma sum)."""
    flops = sum(i.outer_iters * (4.0 * n ** 3 + 6.0 * n * n) + i.total_sweeps * 7.0 * n * n
                for n, i in zip(ns, infos))
    achieved = flops / step_s / 1e12
    return {"kernel": "batched_kernel<float>", "bound": "alu", "achieved": achieved,
            "peak": FP32_ALU_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_ALU_TFLOPS,
            "traffic": None, "per_launch_us": step_s * 1e6,
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz"}


class Packed:
    """One buffer holding a batch's arrays back to back, the address of each
    entry as a uint64 array (a pointer table fram_solve_batched takes as it
    is) and per-entry views.  Every entry starts on a whole element: 8-byte
    aligned for FP64, 4 for int32."""

    def __init__(self, torch, shapes, dtype, device, src=None, pin=False):
        sizes = np.array([int(np.prod(sh)) for sh in shapes], dtype=np.int64)
        off = np.zeros(len(shapes), dtype=np.int64)
        off[1:] = np.cumsum(sizes)[:-1]
        if src is not None:
            host = torch.from_numpy(np.concatenate([np.ravel(a) for a in src]))
            host = host.to(dtype)
            self.buf = host.pin_memory() if pin else host.to(device)
        else:
            self.buf = torch.empty(int(sizes.sum()), dtype=dtype, device=device,
                                   pin_memory=pin)
        self.addr = (np.uint64(self.buf.data_ptr()) +
                     off.astype(np.uint64) * np.uint64(self.buf.element_size()))
        self.views = [self.buf[o:o + z].view(sh) for o, z, sh in zip(off, sizes, shapes)]


def batch_vs_fp64(fr, ctx, stream, flush, ns, As, Bs, params, pairs, args, o):
    """The same pairs through the FP64 batched path: its rate (same timing
    rules: CUDA events per call, L2 flushed before each) and the mixed
    results' distance from it (accuracy, objective, X)."""
    import torch
    p64 = fr.fram_default_params(theta=2.0, precision=fr.FRAM_PREC_FP64)
    vec = [(int(n),) for n in ns]
    mat = [(int(n), int(n)) for n in ns]
    P64 = Packed(torch, vec, torch.int32, "cuda")
    X64 = Packed(torch, mat, torch.float64, "cuda")
    Xm = Packed(torch, mat, torch.float64, "cuda")
    Pm = Packed(torch, vec, torch.int32, "cuda")
    for _ in range(2):  # warm-up: autotune and graph capture for this signature
        fr.fram_solve_batched(ctx, ns, As.addr, Bs.addr, p64, X64.addr, P64.addr)
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 3))
    ms = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, i64 = fr.fram_solve_batched(ctx, ns, As.addr, Bs.addr, p64, X64.addr, P64.addr)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    _, im = fr.fram_solve_batched(ctx, ns, As.addr, Bs.addr, params, Xm.addr, Pm.addr)
    torch.cuda.synchronize()
    acc64 = [o.accuracy(P.cpu().numpy(), g.truth) for P, g in zip(P64.views, pairs)]
    accm = [o.accuracy(P.cpu().numpy(), g.truth) for P, g in zip(Pm.views, pairs)]
    same = [bool(torch.equal(a, b)) for a, b in zip(Pm.views, P64.views)]
    obj = [abs(x.objective - y.objective) / max(abs(y.objective), 1e-300) for x, y in zip(im, i64)]
    xerr = [float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
            for a, b in zip(Xm.views, X64.views)]
    return {"fp64": {"value": len(ns) * steps / (sum(ms) / 1e3), "unit": UNIT,
                     "ms_per_step": sum(ms) / steps,
                     "mean_outer_iters": float(np.mean([i.outer_iters for i in i64])),
                     "mean_accuracy": float(np.mean(acc64))},
            "accuracy": {"accuracy_pp": 100.0 * (float(np.mean(accm)) - float(np.mean(acc64))),
                         "objective_rel_err_max": float(np.max(obj)),
                         "objective_rel_err_mean": float(np.mean(obj)),
                         "X_rel_err_mean": float(np.mean(xerr)),
                         "X_rel_err_max": float(np.max(xerr)),
                         "perm_identical_frac": float(np.mean(same))}}


def run_batch(args):
    """Batched workload: one step = one fram_solve_batched call (one persistent
    kernel launch replayed from a CUDA graph) over 4096 small pairs."""
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_2508_00887_gb300 import build
    if rank == 0 or ws == 1:
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    import paper_2508_00887_gb300 as fr
    fr.load()
    pairs = fi.keypoint_batch(args.batch_count, seed=rank)
    ns = [g.n for g in pairs]
    stream = torch.cuda.current_stream()
    ctx = fr.fram_create(dev, 0, stream.cuda_stream)
    params = fr.fram_default_params(theta=2.0, precision=PRECISIONS[args.precision])
    # Each batch in one packed buffer per argument, passed as address arrays:
    # the binding then hands the pointer tables to the library without a
    # per-tensor check or copy (the way a data loader would deliver a batch).
    mat = [(g.n, g.n) for g in pairs]
    vec = [(g.n,) for g in pairs]
    ns = np.array(ns, dtype=np.int32)
    As = Packed(torch, mat, torch.float64, "cuda", src=[g.A for g in pairs])
    Bs = Packed(torch, mat, torch.float64, "cuda", src=[g.B for g in pairs])
    Ps = Packed(torch, vec, torch.int32, "cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        fr.fram_solve_batched(ctx, ns, As.addr, Bs.addr, params, None, Ps.addr)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    l0 = fr.fram_kernel_launches(ctx)
    with ClockSampler(dev) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            _, infos = fr.fram_solve_batched(ctx, ns, As.addr, Bs.addr, params, None, Ps.addr)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    launches = fr.fram_kernel_launches(ctx) - l0
    ms = [a.elapsed_time(b) for a, b in ev]
    total_s = max_over_ranks(sum(ms) / 1e3, ws)
    value = job_rate(args.steps * len(pairs), ws, total_s)
    chosen = fr.fram_batched_kernel(ctx, PRECISIONS[args.precision])
    # Each kernel form the autotuner chose among, timed on the whole batch
    # (one call each, L2 flushed before), for the record.
    forms = {}
    names = {1: "cta128", 2: "cta256", 3: "cta512", 4: "team_split32", 5: "team_edge64"}
    for v in (1, 2, 3, 4, 5) if args.precision != "fp64" else (1, 2, 3):
        fr.fram_set_batched_kernel(ctx, v)
        fr.fram_solve_batched(ctx, ns, As.addr, Bs.addr, params, None, Ps.addr)  # tune/capture
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fr.fram_solve_batched(ctx, ns, As.addr, Bs.addr, params, None, Ps.addr)
        e1.record(stream)
        torch.cuda.synchronize()
        forms[names[v]] = e0.elapsed_time(e1)
    fr.fram_set_batched_kernel(ctx, 0)
    # End to end with host buffers (pinned): packing, copies and unpacking inside.
    Ah = Packed(torch, mat, torch.float64, "cpu", src=[g.A for g in pairs], pin=True)
    Bh = Packed(torch, mat, torch.float64, "cpu", src=[g.B for g in pairs], pin=True)
    Ph = Packed(torch, vec, torch.int32, "cpu", pin=True)
    fr.fram_solve_batched(ctx, ns, Ah.addr, Bh.addr, params, None, Ph.addr)  # untimed: re-tunes
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        fr.fram_solve_batched(ctx, ns, Ah.addr, Bh.addr, params, None, Ph.addr)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if rank == 0:
        import oracle as o
        acc = float(np.mean([o.accuracy(P.cpu().numpy(), g.truth)
                             for P, g in zip(Ps.views, pairs)]))
        vs64 = batch_vs_fp64(fr, ctx, stream, flush, ns, As, Bs, params, pairs, args, o)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision != "fp64" else "f64", "data": "synthetic",
            "config": {"workload": BATCH_DESC, "pairs": len(pairs), "precision": args.precision,
                       "l2": "flushed between timed steps (256 MiB write)",
                       "kernel_form": {1: "cta128", 2: "cta256", 3: "cta512", 4: "team_split32",
                                       5: "team_edge64"}.get(chosen, str(chosen)),
                       "forms_ms": forms},
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
            "solve": {"mean_accuracy": acc,
                      "mean_outer_iters": float(np.mean([i.outer_iters for i in infos])),
                      "mean_sweeps": float(np.mean([i.total_sweeps for i in infos]))},
            "e2e": {"value": ws * len(pairs) / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(sum(2 * g.n * g.n * 8 for g in pairs)),
                    "d2h_bytes_per_step": int(sum(g.n * 4 for g in pairs))},
            "roofline": batch_roofline(ns, infos, total_s / args.steps),
            "fp64": vs64["fp64"], "speedup_vs_fp64": value / ws / vs64["fp64"]["value"],
            "vs_fp64_accuracy": vs64["accuracy"],
            "gpu_launches": int(launches), "clocks": clk.summary(),
        }
        if not args.no_cpu_baseline and ws == 1:
            sample = pairs[:args.cpu_pairs]
            t0 = time.perf_counter()
            for g in sample:
                o.fram(g.A, g.B, theta=2.0)
            dt = time.perf_counter() - t0
            line["cpu_baseline"] = {"value": len(sample) / dt, "unit": UNIT, "cores": cpu_cores(),
                                    "kind": "oracle",
                                    "sample": f"numpy FP64 oracle on the first {len(sample)} pairs "
                                              f"of the batch ({dt:.1f} s)"}
        print(json.dumps(line), flush=True)
    fr.fram_destroy(ctx)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


SERVE_DESC = ("Poisson stream, n log-uniform on [20, 2048], ER p=0.1 U(0,1) weights, planted "
              "permutation + N(0,0.05) noise, theta=10; offered load 0.7 x measured saturated rate; "
              "requests draw from a pool of pre-generated pairs")


def serve_vs_fp64(fr, ctx, params, reqs, o):
    """The same requests served at FP64 and at the bench precision, each set
    submitted at once (saturated): the two rates and the distance of the
    mixed results from the FP64 ones."""
    p64 = fr.fram_default_params(theta=10.0, precision=fr.FRAM_PREC_FP64)

    def run(p):
        t0 = time.perf_counter()
        tk = [fr.fram_submit(ctx, g.n, g.A, g.B, p)[1] for g in reqs]
        out = []
        for t, g in zip(tk, reqs):
            P = np.empty(g.n, np.int32)
            _, info = fr.fram_poll(ctx, t, None, P, wait_ms=-1)
            out.append((P, info.objective))
        return len(reqs) / (time.perf_counter() - t0), out

    run(p64)  # warm-up at FP64 (kernels and slots)
    r64, o64 = run(p64)
    rm, om = run(params)
    acc64 = [o.accuracy(P, g.truth) for (P, _), g in zip(o64, reqs)]
    accm = [o.accuracy(P, g.truth) for (P, _), g in zip(om, reqs)]
    obj = [abs(a[1] - b[1]) / max(abs(b[1]), 1e-300) for a, b in zip(om, o64)]
    same = [bool(np.array_equal(a[0], b[0])) for a, b in zip(om, o64)]
    return {"fp64": {"value": r64, "unit": UNIT, "requests": len(reqs),
                     "mean_accuracy": float(np.mean(acc64)),
                     "note": "saturated: all requests submitted at once; mixed on the same set: "
                             f"{rm:.2f} solves/s"},
            "speedup": rm / r64,
            "accuracy": {"accuracy_pp": 100.0 * (float(np.mean(accm)) - float(np.mean(acc64))),
                         "objective_rel_err_max": float(np.max(obj)),
                         "objective_rel_err_mean": float(np.mean(obj)),
                         "perm_identical_frac": float(np.mean(same))}}


def run_serve(args):
    """Serving workload (fram_submit / fram_poll): a saturation pass measures
    capacity, then a Poisson stream at 0.7x that rate measures latency."""
    import threading

    import torch
    torch.cuda.set_device(0)
    from paper_2508_00887_gb300 import build
    build.build()
    import paper_2508_00887_gb300 as fr
    fr.load()
    rng = np.random.default_rng(11)
    pool_n = np.unique(np.round(np.exp(rng.uniform(np.log(20), np.log(2048), size=args.serve_pool)))
                       .astype(int))
    pool = [fi.serving_pair(int(n), seed=1000 + k) for k, n in enumerate(pool_n)]
    ctx = fr.fram_create(0, 0, torch.cuda.current_stream().cuda_stream)
    params = fr.fram_default_params(theta=10.0, precision=PRECISIONS[args.precision],
                                    max_polish=args.polish if args.precision != "fp64" else 0)
    pick = np.random.default_rng(12).integers(0, len(pool), size=args.serve_count)

    def submit(g):
        return fr.fram_submit(ctx, g.n, g.A, g.B, params)[1]

    def collect(tickets, gs, out):
        for t, g in zip(tickets, gs):
            P = np.empty(g.n, np.int32)
            st, info = fr.fram_poll(ctx, t, None, P, wait_ms=-1)
            out.append((time.perf_counter(), info.ms_total, P, g))

    # warm-up (kernels, slot cache)
    ws_g = [pool[k] for k in pick[:16]]
    tk = [submit(g) for g in ws_g]
    collect(tk, ws_g, [])
    # saturation: everything submitted at once
    sat_g = [pool[k] for k in pick[:args.serve_sat]]
    l0 = fr.fram_kernel_launches(ctx)
    t0 = time.perf_counter()
    tk = [submit(g) for g in sat_g]
    res = []
    collect(tk, sat_g, res)
    sat_rate = len(sat_g) / (time.perf_counter() - t0)
    # Poisson stream at 0.7 x saturation
    rate = 0.7 * sat_rate
    gaps = np.random.default_rng(13).exponential(1.0 / rate, size=args.serve_count)
    arrivals = np.cumsum(gaps)
    stream_g = [pool[k] for k in pick]
    tickets, done = [], []
    poller_q = []
    lock = threading.Condition()

    def poller():
        i = 0
        while i < len(stream_g):
            with lock:
                while len(poller_q) <= i:
                    lock.wait()
                t = poller_q[i]
            g = stream_g[i]
            P = np.empty(g.n, np.int32)
            st, info = fr.fram_poll(ctx, t, None, P, wait_ms=-1)
            done.append((info.ms_total, P, g))
            i += 1

    th = threading.Thread(target=poller)
    t0_ticks = fr.fram_serve_ticks(ctx)
    l0 = fr.fram_kernel_launches(ctx)
    th.start()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        for k, g in enumerate(stream_g):
            while time.perf_counter() - t0 < arrivals[k]:
                time.sleep(0.0002)
            t = submit(g)
            with lock:
                poller_q.append(t)
                lock.notify()
        th.join()
        elapsed = time.perf_counter() - t0
    launches = fr.fram_kernel_launches(ctx) - l0
    ticks = fr.fram_serve_ticks(ctx) - t0_ticks
    lat = np.array([d[0] for d in done])
    ns_done = np.array([d[2].n for d in done])
    import oracle as o
    vs64 = serve_vs_fp64(fr, ctx, params, sat_g[:args.serve_fp64], o)
    acc = float(np.mean([o.accuracy(d[1], d[2].truth) for d in done]))
    # 1% sample stratified over n (evenly spaced in the n-sorted stream).  The
    # oracle solves the requests it can afford (n <= 400); larger ones are
    # compared with the GPU FP64 path on the same pair, which the parity tests
    # tie to the oracle at 1e-9.
    k = max(1, args.serve_count // 100)
    order = np.argsort(ns_done, kind="stable")
    sample = [done[i] for i in order[np.linspace(0, len(done) - 1, k).round().astype(int)]]
    p64 = fr.fram_default_params(theta=10.0)
    acc_m, acc_r, obj_rel, ref_kind = [], [], [], []
    for d in sample:
        g, P = d[2], d[1]
        if g.n <= 400:
            r = o.fram(g.A, g.B, theta=10.0)
            ref_perm, ref_obj = r.perm, r.objective
            ref_kind.append("oracle")
        else:
            Pr = np.empty(g.n, np.int32)
            _, ir = fr.fram_solve(ctx, g.n, g.A, g.B, None, p64, None, Pr)
            ref_perm, ref_obj = Pr, ir.objective
            ref_kind.append("gpu_fp64")
        acc_m.append(o.accuracy(P, g.truth))
        acc_r.append(o.accuracy(ref_perm, g.truth))
        obj_rel.append(abs(o.objective(g.A, g.B, P) - ref_obj) / max(abs(ref_obj), 1e-300))
    bins = [(20, 100), (100, 400), (400, 1024), (1024, 2049)]
    by_n = {}
    for lo, hi in bins:
        m = (ns_done >= lo) & (ns_done < hi)
        if m.any():
            by_n[f"{lo}-{hi - 1}"] = {"requests": int(m.sum()),
                                     "p50": float(np.percentile(lat[m], 50)),
                                     "p99": float(np.percentile(lat[m], 99))}
    line = {
        "metric": METRIC, "value": len(done) / elapsed, "unit": UNIT, "n_gpus": 1,
        "steps": len(done), "warmup": 16, "ms_per_step": 1e3 * elapsed / len(done),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.precision], "data": "synthetic",
        "config": {"workload": SERVE_DESC, "requests": len(done), "pool_pairs": len(pool),
                   "offered_rate": rate, "saturated_rate": sat_rate, "precision": args.precision},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "by_n": by_n},
        "solve": {"mean_accuracy": acc, "sample_size": len(sample),
                  "sample_n_range": [int(sample[0][2].n), int(sample[-1][2].n)],
                  "sample_reference": {kk: ref_kind.count(kk) for kk in set(ref_kind)},
                  "sample_accuracy": float(np.mean(acc_m)),
                  "sample_reference_accuracy": float(np.mean(acc_r)),
                  "sample_accuracy_pp_max": 100.0 * float(np.max(np.abs(np.subtract(acc_m, acc_r)))),
                  "sample_objective_rel_err_max": float(np.max(obj_rel))},
        "ticks": int(ticks), "launches_per_tick": launches / max(1, ticks),
        # The serving rate is itself end to end: numpy host inputs go in
        # through fram_submit and permutations come back through fram_poll.
        "e2e": {"value": len(done) / elapsed, "unit": UNIT,
                "h2d_bytes_per_step": float(np.mean([16.0 * d[2].n ** 2 for d in done])),
                "d2h_bytes_per_step": float(np.mean([4.0 * d[2].n for d in done]))},
        "fp64": vs64["fp64"], "speedup_vs_fp64": vs64["speedup"],
        "vs_fp64_accuracy": vs64["accuracy"],
        "gpu_launches": int(launches), "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    fr.fram_destroy(ctx)
    return 0


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_2508_00887_gb300 import build
    if rank == 0 or ws == 1:
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    import paper_2508_00887_gb300 as fr
    fr.load()

    desc, make = WORKLOADS[args.workload]
    if args.n and args.workload == "large":
        g = fi.large_gaussian_pair(rank, n=args.n)
        desc = desc.replace("n=8192", f"n={args.n}")
    else:
        g = make(rank)                    # each replica solves its own pair
    n = g.n
    stream = torch.cuda.current_stream()
    ctx = fr.fram_create(dev, 0, stream.cuda_stream)
    mixed = args.precision != "fp64"
    params = fr.fram_default_params(theta=g.theta, precision=PRECISIONS[args.precision],
                                    max_polish=args.polish if mixed else 0)
    if args.projection == "exact":   # step 6 variant: the exact FRA solution (FP64 path)
        params.projection = fr.FRAM_PROJ_EXACT
        params.max_sweeps = args.exact_sweeps
    A = torch.from_numpy(g.A).to("cuda")
    B = torch.from_numpy(g.B).to("cuda")
    node = None
    if g.F is not None:
        d = g.F.shape[1]
        node = (d, torch.from_numpy(g.F).to("cuda"), torch.from_numpy(g.Ft).to("cuda"),
                torch.empty((n, n), dtype=torch.float64, device="cuda"))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    if ws > 1:
        torch.distributed.barrier()

    with ClockSampler(dev) as clk:
        ms, infos, X, P, launches = time_solves(fr, torch, ctx, n, A, B, params, args.steps,
                                                args.warmup, flush, node)
    total_s = max_over_ranks(sum(ms) / 1e3, ws)
    if ws > 1:
        torch.distributed.barrier()
    value = job_rate(args.steps, ws, total_s)

    # The FP64 path on the same input: the comparison the metric asks for
    # (mixed vs FP64 at equal accuracy).
    fp64 = None
    if mixed and not args.no_fp64:
        p64 = fr.fram_default_params(theta=g.theta)
        ms64, infos64, X64, P64, _ = time_solves(fr, torch, ctx, n, A, B, p64,
                                                 max(2, min(args.steps, 5)), 1, flush, node)
        fp64 = {"ms": ms64, "info": infos64[-1], "X": X64.cpu().numpy(), "P": P64.cpu().numpy()}

    # End to end through the public API with host buffers: the library copies
    # A, B host->device inside the call and writes N and perm back to host.
    Ah = torch.from_numpy(g.A).pin_memory()
    Bh = torch.from_numpy(g.B).pin_memory()
    Xh = torch.empty((n, n), dtype=torch.float64).pin_memory()
    Ph = torch.empty(n, dtype=torch.int32).pin_memory()
    node_h2d = 0
    if node is not None:
        Fh = torch.from_numpy(g.F).pin_memory()
        Fth = torch.from_numpy(g.Ft).pin_memory()
        node_h2d = 2 * g.F.size * 8
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        if node is not None:   # descriptors host -> device inside the step
            node[1].copy_(Fh, non_blocking=True)
            node[2].copy_(Fth, non_blocking=True)
        solve_step(fr, ctx, n, Ah, Bh, params, Xh, Ph, node)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, ws)
    e2e = {"value": job_rate(1, ws, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": 2 * n * n * 8 + node_h2d, "d2h_bytes_per_step": n * n * 8 + n * 4}

    if rank == 0:
        import oracle as o
        pk, src = peaks()
        last = infos[-1]
        perm = P.cpu().numpy()
        roof = roofline(infos, n, args.precision, pk, src)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": {"workload": desc, "n": n, "precision": args.precision,
                       "projection": args.projection,
                       "fp64_polish_sweeps": params.max_polish,
                       "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
            "solve": {"outer_iters": last.outer_iters, "total_sweeps": last.total_sweeps,
                      "polish_sweeps": last.polish_sweeps, "objective": last.objective,
                      "lap_augmentations": last.lap_augmentations,
                      "lap_auction_phases": last.lap_auction_phases,
                      "accuracy": o.accuracy(perm, g.truth)},
        }
        if fp64 is not None:
            i64 = fp64["info"]
            v64 = 1e3 / statistics.mean(fp64["ms"])
            Xm = X.cpu().numpy()
            line["fp64"] = {
                "value": v64, "unit": UNIT, "ms_per_step": statistics.mean(fp64["ms"]),
                "outer_iters": i64.outer_iters, "objective": i64.objective,
                "accuracy": o.accuracy(fp64["P"], g.truth)}
            line["speedup_vs_fp64"] = value / ws / v64
            line["vs_fp64_accuracy"] = {
                "X_rel_err": float(np.linalg.norm(Xm - fp64["X"]) / np.linalg.norm(fp64["X"])),
                "objective_rel_err": abs(last.objective - i64.objective) / abs(i64.objective),
                "accuracy_pp": 100.0 * (o.accuracy(perm, g.truth) - o.accuracy(fp64["P"], g.truth)),
                "perm_identical": bool(np.array_equal(perm, fp64["P"]))}
        line.update({"e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary(),
                     "roofline": roof})
        if not args.no_cpu_baseline and ws == 1:
            outer = fp64["info"].outer_iters if fp64 is not None else last.outer_iters
            # n > 2048 (social, dense n = 8192): a complete oracle solve takes
            # many minutes on the host, so one outer iteration is timed instead.
            line["cpu_baseline"] = (cpu_baseline_scaled(g, outer) if n > 2048
                                    else cpu_baseline(g))
        print(json.dumps(line), flush=True)
    fr.fram_destroy(ctx)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def sdsn_traffic(n, s, sweeps_per_launch):
    """DRAM bytes per FP32 SDSN launch (dram__bytes_read.sum +
    dram__bytes_write.sum, one ncu capture of the current kernel), or None
    where no capture covers the size:
      n = 1000: 4.18 MB per launch, whatever the sweep count: the tiles stay
        in shared memory and only X is read (capture of this workload);
      n >= 6144 (the matrix far above L2): 7.80 bytes per element per pass,
        measured at n = 6144 (59.16 GB over 201 passes of 6144^2), scaled to
        n^2 (sweeps + 1) bytes."""
    if s != 4:
        return None
    if n == 1000:
        return 4.18e6
    if n >= 6144:
        return 7.80 * n * n * (sweeps_per_launch + 1.0)
    return None


def roofline(infos, n, precision, pk, src):
    """Roofline of the dominant phase, from the live per-phase device times of
    the timed steps (CUDA events on the solve's stream).

    SDSN: algorithmic bytes per launch = (sweeps + 1) * 2 * n^2 * s (each sweep
    reads and writes the matrix once; the first pass reads X and writes Y),
    s = 4 (FP32 phase of the mixed path) or 8 (FP64).  Gradient GEMMs:
    4 n^3 flops per outer iteration."""
    s = 8 if precision == "fp64" else 4
    ms_sdsn = sum(i.ms_sdsn for i in infos)
    ms_gemm = sum(i.ms_gemm for i in infos)
    sweeps = sum(i.total_sweeps - i.polish_sweeps for i in infos)
    launches = sum(i.outer_iters for i in infos)
    sdsn_bytes = (sweeps + launches) * 2.0 * n * n * s
    gemm_flops = launches * 4.0 * n ** 3
    sdsn = {"kernel": f"sdsn_kernel<{'double' if s == 8 else 'float'}>", "bound": "hbm",
            "achieved": sdsn_bytes / (ms_sdsn / 1e3) / 1e9 if ms_sdsn else None,
            "peak": pk.get("hbm_gbs"), "unit": "GB/s",
            "per_launch_us": 1e3 * ms_sdsn / max(launches, 1),
            "per_sweep_us": 1e3 * ms_sdsn / max(sweeps, 1)}
    if s == 4 and 2 <= n <= 1024:
        # The FP32 iterate stays on chip in one thread-block cluster (DRAM
        # carries X once), so the sweep is bound by its arithmetic and
        # exchange on the cluster's SMs, not by HBM: 5 n^2 FP32 operations
        # per sweep (y + a_i, - b_j, the clamp, the row and the column
        # accumulation) against one operation per lane per clock.
        # Up to n = 64 the iterate sits in the registers of one or two warps
        # (one scheduler each, 32 lanes): the same count against their lanes.
        side = 1 if n <= 256 else (2 if n <= 512 else 4)
        tc = ((-(-n // side)) + 3) // 4 * 4
        sms = side * side
        clock_ghz = 2.07
        ops = 5.0 * n * n * sweeps
        if n <= 64:
            warps = 1 if n <= 32 else 2
            kernel, lanes = f"sdsn_warp_kernel<{warps}>", warps * 32
            where = f"the form's {warps} warp{'s' if warps > 1 else ''} x 32 FP32 lanes"
        else:
            kernel = f"sdsn_cluster_kernel<{'1, 16' if tc <= 128 else '2, 8'}>"
            lanes, where = sms * 128, f"the cluster's {sms} SMs x 128 FP32 lanes"
        sdsn = {"kernel": kernel,
                "bound": "alu",
                "achieved": ops / (ms_sdsn / 1e3) / 1e12 if ms_sdsn else None,
                "peak": lanes * clock_ghz / 1e3, "unit": "TFLOP/s",
                "peak_source": f"derived: {where} x 1 operation per clock x {clock_ghz} GHz "
                               "(adds and max, no FMA)",
                "gpu_peak": 152 * 128 * clock_ghz / 1e3,
                "per_launch_us": 1e3 * ms_sdsn / max(launches, 1),
                "per_sweep_us": 1e3 * ms_sdsn / max(sweeps, 1)}
    if precision == "fp64":
        peak_t, unit_peak = 1.25, "TFLOP/s (nominal FP64, no measured FP64 peak)"
    elif precision == "bf16":
        peak_t, unit_peak = pk.get("bf16_tflops_sustained", 1700.0), "measured bf16 sustained"
    else:
        peak_t, unit_peak = pk.get("bf16_tflops_sustained", 1700.0) / 2.0, \
            "measured bf16 sustained x 1/2 (nominal tf32:bf16 ratio)"
    gemm = {"kernel": "dgemm_kernel" if precision == "fp64" else "gemm_tc_kernel",
            "bound": "alu" if precision == "fp64" else "tensor",
            "achieved": gemm_flops / (ms_gemm / 1e3) / 1e12 if ms_gemm else None,
            "peak": peak_t, "unit": "TFLOP/s", "peak_source": unit_peak}
    sdsn["traffic"] = sdsn_traffic(n, s, sweeps / max(launches, 1))
    gemm["traffic"] = None
    dom, other = (sdsn, gemm) if ms_sdsn >= ms_gemm else (gemm, sdsn)
    dom = dict(dom)
    dom["frac"] = dom["achieved"] / dom["peak"] if dom["achieved"] and dom["peak"] else None
    if dom.get("gpu_peak") and dom["achieved"]:
        dom["gpu_frac"] = dom["achieved"] / dom["gpu_peak"]
    dom["peak_source"] = dom.get("peak_source", f"{src} hbm_gbs")
    dom["time_share"] = {"sdsn_ms": ms_sdsn, "gemm_ms": ms_gemm,
                         "polish_ms": sum(i.ms_polish for i in infos),
                         "update_ms": sum(i.ms_update for i in infos),
                         "rounding_ms": sum(i.ms_rounding for i in infos),
                         "total_ms": sum(i.ms_total for i in infos)}
    other = dict(other)
    other["frac"] = other["achieved"] / other["peak"] if other["achieved"] and other["peak"] else None
    dom["other"] = other
    return dom


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOADS) + ["batch", "serve"], default="medium")
    ap.add_argument("--serve-count", type=int, default=2000)
    ap.add_argument("--serve-sat", type=int, default=400)
    ap.add_argument("--serve-pool", type=int, default=48)
    ap.add_argument("--serve-fp64", type=int, default=100,
                    help="saturation requests also served at FP64 for the comparison")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--n", type=int, default=0, help="size override for --workload large")
    ap.add_argument("--cpu-pairs", type=int, default=100)
    ap.add_argument("--precision", choices=list(PRECISIONS), default="tf32",
                    help="tf32: step 5 in TF32 as in the paper's mixed-precision runs")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--polish", type=int, default=4, help="FP64 polish sweeps (mixed paths)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--projection", choices=["sdsn", "exact"], default="sdsn",
                    help="step 6: the paper's SDSN or the exact FRA projection (fp64 only)")
    ap.add_argument("--exact-sweeps", type=int, default=2000,
                    help="sweep cap of the exact projection")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
