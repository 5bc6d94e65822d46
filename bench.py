"""Benchmark of the direct-summation gravity pass on GB300.

Headline workload: block time-step Hermite-4 in mixed precision, N = 131072
equal-mass Plummer sphere, eps = 1e-4, N_active = 131072 (all sinks), with
nearest neighbours.  One step = the whole hot path: copy kernel for the
N_active updated particles, predictor for all N sources, force pass (and the
split-j reduction when the launch shape uses one).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  `value` is interactions/s (N_active x N per step,
self pair counted) over all ranks with inputs resident in HBM; `e2e` is the
same metric through the C ABI with pinned host buffers (host->device copy of
the updated particles and sink list, device->host copy of every output,
inside the timed region).  With --gpus N > 1 (torchrun) the ranks split the
sources (Sec. 2.2.3): every rank holds the same particle set, runs the pass
for all sinks over its own block of sources, and one exchange per step
(shards.combine: NCCL sum of the force fields, minimum of the nearest
neighbour) gives every rank the full result; `value` is then the job's
N_active x N per step over the slowest rank's time (strong scaling).
--replicas runs N independent replicas instead (weak scaling, no collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "interactions/s & %FP32 peak vs N_active; mixed/batched/adjoint vs FP64"
UNIT = "interactions/s"
WORKLOAD = "Plummer N=131072, eps=1e-4, Hermite-4 block step, mixed precision (double-single positions, FP32 terms, FP64 reduction), N_active=131072, with nearest neighbour"
# FP32 arithmetic operations (add, sub, mul, fma: the FMA pipe) per interaction
# of the mixed Hermite-4 pass: 9 double-single difference, 3 dv, 3 r^2,
# 1 softening add, 4 (rinv^2, m rinv, m rinv^3, potential sum), 3 r.v,
# 2 alpha, 3 acc, 6 jerk.  The rsqrt (SFU) and the two integer operations of
# the nearest-neighbour key run on other pipes and are not counted.  The peak
# is the FMA pipe's 128 lanes per SM per clock; a packed f32x2 instruction
# counts as two lane-operations, as it occupies the pipe for two cycles.
OPS_PER_INTERACTION = 34
L2_FLUSH_BYTES = 512 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=40)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=131072)
    p.add_argument("--n-active", type=int, default=131072)
    p.add_argument("--no-extras", action="store_true", help="skip the sweep / FP64 / batched / adjoint / lists lines")
    p.add_argument("--extras", default="c1,sweep,h6,batched,adjoint,nb,h2,blk,blk6",
                   help="comma-separated secondary sections: c1, sweep, h6, batched, adjoint, nb, h2, blk, blk6")
    p.add_argument("--blk-t-end", type=float, default=0.25,
                   help="end time of the 4th-order block time-step line (blk)")
    p.add_argument("--replicas", action="store_true",
                   help="with --gpus N > 1: N independent replicas instead of the source split")
    p.add_argument("--blk6-t-end", type=float, default=1.0,
                   help="end time of the 6th-order block-step runs (Sec. 3.7 integrates one N-body time unit)")
    p.add_argument("--blk6-n", default="1024,16384", help="particle counts of the 6th-order block-step runs")
    p.add_argument("--blk6-eps", default="1e-3", help="softening lengths of the 6th-order block-step runs")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-tune", action="store_true")
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                   help="precision of the headline step (profiling the FP64 kernel; the metric is quoted on mixed)")
    p.add_argument("--launch", default=None,
                   help="force the force-kernel launch shape: threads,i_per_thread,j_lanes,j_tile,split_j")
    return p.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() and args.impl == "ours" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, x: float) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [q.strip() for q in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


FORCE_SOURCES = ("paper_1510_04068_gb300/csrc/sp2_device.cuh", "paper_1510_04068_gb300/csrc/sp2_kernels_h4m.cu")
TRAFFIC_SUMMARY = "profiles/force_h4_mixed_131072.md"


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in FORCE_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic():
    """DRAM bytes of one full-size (N = N_active = 131072) force launch from the
    committed ncu summary, or None when the kernel source changed since the
    counters were taken."""
    try:
        with open(os.path.join(ROOT, TRAFFIC_SUMMARY)) as fh:
            txt = fh.read()
    except OSError:
        return None, None
    vals = {}
    for ln in txt.splitlines():
        if "=" in ln and ln.strip().startswith("- `"):
            k, _, v = ln.strip()[3:].partition("=")
            vals[k.strip(" `")] = v.strip(" `")
    if vals.get("source_sha256_16") != kernel_source_hash():
        return None, vals.get("source_sha256_16")
    try:
        return float(vals["dram_bytes_per_launch_131072"]), vals.get("source_sha256_16")
    except (KeyError, ValueError):
        return None, None


def make_workload(n, n_active, seed=0):
    m, x, v = W.plummer(n, seed)
    a, jk, _ = W.derivative_noise(n, seed + 1, scales=(1.0, 4.0, 16.0))
    ids = W.particle_ids(n)
    t = 1.0
    tj = W.block_times(n, seed + 2, t)
    idx = W.active_set(n, n_active, seed + 1000)
    return dict(m=m, x=x, v=v, a=a, jerk=jk, ids=ids, tj=tj, t=t, idx=idx)


def run_reference(args, world, rank):
    """The oracle, as it stands, on the host cores (the slow reference arm)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = make_workload(args.n, args.n_active)
    sample = int(min(args.n_active, 512))
    idx = w["idx"][:sample]
    step = lambda: oracle.step(w["t"], idx, w["ids"], w["m"], w["tj"], w["x"], w["v"], w["a"],  # noqa: E731
                               w["jerk"], None, eps2=1e-8, order=4)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    inter = args.steps * sample * args.n
    val = inter / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_sinks_per_step": sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"{sample} of the {args.n_active} sinks per step against all {args.n} "
                                       f"sources, predictor over all {args.n}"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def host_cpu():
    """CPU model string and logical core count of this host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            k, _, v = ln.partition(":")
            if k.strip() == "Model name" and v.strip():
                model = v.strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for ln in fh:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.partition(":")[2].strip()
                        break
        except OSError:
            pass
    return model or "unknown", os.cpu_count() or 1


def cpu_baseline(w, n, budget_s=12.0, budget_1core_s=6.0):
    """The oracle (as it stands) on a bounded sample of the sinks: once on all
    host cores (the reported `value`), once on one core."""
    import oracle
    oracle.build()
    step = lambda k: oracle.step(w["t"], w["idx"][:k], w["ids"], w["m"], w["tj"], w["x"], w["v"], w["a"],  # noqa: E731
                                 w["jerk"], None, eps2=1e-8, order=4)

    def timed_sample(budget):
        k0 = min(64, len(w["idx"]))
        t0 = time.perf_counter()
        step(k0)
        rate = k0 * n / max(time.perf_counter() - t0, 1e-6)
        k = int(min(len(w["idx"]), max(k0, budget * rate / n)))
        t0 = time.perf_counter()
        step(k)
        return k, time.perf_counter() - t0

    cores = oracle.threads()
    k, dt = timed_sample(budget_s)
    oracle.set_threads(1)
    try:
        k1, dt1 = timed_sample(budget_1core_s)
    finally:
        oracle.set_threads(cores)
    model, nproc = host_cpu()
    return {"value": k * n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{k} of the {len(w['idx'])} active sinks against all {n} sources "
                      f"(plus the predictor over all {n}), {dt:.1f} s",
            "value_1core": k1 * n / dt1,
            "sample_1core": f"{k1} sinks against all {n} sources on one core, {dt1:.1f} s",
            "cpu_model": model, "nproc": nproc}


def run_ours(args, world, rank, local):
    import torch
    from paper_1510_04068_gb300 import build as libbuild
    from paper_1510_04068_gb300 import sp2

    assert torch.cuda.is_available(), "bench.py needs a CUDA device (the library has no CPU path)"
    torch.cuda.set_device(local)
    libbuild.build()
    sp2.load()
    dev = torch.device("cuda", local)
    from paper_1510_04068_gb300 import shards
    n, n_act = args.n, args.n_active
    # world > 1: the source split of Sec. 2.2.3 (every rank the same particle
    # set, its own block of sources, one exchange per step), unless --replicas
    jsplit = world > 1 and not args.replicas
    w = make_workload(n, n_act, seed=0 if jsplit else rank)
    j_range = shards.shard_range(n, rank, world) if jsplit else None
    D = lambda q: torch.as_tensor(np.ascontiguousarray(q)).to(dev)  # noqa: E731
    idx_h = w["idx"]
    stream = torch.cuda.Stream(device=dev)
    eps2 = 1e-8
    full = {k: D(w[k]) for k in ("ids", "m", "x", "v", "a", "jerk", "tj")}
    upd = {k: full[k][torch.as_tensor(idx_h.astype(np.int64), device=dev)].contiguous() for k in full}
    idx = D(idx_h)
    out = dict(acc=torch.empty((n_act, 3), dtype=torch.float64, device=dev),
               jerk=torch.empty((n_act, 3), dtype=torch.float64, device=dev),
               pot=torch.empty(n_act, dtype=torch.float64, device=dev),
               nn_id=torch.empty(n_act, dtype=torch.int32, device=dev),
               nn_r2=torch.empty(n_act, dtype=torch.float64, device=dev))
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        prec = sp2.SP2_MIXED if args.precision == "mixed" else sp2.SP2_FP64
        ctx = sp2.Context(order=4, precision=prec, n_max=n, eps2=eps2, profile=1, cuda_stream=stream.cuda_stream)
        ctx.set_j(0, full["ids"], full["m"], full["x"], full["v"], full["a"], full["jerk"], None, full["tj"])
        ctx.predict(w["t"])
        if args.launch:
            th, ipt, jl, tile, split = (int(q) for q in args.launch.split(","))
            ctx.set_launch(n_act, dict(threads=th, i_per_thread=ipt, j_lanes=jl, j_tile=tile, split_j=split,
                                       ctas_per_sm=0))
            tuned = None
        else:
            # the tuner times passes over all sources; a rank of the source
            # split takes the default shape for its block
            tuned = None if (args.no_tune or jsplit) else ctx.autotune(n_act)
        launch = ctx.get_launch(n_act)

        def step(k):
            ctx.set_j(0, upd["ids"], upd["m"], upd["x"], upd["v"], upd["a"], upd["jerk"], None, upd["tj"],
                      slots=idx)
            ctx.predict(w["t"] + k * 2.0 ** -20)
            ctx.compute(idx, j_range=j_range, **out)
            if jsplit:
                shards.combine(out)

        for k in range(args.warmup):
            step(k)
            flush.zero_()
        stream.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier(world)
        torch.cuda.synchronize()
        ctx.profile_reset()
        l0 = ctx.kernel_launches()
        with ClockSampler(local) as clk:
            wall0 = time.perf_counter()
            for k in range(args.steps):
                ev[k][0].record(stream)
                step(k)
                ev[k][1].record(stream)
                flush.zero_()
            stream.synchronize()
            wall1 = time.perf_counter()
        torch.cuda.synchronize()
        barrier(world)
        launches = ctx.kernel_launches() - l0
        prof = ctx.profile_read()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = allmax(world, sum(step_ms))
    inter_step = n_act * n  # per rank and step (replicas) or for the whole job (source split)
    value = (1 if jsplit else world) * args.steps * inter_step / (total_ms / 1e3)
    rank_inter = inter_step * (j_range[1] - j_range[0]) / n if jsplit else inter_step
    fcount, fms = prof["force"]
    force_ms = fms / max(fcount, 1)
    dev_props = torch.cuda.get_device_properties(dev)
    pk = peaks()
    sm_max = pk.get("sm_max_mhz", 2070.0)
    peak_tops = dev_props.multi_processor_count * 128 * sm_max * 1e6 / 1e12
    achieved = rank_inter * OPS_PER_INTERACTION / (force_ms / 1e3) / 1e12
    clocks = clk.summary()
    # measured pipe rates (after the timed region): a second denominator for
    # the FMA-pipe fraction next to the one derived from unit counts and clock
    try:
        pipes = sp2.measure_pipe_peaks()
    except sp2.SP2Error:
        pipes = None
    tb, _sha = committed_traffic()
    traffic = tb if (tb is not None and n == 131072 and n_act == 131072) else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if jsplit else "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if args.precision == "mixed" else WORKLOAD.replace(
                       "mixed precision (double-single positions, FP32 terms, FP64 reduction)", "FP64"),
                   "n": n, "n_active": n_act, "order": 4, "precision": args.precision,
                   "eps": 1e-4, "nearest_neighbour": True,
                   "parallelism": f"jsplit{world}" if jsplit else f"replicas{world}",
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write, outside the step events)",
                   "launch": launch, "autotuned": tuned is not None,
                   "wall_ms_incl_flush": 1e3 * (wall1 - wall0) / args.steps},
        "stages_ms_per_step": {k: (v[1] / args.steps) for k, v in prof.items() if v[0]},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s (FP32 FMA-pipe lane-ops)",
                     "frac": achieved / peak_tops, "traffic": traffic,
                     "traffic_source": TRAFFIC_SUMMARY if traffic is not None else None,
                     "kernel": "pass_kernel<MixedPairForce<4,NN>>", "force_ms_per_launch": force_ms,
                     "ops_per_interaction": OPS_PER_INTERACTION,
                     "peak_basis": f"{dev_props.multi_processor_count} SMs x 128 FMA-pipe lanes x {sm_max:.0f} MHz "
                                   f"(max SM clock, MEASURED_PEAKS.json)",
                     "measured_pipe_peaks": None if pipes is None else {
                         "fp32_fma_lane_tops": pipes["fp32_fma_lane_ops"] / 1e12,
                         "fp32x2_fma_lane_tops": pipes["fp32x2_fma_lane_ops"] / 1e12,
                         "fp64_fma_tops": pipes["fp64_fma_ops"] / 1e12,
                         "rsqrt_tops": pipes["rsqrt_ops"] / 1e12,
                         "probe": "sp2_measure_pipe_peaks: independent FFMA / f32x2 FMA / DFMA / MUFU rsqrt chains"},
                     "frac_of_measured_fma": None if pipes is None else achieved / (
                         max(pipes["fp32_fma_lane_ops"], pipes["fp32x2_fma_lane_ops"]) / 1e12)},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if args.precision != "mixed":
        line["roofline"] = None  # the FP32 FMA-pipe roofline describes the mixed kernel only
    if world == 1 and rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w, n)
    if not args.no_e2e:
        line["e2e"] = e2e(ctx, w, upd, out, args, stream, j_range, world)
    if not args.no_extras and rank == 0:
        line["detail"] = extras(sp2, w, n, eps2, dev, stream, set(args.extras.split(",")), args.blk_t_end,
                                args.blk6_t_end, tuple(int(q) for q in args.blk6_n.split(",")),
                                tuple(float(q) for q in args.blk6_eps.split(",")))
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def e2e(ctx, w, upd, out, args, stream, j_range=None, world=1):
    """Same step through the C ABI with pinned host buffers; copies in the timed
    region.  Source split (j_range set): the rank's pass writes device outputs,
    the exchange combines them, and the combined result is copied to the host."""
    import torch
    from paper_1510_04068_gb300 import shards
    pin = lambda t: t.cpu().pin_memory()  # noqa: E731
    hu = {k: pin(v) for k, v in upd.items()}
    hidx = pin(torch.as_tensor(w["idx"]))
    ho = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
    n_act = len(w["idx"])

    def step(k):
        ctx.set_j(0, hu["ids"], hu["m"], hu["x"], hu["v"], hu["a"], hu["jerk"], None, hu["tj"], slots=hidx)
        ctx.predict(w["t"] + k * 2.0 ** -20)
        if j_range is None:
            ctx.compute(hidx, **ho)
        else:
            upd_idx.copy_(hidx, non_blocking=True)
            ctx.compute(upd_idx, j_range=j_range, **out)
            shards.combine(out)
            for key in out:
                ho[key].copy_(out[key], non_blocking=True)
            stream.synchronize()

    with torch.cuda.stream(stream):
        upd_idx = torch.empty(hidx.shape, dtype=hidx.dtype, device=next(iter(out.values())).device)
        for k in range(max(1, args.warmup)):
            step(k)
        barrier(world)
        t0 = time.perf_counter()
        for k in range(args.steps):
            step(k)
        dt = allmax(world, time.perf_counter() - t0)
    h2d = sum(v.numel() * v.element_size() for v in hu.values()) + 2 * hidx.numel() * 4
    d2h = sum(v.numel() * v.element_size() for v in ho.values())
    return {"value": args.steps * n_act * len(w["m"]) / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * dt / args.steps}


def timed(fn, reps, stream):
    import torch
    fn()
    stream.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        stream.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def extras(sp2, w, n, eps2, dev, stream, sections, blk_t_end=0.25, blk6_t_end=1.0, blk6_n=(1024, 16384),
           blk6_eps=(1e-3,)):
    """N_active sweep (mixed vs FP64), batched systems, adjoint: secondary lines."""
    import torch
    D = lambda q: torch.as_tensor(np.ascontiguousarray(q)).to(dev)  # noqa: E731
    res = {}
    with torch.cuda.stream(stream):
        if "c1" in sections:
            res["c1"] = bench_c1(sp2, dev, stream)
        if "sweep" in sections:
            res["sweep"] = sweep(sp2, w, n, eps2, dev, stream)
            res["graph_launch_floor"] = graph_launch_floor(dev, stream)
        if "h6" in sections:
            res["h6"] = bench_h6(sp2, dev, stream)
        if "batched" in sections:
            res["batched"] = bench_batched(sp2, dev, stream)
        if "adjoint" in sections:
            res["adjoint"] = bench_adjoint(dev, stream)
        if "nb" in sections:
            res["nb"] = bench_nb(sp2, dev, stream)
        if "h2" in sections:
            res["h2"] = bench_h2(sp2, dev, stream)
        if "blk" in sections:
            res["blk"] = bench_blk(sp2, dev, stream, t_end=blk_t_end)
        if "blk6" in sections:
            res["blk6"] = [r for nb in blk6_n for e in blk6_eps
                           for r in bench_blk6(sp2, dev, stream, n=nb, t_end=blk6_t_end, eps=e)]
    return res


def graph_launch_floor(dev, stream):
    """Context for the small-N_active steps: a CUDA graph of one trivial
    kernel (a one-element add), timed as the sweep times its graphs -- once
    per host wait, and replayed 20 times back to back."""
    import torch
    x = torch.zeros(1, device=dev)
    x.add_(1)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        x.add_(1)
    stream.synchronize()
    one = timed(g.replay, 20, stream)
    b2b = timed(lambda: [g.replay() for _ in range(20)], 5, stream) / 20
    return {"kernel": "one-element add", "us_per_launch": 1e3 * one, "back_to_back_us_per_launch": 1e3 * b2b}


def bench_c1(sp2, dev, stream):
    """Plain FP64 Hermite-4 pass, N = 1024 equal-mass Plummer, eps = 1e-3, all
    particles active: one predict + compute (acc, jerk, pot, nearest
    neighbour) per step, and the same through a CUDA graph."""
    import torch
    n = 1024
    m, x, v = W.plummer(n, 0)
    a, jk, _ = W.derivative_noise(n, 1, scales=(1.0, 4.0, 16.0))
    ids = W.particle_ids(n)
    D = lambda q: torch.as_tensor(np.ascontiguousarray(q)).to(dev)  # noqa: E731
    c = sp2.Context(order=4, precision=sp2.SP2_FP64, n_max=n, eps2=1e-6, cuda_stream=stream.cuda_stream)
    c.set_j(0, D(ids), D(m), D(x), D(v), D(a), D(jk), None, D(np.zeros(n)))
    idx = D(np.arange(n, dtype=np.int32))
    o = dict(acc=torch.empty((n, 3), dtype=torch.float64, device=dev),
             jerk=torch.empty((n, 3), dtype=torch.float64, device=dev),
             pot=torch.empty(n, dtype=torch.float64, device=dev),
             nn_id=torch.empty(n, dtype=torch.int32, device=dev),
             nn_r2=torch.empty(n, dtype=torch.float64, device=dev))
    c.predict(0.0)
    c.autotune(n)
    fn = lambda: (c.predict(0.0), c.compute(idx, **o))  # noqa: E731
    ms = timed(fn, 50, stream)
    sp2.sp2_graph_begin(c.ctx)
    fn()
    g = sp2.sp2_graph_end(c.ctx)
    gms = timed(lambda: sp2.sp2_graph_launch(c.ctx, g), 50, stream)
    sp2.sp2_graph_destroy(g)
    c.close()
    return {"n": n, "us_per_step": 1e3 * ms, "graph_us_per_step": 1e3 * gms,
            "interactions_per_s": n * n / (ms / 1e3)}


def sweep(sp2, w, n, eps2, dev, stream):
    """interactions/s per block step vs N_active, mixed and FP64."""
    import torch
    D = lambda q: torch.as_tensor(np.ascontiguousarray(q)).to(dev)  # noqa: E731
    rows = []
    full = {k: D(w[k]) for k in ("ids", "m", "x", "v", "a", "jerk", "tj")}
    ctxs = {}
    for prec in (sp2.SP2_MIXED, sp2.SP2_FP64):
        c = sp2.Context(order=4, precision=prec, n_max=n, eps2=eps2, cuda_stream=stream.cuda_stream)
        c.set_j(0, full["ids"], full["m"], full["x"], full["v"], full["a"], full["jerk"], None, full["tj"])
        c.predict(w["t"])
        ctxs[prec] = c
    for na in (1, 8, 64, 1024, 16384, 131072):
        idx = D(W.active_set(n, na, 1000 + na))
        o = dict(acc=torch.empty((na, 3), dtype=torch.float64, device=dev),
                 jerk=torch.empty((na, 3), dtype=torch.float64, device=dev),
                 pot=torch.empty(na, dtype=torch.float64, device=dev),
                 nn_id=torch.empty(na, dtype=torch.int32, device=dev),
                 nn_r2=torch.empty(na, dtype=torch.float64, device=dev))
        row = {"n_active": na}
        for prec, name in ((sp2.SP2_MIXED, "mixed"), (sp2.SP2_FP64, "fp64")):
            c = ctxs[prec]
            if name == "fp64" and na > 16384:
                reps = 2
            else:
                reps = 20
            c.autotune(na) if (name == "mixed" or na <= 1024) else None
            fn = lambda: (c.predict(w["t"]), c.compute(idx, **o))  # noqa: E731
            ms = timed(fn, reps, stream)
            row[f"{name}_us_per_step"] = 1e3 * ms
            row[f"{name}_interactions_per_s"] = na * n / (ms / 1e3)
            if name == "mixed":
                sp2.sp2_graph_begin(c.ctx)
                fn()
                g = sp2.sp2_graph_end(c.ctx)
                gms = timed(lambda: sp2.sp2_graph_launch(c.ctx, g), reps, stream)
                # the same graph replayed back to back (steps issued without a
                # host wait in between, as a device-driven block loop runs them)
                bms = timed(lambda: [sp2.sp2_graph_launch(c.ctx, g) for _ in range(20)], max(2, reps // 4), stream) / 20
                sp2.sp2_graph_destroy(g)
                row["mixed_graph_us_per_step"] = 1e3 * gms
                row["mixed_graph_back_to_back_us_per_step"] = 1e3 * bms
                if na <= 64:
                    # the fused pass reads each source's double-single cache
                    # once (112 B); the sweep does not flush L2 between steps
                    row["mixed_jstream_gbs_l2_warm"] = n * 112 / (ms / 1e3) / 1e9
                if na <= 1024:
                    # the paper's 1D form: one thread per sink, no source split
                    tuned_shape = c.get_launch(na)
                    c.set_launch(na, dict(threads=max(32, min(256, 32 * ((na + 31) // 32))), i_per_thread=1,
                                          j_lanes=1, j_tile=128, split_j=1, ctas_per_sm=0))
                    ms1 = timed(fn, 3, stream)
                    c.set_launch(na, tuned_shape)
                    row["mixed_1d_us_per_step"] = 1e3 * ms1
                    row["split_speedup_vs_1d"] = ms1 / ms
        row["mixed_over_fp64"] = row["mixed_interactions_per_s"] / row["fp64_interactions_per_s"]
        rows.append(row)
    for c in ctxs.values():
        c.close()
    return rows


def bench_h6(sp2, dev, stream):
    """Hermite-6 on a Salpeter Plummer sphere, N = 65536: mixed vs FP64."""
    import torch
    n = 65536
    m, x, v = W.plummer(n, 3)
    m = W.salpeter_masses(n, 10)
    a, jk, sn = W.derivative_noise(n, 16, scales=(1.0, 4.0, 16.0))
    ids = W.particle_ids(n)
    tj = W.block_times(n, 14, 0.5)
    D = lambda q: torch.as_tensor(np.ascontiguousarray(q)).to(dev)  # noqa: E731
    rows = []
    ctxs = {}
    for prec in (sp2.SP2_MIXED, sp2.SP2_FP64):
        c = sp2.Context(order=6, precision=prec, n_max=n, eps2=1e-8, cuda_stream=stream.cuda_stream)
        c.set_j(0, D(ids), D(m), D(x), D(v), D(a), D(jk), D(sn), D(tj))
        c.predict(0.5)
        ctxs[prec] = c
    for na in (32, 4096, 65536):
        idx = D(W.active_set(n, na, 2000 + na))
        o = dict(acc=torch.empty((na, 3), dtype=torch.float64, device=dev),
                 jerk=torch.empty((na, 3), dtype=torch.float64, device=dev),
                 snap=torch.empty((na, 3), dtype=torch.float64, device=dev),
                 pot=torch.empty(na, dtype=torch.float64, device=dev),
                 nn_id=torch.empty(na, dtype=torch.int32, device=dev),
                 nn_r2=torch.empty(na, dtype=torch.float64, device=dev))
        row = {"n_active": na}
        for prec, name in ((sp2.SP2_MIXED, "mixed"), (sp2.SP2_FP64, "fp64")):
            c = ctxs[prec]
            if name == "mixed" or na <= 4096:
                c.autotune(na)
            fn = lambda: (c.predict(0.5), c.compute(idx, **o))  # noqa: E731
            ms = timed(fn, 2 if (name == "fp64" and na > 4096) else 10, stream)
            row[f"{name}_us_per_step"] = 1e3 * ms
            row[f"{name}_interactions_per_s"] = na * n / (ms / 1e3)
        row["mixed_over_fp64"] = row["mixed_interactions_per_s"] / row["fp64_interactions_per_s"]
        rows.append(row)
    for c in ctxs.values():
        c.close()
    return rows


def bench_nb(sp2, dev, stream):
    """Neighbour lists (radius search riding on the force pass): Plummer
    N = 131072, mixed Hermite-4 + NN, N_active = 16384 and 131072, h^2 = 2.5e-3
    for every sink, capacity 256; the same step with and without lists."""
    import torch
    n = 131072
    m, x, v = W.plummer(n, 0)
    a, jk, _ = W.derivative_noise(n, 1, scales=(1.0, 4.0, 16.0))
    ids = W.particle_ids(n)
    tj = W.block_times(n, 2, 1.0)
    D = lambda q: torch.as_tensor(np.ascontiguousarray(q)).to(dev)  # noqa: E731
    c = sp2.Context(order=4, precision=sp2.SP2_MIXED, n_max=n, eps2=1e-8, cuda_stream=stream.cuda_stream)
    c.set_j(0, D(ids), D(m), D(x), D(v), D(a), D(jk), None, D(tj))
    c.predict(1.0)
    rows = []
    for na in (16384, 131072):
        idx = D(W.active_set(n, na, 3000 + na)) if na < n else D(np.arange(n, dtype=np.int32))
        o = dict(acc=torch.empty((na, 3), dtype=torch.float64, device=dev),
                 jerk=torch.empty((na, 3), dtype=torch.float64, device=dev),
                 pot=torch.empty(na, dtype=torch.float64, device=dev),
                 nn_id=torch.empty(na, dtype=torch.int32, device=dev),
                 nn_r2=torch.empty(na, dtype=torch.float64, device=dev))
        h2 = torch.full((na,), 2.5e-3, dtype=torch.float64, device=dev)
        cnt = torch.empty(na, dtype=torch.int32, device=dev)
        lst = torch.empty((na, 256), dtype=torch.int32, device=dev)
        c.autotune(na)
        ms0 = timed(lambda: (c.predict(1.0), c.compute(idx, **o)), 3, stream)
        ms1 = timed(lambda: (c.predict(1.0), c.compute_nb(idx, h2, 256, cnt, lst, **o)), 3, stream)
        cc = cnt.cpu().numpy()
        rows.append({"n_active": na, "us_per_step_no_lists": 1e3 * ms0, "us_per_step_with_lists": 1e3 * ms1,
                     "interactions_per_s_with_lists": na * n / (ms1 / 1e3), "list_overhead": ms1 / ms0,
                     "mean_neighbours": float(cc.mean()), "max_neighbours": int(cc.max()),
                     "overflowed": int((cc > 256).sum())})
    c.close()
    return rows


# FP32 FMA-pipe lane-operations of a leap-frog (order 2) interaction: 9 double-
# single difference, 3 r^2, 1 softening add, 4 (rinv^2, m rinv, m rinv^3,
# potential sum), 3 acc.
OPS_PER_INTERACTION_H2 = 20


def bench_h2(sp2, dev, stream):
    """Leap-frog / GRAPE-5 pass (order 2: acc + pot + NN of sources at their
    stored positions), Plummer N = 131072: mixed at N_active = 131072 and
    16384, FP64 at 16384."""
    import torch
    n = 131072
    m, x, _ = W.plummer(n, 0)
    ids = W.particle_ids(n)
    D = lambda q: torch.as_tensor(np.ascontiguousarray(q)).to(dev)  # noqa: E731
    props = torch.cuda.get_device_properties(dev)
    peak = props.multi_processor_count * 128 * peaks().get("sm_max_mhz", 2070.0) * 1e6
    rows = []
    for prec, name, actives in ((sp2.SP2_MIXED, "mixed", (131072, 16384)), (sp2.SP2_FP64, "fp64", (16384,))):
        c = sp2.Context(order=2, precision=prec, n_max=n, eps2=1e-8, cuda_stream=stream.cuda_stream)
        c.set_j(0, D(ids), D(m), D(x), None, None, None, None, None)
        c.predict(0.0)
        for na in actives:
            idx = D(W.active_set(n, na, 4000 + na)) if na < n else D(np.arange(n, dtype=np.int32))
            o = dict(acc=torch.empty((na, 3), dtype=torch.float64, device=dev),
                     pot=torch.empty(na, dtype=torch.float64, device=dev),
                     nn_id=torch.empty(na, dtype=torch.int32, device=dev),
                     nn_r2=torch.empty(na, dtype=torch.float64, device=dev))
            c.autotune(na)
            ms = timed(lambda: (c.predict(0.0), c.compute(idx, **o)), 3 if name == "fp64" else 10, stream)
            rate = na * n / (ms / 1e3)
            row = {"precision": name, "n_active": na, "us_per_step": 1e3 * ms, "interactions_per_s": rate}
            if name == "mixed":
                row["fma_pipe_frac"] = rate * OPS_PER_INTERACTION_H2 / peak
            rows.append(row)
        c.close()
    return rows


def bench_blk(sp2, dev, stream, n=16384, t_end=0.25):
    """Block time-step Hermite-4 (Aarseth criterion, eta = 0.01, steps <= 1/16)
    on a Plummer sphere, eps = 1e-3, mixed and FP64: wall time, blocks, mean
    N_active and the relative energy error at t_end (energies evaluated with
    an FP64 context of the library)."""
    import time
    import torch
    eps2 = 1e-6
    m, x, v = W.plummer(n, 21)
    ids = np.arange(n, dtype=np.int32)
    z = np.zeros((n, 3))

    def energy(xx, vv):
        c = sp2.Context(order=4, precision=sp2.SP2_FP64, n_max=n, eps2=eps2, with_nn=0,
                        cuda_stream=stream.cuda_stream)
        c.set_j(0, ids, m, xx, vv, z, z, None, np.zeros(n))
        c.predict(0.0)
        pot = np.empty(n)
        c.compute(ids, pot=pot)
        c.close()
        return 0.5 * float(np.sum(m * np.sum(vv * vv, axis=1))) + 0.5 * float(np.sum(m * pot))

    e0 = energy(x, v)
    rows = []
    for prec, name in ((sp2.SP2_MIXED, "mixed"), (sp2.SP2_FP64, "fp64")):
        c = sp2.Context(order=4, precision=prec, n_max=n, eps2=eps2, with_nn=0, cuda_stream=stream.cuda_stream)
        c.set_j(0, ids, m, x, v, z, z, None, np.zeros(n))
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        c.block_init(0.0, 0.01, 1.0 / 16)
        st = c.block_run(t_end, 0.01, 1.0 / 16)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        xs, vs = np.empty((n, 3)), np.empty((n, 3))
        c.get_j(0, n, x=xs, v=vs)
        c.close()
        rows.append({"precision": name, "n": n, "t_end": t_end, "wall_s": wall, "block_steps": st["block_steps"],
                     "mean_active": st["active_sum"] / max(st["block_steps"], 1),
                     "interactions_per_s": st["active_sum"] * n / wall,
                     "energy_error": abs(energy(xs, vs) / e0 - 1.0)})
    return rows


def bench_blk6(sp2, dev, stream, n=16384, t_end=1.0, eps=1e-3):
    """6th-order block time-steps with the averaged criterion (eta4 = 0.01,
    eta6 = 0.1, steps <= 1/16; the scheme and parameters of Sec. 3.7, one
    N-body time unit by default) on a Plummer sphere (softening eps), mixed and
    FP64: wall time, blocks, mean / min / max N_active and the relative energy
    error at t_end (energies from an FP64 context of the library), or the
    time at which a run stopped on the step-underflow guard."""
    import time
    import torch
    eps2 = eps * eps
    m, x, v = W.plummer(n, 21)
    ids = np.arange(n, dtype=np.int32)
    z = np.zeros((n, 3))

    def energy(xx, vv):
        c = sp2.Context(order=4, precision=sp2.SP2_FP64, n_max=n, eps2=eps2, with_nn=0,
                        cuda_stream=stream.cuda_stream)
        c.set_j(0, ids, m, xx, vv, z, z, None, np.zeros(n))
        c.predict(0.0)
        pot = np.empty(n)
        c.compute(ids, pot=pot)
        c.close()
        return 0.5 * float(np.sum(m * np.sum(vv * vv, axis=1))) + 0.5 * float(np.sum(m * pot))

    e0 = energy(x, v)
    rows = []
    for prec, name in ((sp2.SP2_MIXED, "mixed"), (sp2.SP2_FP64, "fp64")):
        c = sp2.Context(order=6, precision=prec, n_max=n, eps2=eps2, with_nn=0, cuda_stream=stream.cuda_stream)
        c.set_j(0, ids, m, x, v, z, z, z, np.zeros(n))
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        c.block_init(0.0, 0.01, 1.0 / 16)
        try:
            st = c.block_run_h6(t_end, 0.01, 0.1, 1.0 / 16)
        except sp2.SP2Error as e:  # step underflow (the collapse Sec. 3.7 warns of for DS forces)
            torch.cuda.synchronize()
            st = getattr(e, "stats", {})
            rows.append({"precision": name, "n": n, "eps": eps, "t_end": t_end, "wall_s": time.perf_counter() - w0,
                         "stopped": str(e), "stopped_at_t": st.get("t"), "block_steps": st.get("block_steps"),
                         "mean_active": st.get("active_sum", 0) / max(st.get("block_steps") or 1, 1)})
            c.close()
            continue
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        xs, vs = np.empty((n, 3)), np.empty((n, 3))
        c.get_j(0, n, x=xs, v=vs)
        c.close()
        rows.append({"precision": name, "n": n, "eps": eps, "t_end": t_end, "wall_s": wall, "block_steps": st["block_steps"],
                     "mean_active": st["active_sum"] / max(st["block_steps"], 1),
                     "min_active": st["min_active"], "max_active": st["max_active"],
                     "us_per_block": 1e6 * wall / max(st["block_steps"], 1),
                     "interactions_per_s": st["active_sum"] * n / wall,
                     "energy_error": abs(energy(xs, vs) / e0 - 1.0)})
    return rows


def bench_batched(sp2, dev, stream):
    import torch
    offsets, m, x, v = W.planetary_systems(4096, 7)
    total = int(offsets[-1])
    z = np.zeros((total, 3))
    ids = W.particle_ids(total)
    D = lambda q: torch.as_tensor(np.ascontiguousarray(q)).to(dev)  # noqa: E731
    c = sp2.Context(order=4, precision=sp2.SP2_MIXED, n_max=total, eps2=0.0, cuda_stream=stream.cuda_stream)
    c.set_j(0, D(ids), D(m), D(x), D(v), D(z), D(z), None, D(np.zeros(total)))
    c.predict(0.0)
    plan = c.batch_plan(offsets)
    o = dict(acc=torch.empty((total, 3), dtype=torch.float64, device=dev),
             jerk=torch.empty((total, 3), dtype=torch.float64, device=dev),
             pot=torch.empty(total, dtype=torch.float64, device=dev),
             nn_id=torch.empty(total, dtype=torch.int32, device=dev),
             nn_r2=torch.empty(total, dtype=torch.float64, device=dev))
    one = lambda: c.compute_batched(plan, **o)  # noqa: E731
    sp2.sp2_graph_begin(c.ctx)
    c.predict(0.0)
    one()
    g = sp2.sp2_graph_end(c.ctx)
    g_ms = timed(lambda: sp2.sp2_graph_launch(c.ctx, g), 20, stream)
    k_ms = timed(one, 20, stream)
    slots = D(np.arange(total, dtype=np.int32))

    def per_system():
        for s in range(4096):
            a, b = int(offsets[s]), int(offsets[s + 1])
            c.compute(slots[a:b], j_range=(a, b), acc=o["acc"][a:b], jerk=o["jerk"][a:b], pot=o["pot"][a:b],
                      nn_id=o["nn_id"][a:b], nn_r2=o["nn_r2"][a:b])

    s_ms = timed(per_system, 3, stream)
    # the same 4096 per-system passes captured once and replayed as one CUDA
    # graph: the launches' GPU-side cost without the host loop in between
    sp2.sp2_graph_begin(c.ctx)
    per_system()
    gs = sp2.sp2_graph_end(c.ctx)
    gs_ms = timed(lambda: sp2.sp2_graph_launch(c.ctx, gs), 5, stream)
    sp2.sp2_graph_destroy(gs)
    sp2.sp2_graph_destroy(g)
    sp2.sp2_batch_plan_destroy(plan)
    c.close()
    inter = float(np.sum(np.diff(offsets) ** 2))
    return {"systems": 4096, "bodies": total, "interactions": inter, "batched_us": 1e3 * k_ms,
            "batched_graph_us_incl_predict": 1e3 * g_ms, "per_system_launches_us": 1e3 * s_ms,
            "per_system_graph_us": 1e3 * gs_ms, "speedup_vs_per_system_graph": gs_ms / k_ms,
            "speedup_vs_per_system": s_ms / k_ms, "interactions_per_s": inter / (k_ms / 1e3)}


def bench_adjoint(dev, stream):
    import torch
    from paper_1510_04068_gb300 import autograd as AG
    n, steps, dt = 16384, 32, 1.0 / 256
    m, x, v = W.plummer(n, 5)
    w = np.random.default_rng(1005).standard_normal((n, 3))
    T = lambda q: torch.as_tensor(q, device=dev)  # noqa: E731
    x0, v0, mm = T(x).requires_grad_(True), T(v).requires_grad_(True), T(m).requires_grad_(True)
    ww = T(w)
    sim = AG.HermiteSim(n, eps2=1e-6, precision="mixed", stream=stream)
    # one untimed pass loads every kernel module the trajectory uses
    xw, _ = sim.trajectory(x0, v0, mm, dt, 2, checkpoint_every=1)
    (ww * xw).sum().backward()
    x0.grad = v0.grad = mm.grad = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xf, vf = sim.trajectory(x0, v0, mm, dt, steps, checkpoint_every=8)
    loss = (ww * xf).sum()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    sim.close()
    inter = n * n * steps
    return {"n": n, "steps": steps, "forward_ms": 1e3 * (t1 - t0), "backward_ms": 1e3 * (t2 - t1),
            "forward_interactions_per_s": inter / (t1 - t0), "backward_over_forward": (t2 - t1) / (t1 - t0)}


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
