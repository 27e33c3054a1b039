"""Benchmark: indexed k-means on the 3D LiDAR-like workload (n = 1e7 float32
points, k = 1e4, 30 fixed Lloyd iterations, seeded-permutation init).

One step = the whole hot path on one batch: dkm_setup (bounding box, Morton
sort into tiles, tile boxes) + dkm_run (30 passes of candidate search,
assignment and update, then labels back to input order and the final SSE).
value = n * iterations / step time (point-iterations per second).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (plain brute-force Lloyd) on a
bounded sample of the same workload on the host cores.
For N > 1 (torchrun) every rank runs an independent replica (weak scaling).
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import os
import signal
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "point-iterations/s"
WORKLOAD = dict(workload="lidar3d", n=10_000_000, d=3, k=10_000, iterations=30,
                init="first k of a seeded permutation", seed=3,
                l2="inputs larger than L2 (120 MB of points, 160 MB moved per pass)")
FALLBACK_HBM_GBS = 6800.0
# algorithmic bytes of one k_assign launch per point: read x, y, z (12 B) and
# write the label (4 B); no previous-label read in fixed-iteration runs
ASSIGN_BYTES_PER_POINT = 16
# DRAM bytes (read + write) of one k_assign launch from the committed ncu
# capture, valid only while the kernel source is unchanged
NCU_TRAFFIC = {"sha": "6646a5afc6f4a134", "bytes_per_launch": 129_772_800 + 23_162_880,
               "source": "profiles/k_assign_lidar3d_n1e7_k1e4.md"}


def kernel_sha() -> str:
    h = hashlib.sha256()
    for f in ("dkm_iter.cu", "dkm_device.cuh"):
        with open(os.path.join(ROOT, "paper_2412_02244_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples.  Started before the warm-up (the
    tool's start-up must not overlap the timed region); summary() keeps the
    samples taken inside the timed window (the nearest ones if none)."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="dkm_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, window=None):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 10:
                        rows.append(parts)
        except Exception:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.remove(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        if window is not None:
            def ts(r):
                try:
                    return datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    return None
            stamped = [(ts(r), r) for r in rows]
            inside = [r for t, r in stamped if t is not None and window[0] <= t <= window[1]]
            if inside:
                rows = inside
            else:   # a timed region shorter than the poll interval: the nearest sample
                mid = 0.5 * (window[0] + window[1])
                near = [(abs(t - mid), r) for t, r in stamped if t is not None]
                rows = [min(near, key=lambda x: x[0])[1]] if near else rows
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(step_times_s, n: int, iters: int, world: int):
    """Whole-job throughput: every rank processed n*iters point-iterations per
    step; the job's step time is the slowest rank's."""
    t = float(max(step_times_s))
    return world * n * iters / t, t


def load_workload():
    from paper_2412_02244_gb300 import synth
    return synth.lidar3d(seed=WORKLOAD["seed"], n=WORKLOAD["n"], k=WORKLOAD["k"],
                         max_iter=WORKLOAD["iterations"])


def cpu_sample_run(w, m: int, seed: int = 0):
    """The oracle as it stands on a bounded sample: one Lloyd iteration
    (brute-force FP64 assignment against all k centroids + update) of m
    points drawn from the workload.  Returns (point-iterations/s, seconds,
    threads)."""
    import oracle
    o = oracle.get()
    if m >= w.n:
        m = w.n
        sample = w.points
    else:
        rng = np.random.default_rng(seed)
        idx = rng.choice(w.n, size=m, replace=False)
        sample = np.ascontiguousarray(w.points[idx])
    t0 = time.perf_counter()
    o.fit(sample, w.init.astype(np.float64), 1, early_stop=False)
    dt = time.perf_counter() - t0
    return m / dt, dt, o.num_threads()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = load_workload()
    m = args.ref_sample
    vals = []
    for s in range(args.warmup + args.steps):
        v, dt, thr = cpu_sample_run(w, m, seed=s)
        if s >= args.warmup:
            vals.append((v, dt))
    value = float(np.median([v for v, _ in vals]))
    t_step = float(np.median([dt for _, dt in vals]))
    sample = (f"one Lloyd iteration (FP64 brute-force assignment against all k=10000 "
              f"centroids + update) of {m} points drawn from the n=1e7 workload, per step")
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": WORKLOAD, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": thr, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def launches_per_step(iters: int) -> int:
    # dkm_setup: reset_boxes, bbox, lattice, morton (with the sort's digit counts), 3
    # one-sweep radix-sort passes over the top 24 key bits, gather, levels, choose_levels,
    # tiles (count, scan, ranges and boxes)
    setup = 2 + 1 + 1 + 3 + 1 + 1 + 1 + 3
    # dkm_run: centroid reset_boxes + bbox + exponents; graph: reset_run, prep,
    # iters x (search, assign, centroids); finalize, collect, export
    run = 3 + 2 + 3 * iters + 3
    return setup + run


DEFAULT_TUNING = dict(cells_per_centroid=1.0, tile_cut_div=8, row_filter_min=48, sort_max=0,
                      tile_group=1, stay_test=0)
ABLATIONS = [
    ("stay_test (bound layer)", {"stay_test": 1}),
    ("tile_group 4 (hierarchical tiles)", {"tile_group": 4}),
    ("tile_group 8 (hierarchical tiles)", {"tile_group": 8}),
    ("sort_max 32 (sorted early exit)", {"sort_max": 32}),
    ("row_filter_min 48 (per-row refilter)", {"row_filter_min": 48}),
    ("tile_cut_div 8 (coarser tiles)", {"tile_cut_div": 8}),
    ("cells_per_centroid 2", {"cells_per_centroid": 2.0}),
]


def bench_ablations(dkm, pts, n, d, k, C, stream, tune):
    """Per-pass time of one Lloyd pass from the given centroids under each
    setting (the tuned one, then single changes from it)."""
    import torch
    o = dkm.dkm_default_options(early_stop=0, profile=1, stream=stream.cuda_stream)
    ctx = dkm.dkm_create(pts, n, d, k, o)
    base = dkm.dkm_get_tuning(ctx) if tune is None else tune
    C2 = torch.empty_like(C)
    lab = torch.empty(n, dtype=torch.int32, device=pts.device)
    out = []
    for name, change in [("tuned", {})] + ABLATIONS + [("defaults", DEFAULT_TUNING)]:
        t = dkm.dkm_tuning()
        for f, _ in dkm.dkm_tuning._fields_:
            setattr(t, f, getattr(base, f))
        for key, v in change.items():
            setattr(t, key, v)
        dkm.dkm_set_tuning(ctx, t)
        ms = []
        for _ in range(3):
            dkm.dkm_run(ctx, C, 1, C2, lab)
            T = dkm.dkm_last_timings(ctx)
            ms.append(T.search_ms + T.assign_ms + T.update_ms)
        st = dkm.dkm_last_stats(ctx)
        out.append({"setting": name, "ms_per_pass": float(np.median(ms[1:])),
                    "evals_per_point": st.evals_per_point,
                    "candidates_per_tile": st.candidates_per_tile, "tiles": st.tiles,
                    "stayed_tiles": st.stayed_tiles})
    ctx.close()
    return {"from": "one pass from the timed run's final centroids per setting",
            "settings": out}


BATCHED = dict(workload="batched3d", clouds=512, n_i="round(2^U[10,17])",
               k_i="max(8, n_i // 100)", d=3, iterations=25, seed=4)
SOFT = dict(workload="soft3d", clouds=64, n_i=16384, k=256, d=3, T=10, seed=5)


def bench_batched(dkm, torch, dev, stream, steps: int, hbm: float):
    """The uneven-batch workload: 512 clouds in one context, autotuned index,
    25 fixed passes per step (dkm_setup + dkm_run_batched), plus the same
    passes by brute force from the run's final centroids."""
    from paper_2412_02244_gb300 import synth
    ws = synth.batched3d(seed=BATCHED["seed"])
    P = np.ascontiguousarray(np.concatenate([w.points for w in ws]).astype(np.float32))
    off = np.zeros(len(ws) + 1, np.int64)
    off[1:] = np.cumsum([w.n for w in ws])
    ks = np.array([w.k for w in ws], np.int32)
    init = np.ascontiguousarray(np.concatenate([w.init for w in ws]).astype(np.float32))
    n, K, it = int(off[-1]), int(ks.sum()), BATCHED["iterations"]
    pts = torch.from_numpy(P).to(dev)
    ini = torch.from_numpy(init).to(dev)
    C = torch.empty(K * 3, dtype=torch.float32, device=dev)
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    opts = dkm.dkm_default_options(early_stop=0, profile=it, stream=stream.cuda_stream)
    ctx = dkm.dkm_create_batched(pts, off, 3, ks, opts)
    tune = dkm.dkm_autotune(ctx, ini, passes=3, use_cache=False)

    def step():
        dkm.dkm_setup(ctx, pts)
        return dkm.dkm_run_batched(ctx, ini, it, C, lab)

    for _ in range(2):
        step()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    a_ms, s_ms, u_ms, setup_ms = [], [], [], []
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    T = dkm.dkm_last_timings(ctx)   # the last timed step's profiled (middle) pass
    a_ms.append(T.assign_ms)
    s_ms.append(T.search_ms)
    u_ms.append(T.update_ms)
    setup_ms.append(T.setup_ms)
    t_step = ev0.elapsed_time(ev1) / 1e3 / steps
    st = dkm.dkm_last_stats(ctx)
    per_pass = float(np.mean(s_ms) + np.mean(a_ms) + np.mean(u_ms))
    ob = dkm.dkm_default_options(early_stop=0, profile=1, algo=dkm.DKM_ALGO_BRUTE,
                                 stream=stream.cuda_stream)
    cb = dkm.dkm_create_batched(pts, off, 3, ks, ob)
    Cb = torch.empty(K * 3, dtype=torch.float32, device=dev)
    lb = torch.empty(n, dtype=torch.int32, device=dev)
    dkm.dkm_run_batched(cb, C, 2, Cb, lb)
    Tb = dkm.dkm_last_timings(cb)
    dkm.dkm_run_batched(ctx, C, 2, Cb, lb)
    Ti = dkm.dkm_last_timings(ctx)
    per_b = Tb.search_ms + Tb.assign_ms + Tb.update_ms
    per_i = Ti.search_ms + Ti.assign_ms + Ti.update_ms
    cb.close()
    ctx.close()
    am = float(np.mean(a_ms))
    achieved = n * ASSIGN_BYTES_PER_POINT / (am * 1e-3) / 1e9
    return {"config": dict(BATCHED, n_total=n, k_total=K),
            "value": n * it / t_step, "unit": METRIC, "ms_per_step": t_step * 1e3,
            "per_pass_ms": per_pass, "search_ms": float(np.mean(s_ms)), "assign_ms": am,
            "update_ms": float(np.mean(u_ms)), "setup_ms": float(np.mean(setup_ms)),
            "roofline_k_assign": {"bound": "hbm", "achieved": achieved, "peak": hbm,
                                  "unit": "GB/s", "frac": achieved / hbm},
            "tuning": {"cells_per_centroid": tune.cells_per_centroid,
                       "tile_cut_div": tune.tile_cut_div, "row_filter_min": tune.row_filter_min,
                       "sort_max": tune.sort_max, "tile_group": tune.tile_group,
                       "stay_test": tune.stay_test,
                       "ms_per_pass": tune.ms_per_pass,
                       "ms_per_pass_default": tune.ms_per_pass_before, "trials": tune.trials},
            "pruning": {"evals_per_point": st.evals_per_point,
                        "candidates_per_tile": st.candidates_per_tile, "tiles": st.tiles,
                        "stayed_tiles": st.stayed_tiles},
            "brute_force": {"ms_per_pass": per_b, "indexed_ms_per_pass": per_i,
                            "speedup_indexed_over_brute": per_b / per_i if per_i > 0 else None,
                            "from": "final centroids of the timed run, 2 passes each"},
            "launches_per_pass": 3}


def bench_soft(dkm, torch, dev, stream, steps: int):
    """The differentiable workload: 64 clouds x 16384 points, k = 256; soft
    k-means with T = 10 unrolled steps forward + backward, and the hard SSE
    with its gradient."""
    from paper_2412_02244_gb300 import synth
    from paper_2412_02244_gb300.autograd import temperature
    ws = synth.soft3d(seed=SOFT["seed"], n_clouds=SOFT["clouds"])
    P = torch.from_numpy(np.concatenate([w.points for w in ws])).to(dev)
    init = torch.from_numpy(np.stack([w.init for w in ws])).to(dev)
    B, k, T = SOFT["clouds"], SOFT["k"], SOFT["T"]
    off = np.zeros(B + 1, np.int64)
    off[1:] = np.cumsum([w.n for w in ws])
    tau = temperature(P, torch.from_numpy(off)).numpy()
    ck = torch.empty((T + 1, B, k, 3), dtype=torch.float32, device=dev)
    loss = torch.empty(B, dtype=torch.float64, device=dev)
    gp = torch.empty_like(P)
    gi = torch.empty_like(init)
    gc = torch.empty_like(init)
    stats = torch.empty((T, 2, P.shape[0]), dtype=torch.float32, device=dev)
    norms = torch.empty((T, B, k), dtype=torch.float32, device=dev)
    dl = np.ones(B)
    s = stream.cuda_stream

    def fwd_bwd():
        dkm.dkm_soft_forward(P, off, B, 3, k, init, T, tau, ck, loss, s, stats=stats, norms=norms)
        dkm.dkm_soft_backward(P, off, B, 3, k, ck, T, tau, dl, gp, gi, s, stats=stats, norms=norms)

    def hard():
        dkm.dkm_hard_sse(P, off, B, 3, k, init, None, loss, gp, gc, s)

    out = {"config": SOFT}
    for name, fn in (("soft_forward_backward_ms", fwd_bwd), ("hard_sse_with_grad_ms", hard)):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) / steps
    n = int(off[-1])
    # forward: T + 1 weight passes over n x k distances; backward: recompute
    # + adjoint, about 3 passes per step
    out["soft_point_centroid_pairs_per_s"] = n * k * (T + 1) / (out["soft_forward_backward_ms"] * 1e-3)
    return out


def run_ours(args):
    import torch
    from paper_2412_02244_gb300 import build as b
    b.build()
    from paper_2412_02244_gb300 import dkm

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = load_workload()
    n, d, k, iters = w.n, w.d, w.k, WORKLOAD["iterations"]
    stream = torch.cuda.Stream(device=dev)
    pts = torch.from_numpy(w.points).to(dev)
    init = torch.from_numpy(w.init).to(dev)
    C = torch.empty(k * d, dtype=torch.float32, device=dev)
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    # one profiled pass per step (the middle one): the events around its
    # kernels give the per-kernel times inside the timed region, and a
    # single profiled pass keeps their cost to the step at about 1%
    opts = dkm.dkm_default_options(early_stop=0, profile=iters if args.profile else 0,
                                   stream=stream.cuda_stream)
    torch.cuda.synchronize()
    ctx = dkm.dkm_create(pts, n, d, k, opts)
    # index settings measured by the autotuner, once, before the warm-up, or
    # given explicitly (--set, e.g. to profile the tuned configuration)
    tune = None
    if args.set:
        kw = {}
        for item in args.set.split(","):
            key, v = item.split("=")
            kw[key] = float(v) if key == "cells_per_centroid" else int(v)
        dkm.dkm_set_tuning(ctx, **kw)
        tune = dkm.dkm_get_tuning(ctx)
    elif args.tune:
        tune = dkm.dkm_autotune(ctx, init, passes=3, use_cache=False)

    def step():
        dkm.dkm_setup(ctx, pts)
        return dkm.dkm_run(ctx, init, iters, C, lab)

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    assign_ms, search_ms, update_ms, setup_ms = [], [], [], []
    # the clock sampler starts before the warm-up: its start-up (NVML
    # initialisation) would otherwise overlap the timed steps
    with ClockSampler(local) as clk:
        time.sleep(0.5)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        w0 = time.time()
        ev0.record(stream)
        for _ in range(args.steps):
            it, sse = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        w1 = time.time()
        time.sleep(0.25)   # let a sample land after the window (for short timed regions)
    if args.profile:
        # per-kernel times of the last timed step (CUDA events around the
        # kernels of its middle pass, recorded inside the captured graph)
        T = dkm.dkm_last_timings(ctx)
        assign_ms.append(T.assign_ms)
        search_ms.append(T.search_ms)
        update_ms.append(T.update_ms)
        setup_ms.append(T.setup_ms)
    t_step = ev0.elapsed_time(ev1) / 1e3 / args.steps
    times = [t_step]
    if dist:
        tt = torch.tensor([t_step], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        times = [float(tt.item())]
    value, t_job = aggregate(times, n, iters, ws)
    stats = dkm.dkm_last_stats(ctx)

    # end to end through the public API with host (pinned) buffers
    pts_h = torch.from_numpy(w.points).pin_memory()
    init_h = torch.from_numpy(w.init).pin_memory()
    C_h = torch.empty(k * d, dtype=torch.float32).pin_memory()
    lab_h = torch.empty(n, dtype=torch.int32).pin_memory()
    dkm.dkm_setup(ctx, pts_h)
    dkm.dkm_run(ctx, init_h, iters, C_h, lab_h)
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        dkm.dkm_setup(ctx, pts_h)
        dkm.dkm_run(ctx, init_h, iters, C_h, lab_h)
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / e2e_steps
    if dist:
        tt = torch.tensor([t_e2e], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_e2e = float(tt.item())
    e2e_value = ws * n * iters / t_e2e

    # brute-force Lloyd on the same GPU, from the same converged centroids
    brute = None
    if rank == 0 and not args.no_brute:
        ob = dkm.dkm_default_options(early_stop=0, profile=1, algo=dkm.DKM_ALGO_BRUTE,
                                     stream=stream.cuda_stream)
        cb = dkm.dkm_create(pts, n, d, k, ob)
        Cb = torch.empty(k * d, dtype=torch.float32, device=dev)
        lb = torch.empty(n, dtype=torch.int32, device=dev)
        dkm.dkm_run(cb, C, 2, Cb, lb)
        Tb = dkm.dkm_last_timings(cb)
        oi = dkm.dkm_default_options(early_stop=0, profile=1, stream=stream.cuda_stream)
        ci = dkm.dkm_create(pts, n, d, k, oi)
        if tune is not None:
            dkm.dkm_set_tuning(ci, tune)
        dkm.dkm_run(ci, C, 2, Cb, lb)
        dkm.dkm_run(ci, C, 2, Cb, lb)
        Ti = dkm.dkm_last_timings(ci)
        per_b = Tb.search_ms + Tb.assign_ms + Tb.update_ms
        per_i = Ti.search_ms + Ti.assign_ms + Ti.update_ms
        brute = {"ms_per_iteration": per_b, "indexed_ms_per_iteration": per_i,
                 "speedup_indexed_over_brute": per_b / per_i if per_i > 0 else None,
                 "from": "converged centroids of the timed run, 2 passes each"}
        cb.close()
        ci.close()

    # measured effect of each index option on this workload: one pass from
    # the run's final centroids per setting, on a fresh context
    ablations = None
    if rank == 0 and not args.no_extra:
        ablations = bench_ablations(dkm, pts, n, d, k, C, stream, tune)

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return 0
    hbm, src = peaks()
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_job * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": WORKLOAD}
    if args.profile and assign_ms:
        a_ms = float(np.mean(assign_ms))
        achieved = n * ASSIGN_BYTES_PER_POINT / (a_ms * 1e-3) / 1e9
        traffic = None
        if NCU_TRAFFIC and NCU_TRAFFIC.get("sha") == kernel_sha():
            traffic = NCU_TRAFFIC["bytes_per_launch"]
        line["roofline"] = {"bound": "hbm", "kernel": "k_assign", "achieved": achieved,
                            "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                            "peak_source": src, "traffic": traffic,
                            "algorithmic_bytes_per_launch": n * ASSIGN_BYTES_PER_POINT,
                            "launch_ms": a_ms}
        per_iter = float(np.mean(search_ms) + np.mean(assign_ms) + np.mean(update_ms))
        line["per_iteration"] = {"ms": per_iter, "search_ms": float(np.mean(search_ms)),
                                 "assign_ms": a_ms, "update_ms": float(np.mean(update_ms)),
                                 "point_iterations_per_s": n / (per_iter * 1e-3),
                                 "hbm_frac_of_iteration": n * ASSIGN_BYTES_PER_POINT
                                 / (per_iter * 1e-3) / 1e9 / hbm,
                                 "setup_ms": float(np.mean(setup_ms))}
    if tune is not None:
        line["tuning"] = {"cells_per_centroid": tune.cells_per_centroid,
                          "tile_cut_div": tune.tile_cut_div,
                          "row_filter_min": tune.row_filter_min, "sort_max": tune.sort_max,
                          "tile_group": tune.tile_group, "stay_test": tune.stay_test,
                          "ms_per_pass": tune.ms_per_pass,
                          "ms_per_pass_default": tune.ms_per_pass_before, "trials": tune.trials,
                          "note": ("given with --set" if args.set else
                                   "chosen by dkm_autotune before the warm-up, outside the "
                                   "timed region")}
    line["pruning"] = {"evals_per_point": stats.evals_per_point,
                       "candidates_per_tile": stats.candidates_per_tile,
                       "fallback_tiles": stats.fallback_tiles,
                       "stayed_tiles": stats.stayed_tiles,
                       "tiles": stats.tiles, "tile_level": stats.tile_level,
                       "grid_overflow": stats.grid_overflow}
    if brute:
        line["brute_force"] = brute
    line["e2e"] = {"value": e2e_value, "unit": METRIC,
                   "h2d_bytes_per_step": n * d * 4 + k * d * 4,
                   "d2h_bytes_per_step": n * 4 + k * d * 4, "steps": e2e_steps}
    line["gpu_launches"] = launches_per_step(iters) * args.steps
    line["clocks"] = clk.summary(window=(w0, w1))
    if ws == 1 and not args.no_cpu_baseline:
        v, dt, thr = cpu_sample_run(w, args.cpu_sample)
        line["cpu_baseline"] = {"value": v, "unit": METRIC, "cores": thr, "kind": "oracle",
                                "sample": f"one FP64 brute-force Lloyd iteration (assignment "
                                          f"against all k=10000 centroids + update) of "
                                          f"{min(args.cpu_sample, n)} of the workload's {n} "
                                          f"points ({dt:.1f} s)"}
    if ablations:
        line["ablations"] = ablations
    if ws == 1 and not args.no_extra:
        ctx.close()
        line["batched"] = bench_batched(dkm, torch, dev, stream, max(2, min(args.steps, 5)), hbm)
        line["differentiable"] = bench_soft(dkm, torch, dev, stream, max(2, min(args.steps, 5)))
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--profile", type=int, default=1,
                    help="record per-kernel CUDA events around the middle pass of every "
                         "timed step, inside the run graph (roofline)")
    ap.add_argument("--cpu-sample", type=int, default=10_000_000)
    ap.add_argument("--ref-sample", type=int, default=500_000)
    ap.add_argument("--no-brute", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune", type=int, default=1,
                    help="run dkm_autotune on the workload before the warm-up (0 = defaults)")
    ap.add_argument("--set", default="",
                    help="explicit index settings instead of the autotuner, e.g. "
                         "tile_cut_div=1,row_filter_min=256")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched-cloud and differentiable side measurements")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
