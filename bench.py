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
NCU_TRAFFIC = {"sha": "22bdb079b0baa2f4", "bytes_per_launch": 129_609_984 + 22_913_536,
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


class NvmlClocks:
    """SM clock, power and clock-event reasons read through NVML (the
    driver's libnvidia-ml, loaded with ctypes) every `period` seconds on a
    background thread: enough samples even inside a timed region of a
    fraction of a second.  Only reads; changes no setting."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, gpu: int, period: float = 0.01):
        import ctypes
        import threading
        self.ct = ctypes
        lib = None
        for name in ("libnvidia-ml.so.1", "libnvidia-ml.so"):
            try:
                lib = ctypes.CDLL(name)
                break
            except OSError:
                continue
        if lib is None or lib.nvmlInit_v2() != 0:
            raise RuntimeError("NVML not available")
        self.lib = lib
        cnt = ctypes.c_uint(0)
        lib.nvmlDeviceGetCount_v2(ctypes.byref(cnt))
        idx = gpu if cnt.value > gpu else 0
        self.h = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByIndex_v2(idx, ctypes.byref(self.h)) != 0:
            raise RuntimeError("NVML device handle")
        self.reason_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        mx = ctypes.c_uint(0)
        lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx))
        self.max_mhz = float(mx.value)
        self.period = period
        self.rows = []
        self.stop = threading.Event()
        self.thread = threading.Thread(target=self._loop, daemon=True)

    def _loop(self):
        ct = self.ct
        mhz, mw, rs = ct.c_uint(0), ct.c_uint(0), ct.c_ulonglong(0)
        while not self.stop.is_set():
            self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(mhz))
            self.lib.nvmlDeviceGetPowerUsage(self.h, ct.byref(mw))
            self.reason_fn(self.h, ct.byref(rs))
            self.rows.append((time.time(), float(mhz.value), mw.value / 1000.0, int(rs.value)))
            time.sleep(self.period)

    def start(self):
        self.thread.start()

    def finish(self):
        self.stop.set()
        self.thread.join(timeout=2)

    def summary(self, window):
        rows = [r for r in self.rows if window[0] <= r[0] <= window[1]]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["no samples"],
                    "samples": 0, "source": "nvml"}
        reasons = sorted({name for r in rows for bit, name in self.REASONS.items() if r[3] & bit})
        return {"sm_mhz": float(np.median([r[1] for r in rows])), "sm_max_mhz": self.max_mhz,
                "sm_mhz_min": min(r[1] for r in rows), "power_w_max": max(r[2] for r in rows),
                "reasons": reasons, "samples": len(rows), "source": "nvml",
                "period_ms": self.period * 1e3}


class ClockSampler:
    """Clock / throttle samples during the timed region: NVML every 10 ms
    when the driver library loads, else nvidia-smi every 100 ms.  Started
    before the warm-up (the tool's start-up must not overlap the timed
    steps); summary() keeps the samples taken inside the timed window (the
    nearest one if none)."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None
        self.nvml = None

    def __enter__(self):
        try:
            self.nvml = NvmlClocks(self.gpu)
            self.nvml.start()
            return self
        except Exception:
            self.nvml = None
        fd, self.path = tempfile.mkstemp(prefix="dkm_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.nvml is not None:
            self.nvml.finish()
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, window=None):
        if self.nvml is not None:
            return self.nvml.summary(window)
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
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "source": "nvidia-smi"}


def cpu_model() -> str:
    """The host CPU's model name (/proc/cpuinfo, else lscpu, else platform)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


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


def _oracle(single_thread: bool):
    """The oracle as it stands: the OpenMP build, or the same source built
    without OpenMP (one host thread)."""
    import oracle
    if not single_thread:
        return oracle.get()
    path = os.path.join(os.path.dirname(os.path.abspath(oracle.__file__)), "_build",
                        "libdkm_oracle_st.so")
    if not os.path.exists(path):
        oracle.build(out=path, openmp=False)
    return oracle.Oracle(path)


def cpu_sample_run(w, m: int, seed: int = 0, single_thread: bool = False):
    """The oracle as it stands on a bounded sample: one Lloyd iteration
    (brute-force FP64 assignment against all k centroids + update) of m
    points drawn from the workload.  Returns (point-iterations/s, seconds,
    threads)."""
    o = _oracle(single_thread)
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
    return m / dt, dt, (1 if single_thread else o.num_threads())


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


DEFAULT_TUNING = dict(cells_per_centroid=1.0, tile_cut_div=2, row_filter_min=48, sort_max=0,
                      tile_group=1, stay_test=0)
ABLATIONS = [
    ("stay_test 1 (bound layer: tile test)", {"stay_test": 1}),
    ("stay_test 2 (bound layer: tile and point tests)", {"stay_test": 2}),
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
                    "search_ms": T.search_ms, "assign_ms": T.assign_ms, "update_ms": T.update_ms,
                    "evals_per_point": st.evals_per_point,
                    "candidates_per_tile": st.candidates_per_tile, "tiles": st.tiles,
                    "stayed_tiles": st.stayed_tiles, "stayed_points": st.stayed_points,
                    "stayed_point_fraction": st.stayed_points / n})
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
    torch.cuda.synchronize()
    t_step, per = timed_steps(step, stream, steps, ctx, dkm)
    s_ms, a_ms, u_ms, setup_ms = (per[:, i] for i in range(4))
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
    # the bound layer's stay tests from the run's final centroids (two
    # passes, the second measured): how many tiles and points keep their label
    stays = []
    for level in (1, 2):
        t = dkm.dkm_get_tuning(ctx)
        dkm.dkm_set_tuning(ctx, tile_group=1, stay_test=level)
        dkm.dkm_run_batched(ctx, C, 2, Cb, lb)
        ss = dkm.dkm_last_stats(ctx)
        stays.append({"stay_test": level, "pass": 2,
                      "stayed_tiles": ss.stayed_tiles, "tiles": ss.tiles,
                      "stayed_points": ss.stayed_points, "stayed_point_fraction": ss.stayed_points / n,
                      "evals_per_point": ss.evals_per_point})
        dkm.dkm_set_tuning(ctx, t)
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
            "bound_layer": stays,
            "launches_per_pass": 3}


def bench_soft(dkm, torch, dev, stream, steps: int, peaks_dev=None):
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
    if peaks_dev is not None:
        fl = soft_flops_per_pair(T) * n * k
        ach = fl / (out["soft_forward_backward_ms"] * 1e-3) / 1e12
        pk2 = peaks_dev.fp32x2_fma_tflops
        out["alu_roofline"] = {"bound": "alu", "kernel": "soft forward + backward (all passes)",
                               "achieved": ach, "peak": pk2,
                               "unit": "TFLOP/s", "frac": ach / pk2,
                               "flops_per_pair": soft_flops_per_pair(T),
                               "peak_source": "measured packed f32x2 FMA rate (dkm_device_peaks); "
                                              "the soft passes use packed f32x2 arithmetic"}
        hf = BRUTE_FLOPS_PER_PAIR * n * k / (out["hard_sse_with_grad_ms"] * 1e-3) / 1e12
        out["hard_alu_roofline"] = {"bound": "alu", "achieved": hf,
                                    "peak": pk2, "unit": "TFLOP/s", "frac": hf / pk2,
                                    "flops_per_pair": BRUTE_FLOPS_PER_PAIR,
                                    "peak_source": "measured packed f32x2 FMA rate (the hard "
                                                   "row pass computes distances in packed "
                                                   "f32x2 arithmetic)"}
    return out


# FP32 floating-point operations per (point, centroid) pair, counted in the
# kernel source (an FMA counts 2, a min/compare 0, the exponential 1 for its
# argument scaling): distance 8; soft forward step 39 (row statistics 20,
# column mean 19), forward loss 34, backward loss stage 70 (row 47, column
# 23), backward step 82 with the forward's statistics (row 47, column 35).
BRUTE_FLOPS_PER_PAIR = 8


def soft_flops_per_pair(T: int) -> int:
    return 39 * T + 34 + 70 + 82 * T


def timed_steps(step, stream, steps, ctx, dkm):
    """Run `steps` steps between two CUDA events on the stream; after each
    step, read that step's profiled-pass kernel times (dkm_run returns after
    its outputs are ready, so this costs host microseconds)."""
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    per = []
    ev0.record(stream)
    for _ in range(steps):
        step()
        T = dkm.dkm_last_timings(ctx)
        per.append((T.search_ms, T.assign_ms, T.update_ms, T.setup_ms))
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / 1e3 / steps, np.array(per, np.float64)


def bench_2d(dkm, torch, dev, stream, name: str, steps: int, hbm: float):
    """A 2D side line (geo2d-blobs: early stop; geo2d-roads: 50 fixed
    passes): point-iterations/s with the index the autotuner picks, the
    per-pass HBM fraction and the brute-force ratio on the same GPU."""
    from paper_2412_02244_gb300 import synth
    w = synth.by_name(name)
    n, d, k = w.n, w.d, w.k
    early = 1 if name == "geo2d-blobs" else 0
    iters = 20 if early else 50
    # bytes per point of one assignment: the point, the label written, and
    # the previous label read when the early stop needs the change count
    bpp = 4 * d + 4 + (4 if early else 0)
    pts = torch.from_numpy(w.points).to(dev)
    init = torch.from_numpy(w.init).to(dev)
    C = torch.empty(k * d, dtype=torch.float32, device=dev)
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    opts = dkm.dkm_default_options(early_stop=early, profile=1, stream=stream.cuda_stream)
    ctx = dkm.dkm_create(pts, n, d, k, opts)
    tune = dkm.dkm_autotune(ctx, init, passes=3, use_cache=False)
    passes = [0]

    def step():
        dkm.dkm_setup(ctx, pts)
        it, _ = dkm.dkm_run(ctx, init, iters, C, lab)
        passes[0] = it

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    t_step, per = timed_steps(step, stream, steps, ctx, dkm)
    it = passes[0]
    s_ms, a_ms, u_ms = (float(per[:, i].mean()) for i in range(3))
    per_pass = s_ms + a_ms + u_ms
    ob = dkm.dkm_default_options(early_stop=0, profile=1, algo=dkm.DKM_ALGO_BRUTE,
                                 stream=stream.cuda_stream)
    cb = dkm.dkm_create(pts, n, d, k, ob)
    Cb = torch.empty(k * d, dtype=torch.float32, device=dev)
    lb = torch.empty(n, dtype=torch.int32, device=dev)
    dkm.dkm_run(cb, C, 2, Cb, lb)
    dkm.dkm_run(cb, C, 2, Cb, lb)
    Tb = dkm.dkm_last_timings(cb)
    per_b = Tb.search_ms + Tb.assign_ms + Tb.update_ms
    cb.close()
    ctx.close()
    return {"config": {"workload": name, "n": n, "d": d, "k": k,
                       "iterations": ("<= 20, early stop" if early else iters), "seed": w.seed},
            "value": n * it / t_step, "unit": METRIC, "ms_per_step": t_step * 1e3,
            "passes_per_step": it, "per_pass_ms": per_pass, "search_ms": s_ms, "assign_ms": a_ms,
            "update_ms": u_ms, "setup_ms": float(per[:, 3].mean()),
            "hbm_frac_per_pass": n * bpp / (per_pass * 1e-3) / 1e9 / hbm,
            "k_assign_hbm_frac": n * bpp / (a_ms * 1e-3) / 1e9 / hbm,
            "algorithmic_bytes_per_point": bpp,
            "brute_force": {"ms_per_pass": per_b,
                            "speedup_indexed_over_brute": per_b / per_pass if per_pass else None},
            "tuning": {"cells_per_centroid": tune.cells_per_centroid,
                       "tile_cut_div": tune.tile_cut_div, "row_filter_min": tune.row_filter_min,
                       "sort_max": tune.sort_max, "tile_group": tune.tile_group,
                       "stay_test": tune.stay_test}}


def bench_cold(dkm, torch, dev, stream, w, tune, iters):
    """The first step a one-shot user sees: a fresh context (candidate lists
    empty, so pass 1 searches from scratch), one dkm_setup + dkm_run timed
    with CUDA events; and dkm_fit end to end (create + run + destroy, device
    buffers) timed on the host."""
    n, d, k = w.n, w.d, w.k
    pts = torch.from_numpy(w.points).to(dev)
    init = torch.from_numpy(w.init).to(dev)
    C = torch.empty(k * d, dtype=torch.float32, device=dev)
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    opts = dkm.dkm_default_options(early_stop=0, profile=0, stream=stream.cuda_stream)
    ctx = dkm.dkm_create(pts, n, d, k, opts)
    if tune is not None:
        dkm.dkm_set_tuning(ctx, tune)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    dkm.dkm_setup(ctx, pts)
    dkm.dkm_run(ctx, init, iters, C, lab)
    e1.record(stream)
    torch.cuda.synchronize()
    cold_ms = e0.elapsed_time(e1)
    ctx.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dkm.dkm_fit(pts, n, d, k, init, iters, C, lab,
                dkm.dkm_default_options(early_stop=0, stream=stream.cuda_stream))
    torch.cuda.synchronize()
    fit_ms = (time.perf_counter() - t0) * 1e3
    return {"step_ms": cold_ms, "value": n * iters / (cold_ms * 1e-3), "unit": METRIC,
            "dkm_fit_ms": fit_ms,
            "what": "one dkm_setup + dkm_run on a fresh context (no candidate lists kept from "
                    "an earlier step; the autotuned setting applied); dkm_fit = create + run + "
                    "destroy with default settings, host wall time"}


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
        t_step, per = timed_steps(step, stream, args.steps, ctx, dkm)
        w1 = time.time()
        time.sleep(0.25)
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
    e2e_steps = max(3, min(args.steps, 10))
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

    peaks_dev = None
    try:
        peaks_dev = dkm.dkm_device_peaks(stream.cuda_stream)
    except Exception:
        peaks_dev = None

    # brute-force Lloyd on the same GPU, from the same converged centroids
    brute = None
    if rank == 0 and not args.no_brute:
        ob = dkm.dkm_default_options(early_stop=0, profile=1, algo=dkm.DKM_ALGO_BRUTE,
                                     stream=stream.cuda_stream)
        cb = dkm.dkm_create(pts, n, d, k, ob)
        Cb = torch.empty(k * d, dtype=torch.float32, device=dev)
        lb = torch.empty(n, dtype=torch.int32, device=dev)
        dkm.dkm_run(cb, C, 2, Cb, lb)
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
        if peaks_dev is not None and Tb.assign_ms > 0:
            ach = BRUTE_FLOPS_PER_PAIR * n * k / (Tb.assign_ms * 1e-3) / 1e12
            brute["alu_roofline"] = {
                "bound": "alu", "kernel": "k_assign (brute force)", "achieved": ach,
                "peak": peaks_dev.fp32x2_fma_tflops, "unit": "TFLOP/s",
                "frac": ach / peaks_dev.fp32x2_fma_tflops,
                "peak_source": "measured packed f32x2 FMA rate (dkm_device_peaks); the kernel's "
                               "distances use packed f32x2 arithmetic",
                "flops_per_pair": BRUTE_FLOPS_PER_PAIR}
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
    if args.profile and len(per):
        s_ms, a_ms, u_ms = (float(per[:, i].mean()) for i in range(3))
        achieved = n * ASSIGN_BYTES_PER_POINT / (a_ms * 1e-3) / 1e9
        traffic = None
        if NCU_TRAFFIC and NCU_TRAFFIC.get("sha") == kernel_sha():
            traffic = NCU_TRAFFIC["bytes_per_launch"]
        line["roofline"] = {"bound": "hbm", "kernel": "k_assign", "achieved": achieved,
                            "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                            "peak_source": src, "traffic": traffic,
                            "algorithmic_bytes_per_launch": n * ASSIGN_BYTES_PER_POINT,
                            "launch_ms": a_ms, "launch_ms_min": float(per[:, 1].min()),
                            "launch_ms_max": float(per[:, 1].max()),
                            "launches_averaged": int(len(per)),
                            "how": "CUDA events around k_assign of the middle pass of every "
                                   "timed step, inside the run graph, averaged"}
        per_iter = s_ms + a_ms + u_ms
        line["per_iteration"] = {"ms": per_iter, "search_ms": s_ms, "assign_ms": a_ms,
                                 "update_ms": u_ms,
                                 "point_iterations_per_s": n / (per_iter * 1e-3),
                                 "hbm_frac_of_iteration": n * ASSIGN_BYTES_PER_POINT
                                 / (per_iter * 1e-3) / 1e9 / hbm,
                                 "setup_ms": float(per[:, 3].mean())}
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
                       "stayed_points": stats.stayed_points,
                       "tiles": stats.tiles, "tile_level": stats.tile_level,
                       "grid_overflow": stats.grid_overflow}
    line["steady_state"] = ("every timed step repeats dkm_setup + dkm_run on the same context: "
                            "the candidate lists of the previous step seed pass 1's search "
                            "bound (see 'cold' for a fresh context)")
    if brute:
        line["brute_force"] = brute
    line["e2e"] = {"value": e2e_value, "unit": METRIC,
                   "h2d_bytes_per_step": n * d * 4 + k * d * 4,
                   "d2h_bytes_per_step": n * 4 + k * d * 4, "steps": e2e_steps}
    line["gpu_launches"] = launches_per_step(iters) * args.steps
    clocks = clk.summary(window=(w0, w1))
    if clocks.get("sm_mhz"):
        clocks["kcycles_per_step"] = t_job * 1e3 * clocks["sm_mhz"]
    line["clocks"] = clocks
    if peaks_dev is not None:
        line["device"] = {"sm_count": peaks_dev.sm_count, "sm_clock_mhz": peaks_dev.sm_clock_mhz,
                          "fp32_fma_tflops": peaks_dev.fp32_fma_tflops,
                          "fp32x2_fma_tflops": peaks_dev.fp32x2_fma_tflops,
                          "how": "dkm_device_peaks: FMA-chain kernels, CUDA events"}
    if ws == 1 and not args.no_cpu_baseline:
        v, dt, thr = cpu_sample_run(w, args.cpu_sample)
        m1 = max(1, args.cpu_sample // 16)
        v1, dt1, _ = cpu_sample_run(w, m1, seed=1, single_thread=True)
        line["cpu_baseline"] = {"value": v, "unit": METRIC, "cores": thr, "kind": "oracle",
                                "cpu_model": cpu_model(),
                                "sample": f"one FP64 brute-force Lloyd iteration (assignment "
                                          f"against all k=10000 centroids + update) of "
                                          f"{min(args.cpu_sample, n)} of the workload's {n} "
                                          f"points ({dt:.1f} s)",
                                "single_thread": {"value": v1, "unit": METRIC, "cores": 1,
                                                  "sample": f"the same iteration on {m1} "
                                                            f"points, the oracle built without "
                                                            f"OpenMP ({dt1:.1f} s)"}}
    if ablations:
        line["ablations"] = ablations
    if ws == 1 and not args.no_extra:
        line["cold"] = bench_cold(dkm, torch, dev, stream, w, tune, iters)
        ctx.close()
        side = max(3, min(args.steps, 10))
        line["geo2d_blobs"] = bench_2d(dkm, torch, dev, stream, "geo2d-blobs", side, hbm)
        line["geo2d_roads"] = bench_2d(dkm, torch, dev, stream, "geo2d-roads", side, hbm)
        line["batched"] = bench_batched(dkm, torch, dev, stream, max(2, min(args.steps, 5)), hbm)
        line["differentiable"] = bench_soft(dkm, torch, dev, stream, max(2, min(args.steps, 5)),
                                            peaks_dev)
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--profile", type=int, default=1,
                    help="record per-kernel CUDA events around the middle pass of every "
                         "timed step, inside the run graph (roofline)")
    ap.add_argument("--cpu-sample", type=int, default=4_000_000)
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
    ap.add_argument("--batched-only", action="store_true",
                    help="time only the 512-cloud workload (autotuned, --steps timed steps of "
                         "setup + 25 passes, and its brute-force comparison) and print its JSON "
                         "object")
    ap.add_argument("--soft-only", action="store_true",
                    help="time only the differentiable workload (soft k-means forward + "
                         "backward and the hard SSE, --steps timed calls each) and print its "
                         "JSON object")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.soft_only:
        return run_soft_only(args)
    if args.batched_only:
        return run_batched_only(args)
    return run_ours(args)


def run_batched_only(args):
    import torch
    from paper_2412_02244_gb300 import build as b
    b.build()
    from paper_2412_02244_gb300 import dkm
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    hbm, _ = peaks()
    print(json.dumps(bench_batched(dkm, torch, dev, stream, max(1, args.steps), hbm)), flush=True)
    return 0


def run_soft_only(args):
    import torch
    from paper_2412_02244_gb300 import build as b
    b.build()
    from paper_2412_02244_gb300 import dkm
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    peaks_dev = dkm.dkm_device_peaks(stream.cuda_stream)
    print(json.dumps(bench_soft(dkm, torch, dev, stream, max(1, args.steps), peaks_dev)),
          flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
