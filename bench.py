"""Benchmark of the collage hot path: fwd + bwd + Adam iterations per second.

Workload (one step = one iteration of transform -> bin -> raster + losses -> distribution term ->
adjoint -> Adam): 1000 mixed elements (60% cubic blobs, 30% convex polygons, 10% open polylines)
in an annulus container at the 1024^2 level of the 128 -> 256 -> 512 -> 1024 pyramid, padding
2 px, full loss of Eq. 8.  The timed path is the graph-captured, persistent, autotuned one; the
same workload is also timed on the plain path (eager launches, one block per tile, 16 px tiles).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU (torchrun): collages are independent problems, so each rank optimises its own collage
(seeded by its rank) with no collective on the data path; the whole-job value is the iterations of
all ranks over the slowest rank's time ("weak" scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd+step iters/s at 1024², 1000 elems (batched vs plain); % roofline"
WORKLOAD = "mixed1000_annulus_1024: 1000 elements (600 cubic blobs, 300 convex polygons, " \
           "100 open polylines), annulus 0.2/0.48, level 1024^2 of 128/256/512/1024, pad 2 px"
L2_FLUSH_BYTES = 512 << 20
# Algorithmic work of the raster forward per pixel-segment pair (the method's definition: every
# pixel of an element's grown bounding box against every segment of the element): distance 9,
# crossing 3, min/select 2 FP32 operations.  The kernel skips most of these pairs exactly (segments
# beyond the coverage margin of a tile only add to a winding backdrop), so the achieved figure is
# method work per second, not instructions per second.
FLOP_PER_PAIR = 14
# ncu capture of the raster forward kernel (dram__bytes_read.sum + dram__bytes_write.sum per
# launch) and the hash of raster.cu it was taken with; the figure is reported only while the
# source is unchanged.
NCU_TRAFFIC = {"raster_src_sha1": "c918ebbd15d27ab3b3ecf8139c82efc47c2c40c4", "bytes_per_launch": 2422528}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def _measured_fp32_peak(torch):
    """FP32 FMA rate of this GPU in TFLOP/s, from the library's FMA-chain kernel."""
    import ctypes as C
    from paper_2406_04008_gb300 import _lib
    out = C.c_float()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    _lib.check(_lib.load().collage_fp32_peak(stream, C.byref(out)))
    return float(out.value)


def _raster_src_sha1():
    with open(os.path.join(ROOT, "paper_2406_04008_gb300", "csrc", "raster.cu"), "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()


class _Nvml:
    """Read-only NVML queries through ctypes (the driver's libnvidia-ml): SM clock, its maximum and
    the active clock-event reasons of one GPU, found by the UUID torch reports."""
    SM = 1  # NVML_CLOCK_SM
    BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
            0x40: "hw_thermal_slowdown"}

    def __init__(self, uuid, index):
        import ctypes as C
        self.C = C
        self.lib = C.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = C.c_void_p()
        ok = False
        if uuid:
            ok = self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), C.byref(self.h)) == 0
        if not ok and self.lib.nvmlDeviceGetHandleByIndex_v2(index, C.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        f = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.reasons_fn = f or self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def sample(self):
        C = self.C
        clk, mx, rs = C.c_uint(), C.c_uint(), C.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, C.byref(clk)) != 0:
            return None
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.SM, C.byref(mx))
        self.reasons_fn(self.h, C.byref(rs))
        return float(clk.value), float(mx.value), [n for b, n in self.BITS.items() if rs.value & b]


class ClockSampler:
    """SM clock and throttle reasons while the timed region runs: nvidia-smi every 50 ms (as the
    profiling recipe does) and NVML every millisecond (a timed region of a few milliseconds falls
    between nvidia-smi samples)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, uuid=None):
        self.index = index
        self.uuid = uuid
        self.proc = None
        self.lines = []
        self.fast = []
        self.stop = threading.Event()
        self.nvml = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.perf_counter()  # the timed region starts once samples flow
            while not self.lines and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines.clear()
        except OSError:
            self.proc = None
        try:
            self.nvml = _Nvml(self.uuid, self.index)
            self.ft = threading.Thread(target=self._poll, daemon=True)
            self.ft.start()
        except (OSError, AttributeError):
            self.nvml = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def _poll(self):
        while not self.stop.is_set():
            s = self.nvml.sample()
            if s:
                self.fast.append(s)
            time.sleep(0.001)

    def __exit__(self, *a):
        self.stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        n_smi = 0
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            n_smi += 1
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        for c, m, rs in self.fast:
            sm.append(c)
            mx.append(m)
            reasons.update(rs)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "samples_nvidia_smi": n_smi, "samples_nvml": len(self.fast)}


def _config(world):
    """The workload's description, the same on both arms."""
    return {"workload": WORKLOAD, "grid": 1024, "elements": 1000,
            "path": "graph-captured persistent autotuned",
            "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
            "parallelism": f"replicas x{world}"}


def _workload(rank=0):
    from paper_2406_04008_gb300 import workloads as W
    return W.config_problem(3, collage_index=rank)


def _opts(**kw):
    o = dict(pad_px=2.0, n_levels=4, level_res=[128, 256, 512, 1024],
             level_iters=[300, 200, 100, 50])
    o.update(kw)
    return o


def _time_steps(col, steps, flush, torch):
    """Per-step device time with CUDA events on the launching stream, L2 flushed between steps.
    Steps are enqueued without a host round trip (collage_step_async); the status word is checked
    once after the loop, and a run that met a bin overflow (iterations skipped) is an error."""
    stream = torch.cuda.current_stream()
    _, step0, _ = col.get_state()
    ev = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        col.step_async(1)
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    col.sync()
    _, step1, _ = col.get_state()
    assert step1 - step0 == steps, "iterations were skipped inside the timed region"
    return [a.elapsed_time(b) / 1e3 for a, b in ev]


def run_reference(args):
    """The oracle (FP64 CPU) on the same workload: the reference arm."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    from oracle import oracle as O
    O.build()
    prob = _workload()
    sc = O.Scene(prob)
    o = O.options(pad_px=2.0)
    q = prob["params0"].astype(np.float64)
    m, v = np.zeros_like(q), np.zeros_like(q)
    # one oracle iteration takes ~0.4 s on 16 cores: the sample is capped so that the run ends in
    # well under a minute
    warm, steps = min(args.warmup, 10), min(args.steps, 20)
    for i in range(warm):
        g = sc.eval(q, 1024, o)["grad_a"]
        q, m, v = O.adam(q, m, v, g, i + 1)
    t0 = time.perf_counter()
    for i in range(steps):
        g = sc.eval(q, 1024, o)["grad_a"]
        q, m, v = O.adam(q, m, v, g, warm + i + 1)
    dt = time.perf_counter() - t0
    val = steps / dt
    cores = os.cpu_count()
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "iters/s",
           "n_gpus": args.gpus, "steps": steps, "warmup": warm,
           "ms_per_step": 1e3 * dt / steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _config(args.gpus),
           "cpu_baseline": {"value": val, "unit": "iters/s", "cores": cores, "kind": "oracle",
                            "sample": f"{steps} full FP64 oracle iterations (forward, "
                                      "gradient, Adam) of the 1024^2 workload (at most 20 of "
                                      "the requested steps)"},
           "e2e": {"value": val, "unit": "iters/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_profile(args):
    """A fixed launch sequence for ncu: level 1024^2, W eager warm-up iterations, N eager ones.
    --profile-workload fit20: the outline fitting of one 20-cubic star at 256^2 instead;
    mat_init: N skeleton-based initialisations of the 1024^2 workload."""
    import torch

    from paper_2406_04008_gb300 import build
    build.build()
    from paper_2406_04008_gb300.collage import Collage
    if args.profile_workload == "fit20":
        from paper_2406_04008_gb300 import workloads as W
        kw = dict(W.FIT_LOSS)
        kw["delta_down"] = kw.pop("delta")
        col = Collage(W.fit_problem(0), fit_controls=1, n_levels=1, level_res=[256], level_iters=[50],
                      n_dilations=0, use_graphs=0, persistent=1, tile=args.tile, **kw)
        col.step(args.warmup)
        col.step(args.profile_iters)
        torch.cuda.synchronize()
        print(json.dumps({"profile_iters": args.profile_iters, "info": col.info()}))
        col.close()
        return
    if args.profile_workload == "mat_init":
        col = Collage(_workload(), level_res=[1024], tile=args.tile)
        for _ in range(args.warmup + args.profile_iters):
            col.mat_init()
        torch.cuda.synchronize()
        print(json.dumps({"profile_iters": args.profile_iters, "info": col.info()}))
        col.close()
        return
    col = Collage(_workload(), **_opts(use_graphs=0, persistent=1, tile=args.tile))
    col.set_level(3)
    col.step(args.warmup)
    col.step(args.profile_iters)
    torch.cuda.synchronize()
    print(json.dumps({"profile_iters": args.profile_iters, "info": col.info()}))
    col.close()


def cpu_baseline(max_seconds=20.0):
    """The FP64 oracle as it stands, timed on this host's cores on full 1024^2 iterations."""
    import numpy as np

    from oracle import oracle as O
    O.build()
    prob = _workload()
    sc = O.Scene(prob)
    o = O.options(pad_px=2.0)
    q = prob["params0"].astype(np.float64)
    m, v = np.zeros_like(q), np.zeros_like(q)
    n, t0 = 0, time.perf_counter()
    while True:
        g = sc.eval(q, 1024, o)["grad_a"]
        q, m, v = O.adam(q, m, v, g, n + 1)
        n += 1
        if time.perf_counter() - t0 > max_seconds or n >= 8:
            break
    dt = time.perf_counter() - t0
    pairs = sc.pair_work(prob["params0"].astype(np.float64), 1024, o)
    return {"value": n / dt, "unit": "iters/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} full FP64 oracle iterations (forward, gradient, Adam) of the 1024^2 "
                      f"workload, OpenMP over pixel rows"}, pairs


def cpu_per_config():
    """Seconds per FP64 oracle iteration (forward, gradient, Adam) at each workload's finest level,
    on all host cores, plus the 1024^2 workload on one core.  One iteration each (three for the
    16-disk case); for the 64-collage batch, 8 of its collages (the seconds are for those 8)."""
    import numpy as np

    from oracle import oracle as O
    from paper_2406_04008_gb300 import workloads as W

    def per_iter(prob, grid, opts, iters=1):
        sc = O.Scene(prob)
        o = O.options(**opts)
        q = prob["params0"].astype(np.float64)
        m, v = np.zeros_like(q), np.zeros_like(q)
        t0 = time.perf_counter()
        for i in range(iters):
            g = sc.eval(q, grid, o)["grad_a"]
            q, m, v = O.adam(q, m, v, g, i + 1)
        return (time.perf_counter() - t0) / iters

    out = {"unit": "s/iteration", "cores": os.cpu_count()}
    # the method work of configs 1 and 2 (pixel-segment pairs, the roofline's denominator)
    out["pairs"] = {name: O.Scene(W.config_problem(cfg)).pair_work(
        W.config_problem(cfg)["params0"].astype(np.float64), grid, O.options(**kw))
        for name, cfg, grid, kw in CONFIG_LINES}
    out["disks16_128"] = per_iter(W.config_problem(1), 128, dict(gamma=0.0), 3)
    out["blobs200_star_512"] = per_iter(W.config_problem(2), 512, {})
    t0 = time.perf_counter()
    for i in range(8):
        p = W.config_problem(4, i)
        per_iter(p, p["grid"], {})
    out["batch64_first8"] = time.perf_counter() - t0
    out["open5000_rect_2048"] = per_iter(W.config_problem(5), 2048, dict(pad_px=1.0, delta=1e3))
    # outline fitting: gradient of the 60 control points and their Adam step, 256^2
    fp = W.fit_problem(0)
    t0 = time.perf_counter()
    g, _ = O.control_grad(fp, fp["params0"], 256, O.options(**W.FIT_LOSS))
    O.adam_points(np.asarray(fp["pts"]).reshape(-1, 2), 0.0, 0.0, g, 1)
    out["fit20_star_256"] = time.perf_counter() - t0
    # skeleton-based initialisation of the 1024^2 workload (one call, s)
    t0 = time.perf_counter()
    O.mat_init(_workload(), _workload()["params0"], 1024, O.options())
    out["mat_init_mixed1000_1024"] = time.perf_counter() - t0
    prev = O.set_threads(1)
    try:
        out["mixed1000_annulus_1024_1core"] = per_iter(_workload(), 1024, dict(pad_px=2.0))
    finally:
        O.set_threads(prev)
    return out


def batch_vs_plain(steps, flush, torch):
    """64 independent collages (n ~ U[20, 800], grids 256/512/1024, stars and annuli): one batched,
    graph-captured, persistent, autotuned handle against 64 plain handles stepped one after
    another.  A step advances every collage by one iteration."""
    from paper_2406_04008_gb300 import workloads as W
    from paper_2406_04008_gb300.collage import Collage
    probs = [W.config_problem(4, i) for i in range(64)]
    kw = dict(n_levels=1, level_res=[1], level_iters=[50])
    col = Collage(probs, use_graphs=1, persistent=1, tile=0, **kw)
    tile, _ = col.autotune()
    tuning = col.tuning()
    col.step(3)
    torch.cuda.synchronize()
    bt = sum(_time_steps(col, steps, flush, torch))
    n_elems = col.n_elems
    col.close()
    plain = [Collage(p, use_graphs=0, persistent=0, tile=16, **kw) for p in probs]
    for c in plain:
        c.step(1)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    pt = 0.0
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for c in plain:
            c.step_async(1)
        b.record(stream)
        b.synchronize()
        pt += a.elapsed_time(b) / 1e3
    for c in plain:
        c.sync()
        c.close()
    return {"workload": "batch64: 64 collages, %d elements in all, grids 256/512/1024" % n_elems,
            "batched": steps / bt, "plain_sequential": steps / pt, "speedup": pt / bt,
            "unit": "batch iterations/s (every collage one fwd+bwd+Adam iteration)", "tile": tile,
            "tuning": dict(tuning, gain_over_defaults=(tuning["default_ms"] / tuning["best_ms"]
                                                       if tuning["default_ms"] else None))}


def batch_sharded(steps, flush, torch, world, rank, barrier, max_over_ranks):
    """The 64-collage batch split across the ranks by whole collages (sharding.shard: greedy LPT on
    estimated work, the same on every rank without communication, no collective on the data
    path): each rank steps its shard in one batched, graph-captured, autotuned handle.  A step
    advances every collage of the batch by one iteration; the time is the slowest rank's."""
    from paper_2406_04008_gb300 import sharding
    from paper_2406_04008_gb300 import workloads as W
    from paper_2406_04008_gb300.collage import Collage
    probs = [W.config_problem(4, i) for i in range(64)]
    mine = sharding.shard(probs, world, rank)
    col = Collage([probs[i] for i in mine], use_graphs=1, persistent=1, tile=0, n_levels=1,
                  level_res=[1], level_iters=[50])
    col.autotune()
    col.step(3)
    torch.cuda.synchronize()
    barrier()
    t = max_over_ranks(sum(_time_steps(col, steps, flush, torch)))
    col.close()
    return {"workload": "batch64 sharded by whole collages over %d rank(s) (LPT)" % world,
            "value": steps / t, "unit": "batch iterations/s (every collage of the 64 one iteration)",
            "collages_on_rank0": len(sharding.shard(probs, world, 0)), "scaling": "strong"}


CONFIG_LINES = (("disks16_disk_128", 1, 128, dict(gamma=0.0)), ("blobs200_star_512", 2, 512, {}))


def config_lines(steps, flush, torch):
    """Configs 1 (16 disks, 128^2) and 2 (200 blobs, 512^2) of the workload list: the graph-captured,
    persistent, autotuned path against the plain one (eager launches, one block per tile, 16-px
    tiles), and the forward and backward raster stages' times (the forward's method work comes
    from the CPU-baseline leg)."""
    from paper_2406_04008_gb300 import workloads as W
    from paper_2406_04008_gb300.collage import Collage
    out = {}
    for name, cfg, grid, kw in CONFIG_LINES:
        prob = W.config_problem(cfg)
        base = dict(n_levels=1, level_res=[grid], level_iters=[50], **kw)
        col = Collage(prob, use_graphs=1, persistent=1, tile=0, **base)
        col.autotune()
        col.step(3)
        torch.cuda.synchronize()
        tuned = 1.0 / statistics.median(_time_steps(col, steps, flush, torch))
        stages = col.stage_times(20)
        col.close()
        plain = Collage(prob, use_graphs=0, persistent=0, tile=16, **base)
        plain.step(3)
        torch.cuda.synchronize()
        pl = 1.0 / statistics.median(_time_steps(plain, steps, flush, torch))
        plain.close()
        out[name] = {"tuned": tuned, "plain": pl, "speedup": tuned / pl, "unit": "iters/s",
                     "raster_fwd_ms": stages["raster_fwd"], "raster_bwd_ms": stages["raster_bwd"]}
    return out


def outline_fitting(steps, flush, torch):
    """Outline fitting (Sec. 3, Vector Representation): closed paths of 20 cubics (the paper's N)
    fitted to seeded star silhouettes at 256^2 by Adam on their control points; one outline, and 64
    outlines in one batched handle.  A step is one fwd+bwd+Adam iteration of every outline."""
    from paper_2406_04008_gb300 import workloads as W
    from paper_2406_04008_gb300.collage import Collage
    kw = dict(W.FIT_LOSS)
    kw["delta_down"] = kw.pop("delta")
    kw.update(fit_controls=1, n_levels=1, level_res=[256], level_iters=[50], n_dilations=0)
    out = {"workload": "fit20_star_256: closed paths of 20 cubics (320 segments) fitted to 12-point "
                       "star silhouettes at 256^2, L_c with w_in = w_out = 1",
           "unit": "iters/s (one fwd+bwd+Adam iteration of every outline)"}
    for name, probs in (("one", [W.fit_problem(0)]), ("batch64", [W.fit_problem(i) for i in range(64)])):
        col = Collage(probs, use_graphs=1, persistent=1, tile=0, **kw)
        col.autotune()
        # the outlines grow towards the star tips: the synchronous warm-up regrows the bins, so
        # the timed asynchronous steps meet no overflow
        col.step(150)
        torch.cuda.synchronize()
        out[name] = steps / sum(_time_steps(col, steps, flush, torch))
        col.close()
    return out


def mat_initialisation(torch):
    """Skeleton-based initialisation (Sec. 4.1) of the 1000-element workload at its 1024^2 level:
    medial width, ridge axis and greedy placement (collage_mat_init), milliseconds per call."""
    from paper_2406_04008_gb300.collage import Collage
    col = Collage(_workload(), level_res=[1024], tile=8)
    col.mat_init()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    a.record(stream)
    for _ in range(reps):
        col.mat_init()
    b.record(stream)
    b.synchronize()
    col.close()
    return {"workload": "mixed1000_annulus_1024: medial axis of the annulus at 1024^2, 1000 elements "
                        "placed", "ms": a.elapsed_time(b) / reps}


def open_packing(steps, flush, torch):
    """5000 mixed elements in an open-top rectangle at 2048^2 with the downward force and 1 px
    padding, atomic and deterministic gradient modes."""
    from paper_2406_04008_gb300 import workloads as W
    from paper_2406_04008_gb300.collage import Collage
    prob = W.config_problem(5)
    out = {"workload": "open5000_rect_2048: 5000 elements, 2048^2, pad 1 px, downward force 1e3",
           "unit": "iters/s"}
    for name, det in (("atomic", 0), ("deterministic", 1)):
        col = Collage(prob, n_levels=1, level_res=[2048], pad_px=1.0, delta_down=1e3,
                      deterministic=det, use_graphs=1, persistent=1, tile=8)
        col.step(3)
        torch.cuda.synchronize()
        out[name] = steps / sum(_time_steps(col, steps, flush, torch))
        col.close()
    return out


def schedule_time(torch):
    """The whole 128 -> 256 -> 512 -> 1024 schedule (300/200/100/50 iterations) as one captured
    graph (collage_run_schedule): wall time of a run with the graph cached, of the first run (which
    probes every level and captures), and each level's device time on its own (CUDA events around
    the level's iterations on its one-iteration graph)."""
    from paper_2406_04008_gb300.collage import Collage
    levels, iters = [128, 256, 512, 1024], [300, 200, 100, 50]
    col = Collage(_workload(), **_opts(use_graphs=1, persistent=1, tile=8))
    stream = torch.cuda.current_stream()
    per_level = []
    for lv, n in enumerate(iters):
        col.set_level(lv)
        col.step(2)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        col.step_async(n)
        b.record(stream)
        b.synchronize()
        col.sync()
        ms = a.elapsed_time(b)
        per_level.append({"res": levels[lv], "iterations": n, "device_ms": ms, "us_per_iter": 1e3 * ms / n})
    walls = []
    for _ in range(3):
        col.set_level(0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        col.run_schedule()
        torch.cuda.synchronize()
        walls.append(time.perf_counter() - t0)
    col.close()
    dev = sum(x["device_ms"] for x in per_level) / 1e3
    return {"iterations": sum(iters), "levels": "128/256/512/1024 x 300/200/100/50",
            "path": "one CUDA graph: per level the level switch and a device-decided WHILE loop",
            "seconds": statistics.median(walls[1:]), "first_run_seconds": walls[0],
            "sum_level_device_seconds": dev, "wall_over_device": statistics.median(walls[1:]) / dev,
            "per_level": per_level}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batch64 / open5000 / schedule measurements")
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="for ncu: W warm-up then N eager iterations of the 1024^2 step, no timing")
    ap.add_argument("--tile", type=int, default=16, help="raster tile of --profile-iters")
    ap.add_argument("--profile-workload", default="mixed1000", choices=["mixed1000", "fit20", "mat_init"],
                    help="what --profile-iters runs")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_iters:
        return run_profile(args)
    args.warmup = max(args.warmup, 3)

    import numpy as np
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_2406_04008_gb300 import build
    build.build()
    from paper_2406_04008_gb300.collage import Collage

    prob = _workload(rank)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda", dtype=torch.float32)

    # ---- the timed path: graph-captured, persistent, autotuned ----
    col = Collage(prob, **_opts(use_graphs=1, persistent=1, tile=0))
    col.set_level(3)
    tile, _ = col.autotune()
    tuning = col.tuning()
    col.step(args.warmup)
    torch.cuda.synchronize()
    info = col.info()
    barrier()
    torch.cuda.synchronize()
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except (AttributeError, RuntimeError):
        uuid = None
    with ClockSampler(local, uuid) as clk:
        t_wall0 = time.perf_counter()
        times = _time_steps(col, args.steps, flush, torch)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    barrier()
    # the statistic: the median step time (p10 / p90 and the mean beside it), max over ranks
    med = statistics.median(times)
    total = sum(times)
    if world > 1:
        t = torch.tensor([med, total], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        med, total = float(t[0].item()), float(t[1].item())
    value = world / med
    qs = statistics.quantiles(times, n=10) if len(times) >= 2 else [times[0]] * 9
    spread = {"statistic": "median of per-step CUDA-event times, max over ranks",
              "p10_ms": 1e3 * qs[0], "median_ms": 1e3 * med, "p90_ms": 1e3 * qs[-1],
              "mean_ms": 1e3 * total / len(times), "mean_value": world * len(times) / total}

    # ---- end to end through the host-buffer entry point ----
    p0 = np.ascontiguousarray(prob["params0"], np.float32)
    pin_out = torch.from_numpy(p0.copy()).pin_memory()  # params in and out, updated in place
    pin_loss = torch.empty(5, dtype=torch.float32).pin_memory()
    import ctypes as C
    lib, h = col.lib, col.h
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    vp = lambda t: C.c_void_p(t.data_ptr())
    for _ in range(2):
        lib.collage_step_host(h, stream, 1, vp(pin_out), vp(pin_out), vp(pin_loss))
    barrier()
    e2e_t = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = lib.collage_step_host(h, stream, 1, vp(pin_out), vp(pin_out), vp(pin_loss))
        e2e_t += time.perf_counter() - t0
        assert st == 0
    if world > 1:
        t = torch.tensor([e2e_t], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_t = float(t.item())
    e2e = {"value": world * args.steps / e2e_t, "unit": "iters/s",
           "h2d_bytes_per_step": int(p0.nbytes), "d2h_bytes_per_step": int(p0.nbytes + 20)}

    # ---- per-kernel times at the initial params (for the roofline) ----
    col.set_params(torch.from_numpy(p0).cuda())
    stages = col.stage_times(20)
    col.close()

    # ---- the plain path on the same workload ----
    plain = Collage(prob, **_opts(use_graphs=0, persistent=0, tile=16))
    plain.set_level(3)
    plain.step(args.warmup)
    torch.cuda.synchronize()
    ptimes = _time_steps(plain, min(args.steps, 50), flush, torch)
    plain.close()
    plain_value = 1.0 / statistics.median(ptimes)

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    extra = {}
    if world == 1 and not args.no_extra:  # first: its autotuner search is the one reported
        extra["batch64"] = batch_vs_plain(10, flush, torch)
    if not args.no_extra:
        extra["batch64_sharded"] = batch_sharded(10, flush, torch, world, rank, barrier, max_over_ranks)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    if world == 1 and not args.no_extra:
        extra["open5000"] = open_packing(10, flush, torch)
        extra["schedule_mixed1000"] = schedule_time(torch)
        extra["fit20"] = outline_fitting(50, flush, torch)
        extra["mat_init"] = mat_initialisation(torch)

    peaks = _peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fp32_nominal = sms * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s, FMA = 2
    fp32_peak = _measured_fp32_peak(torch)
    if world == 1 and not args.no_extra:
        extra["configs_1_2"] = config_lines(50, flush, torch)
    cpu = None
    pairs = None
    if not args.no_cpu_baseline and world == 1:
        cpu, pairs = cpu_baseline()
        cpu["per_workload"] = cpu_per_config()
        for name, line in extra.get("configs_1_2", {}).items():
            pw = cpu["per_workload"]["pairs"][name]
            line["pairs"] = pw
            line["raster_fwd_frac_fp32"] = pw * FLOP_PER_PAIR / (line["raster_fwd_ms"] / 1e3) / 1e12 / fp32_peak
    roof = None
    if pairs is not None:
        t_fwd = stages["raster_fwd"] / 1e3
        achieved = pairs * FLOP_PER_PAIR / t_fwd / 1e12
        traffic = NCU_TRAFFIC["bytes_per_launch"] \
            if NCU_TRAFFIC["raster_src_sha1"] == _raster_src_sha1() else None
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": traffic, "kernel": "k_raster_chunks",
                "peak_source": "measured: FP32 FMA-chain kernel (collage_fp32_peak), burst",
                "peak_nominal": fp32_nominal,
                "peak_nominal_source": f"{sms} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
                "work": f"{pairs:.4g} pixel-segment pairs x {FLOP_PER_PAIR} flop",
                "launch_ms": stages["raster_fwd"]}
    out = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * med,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": _config(world),
           "tile": tile, "step_time": spread,
           "tuning": dict(tuning, gain_over_defaults=(tuning["default_ms"] / tuning["best_ms"]
                                                      if tuning["default_ms"] else None)),
           "plain": {"value": plain_value, "unit": "iters/s",
                     "path": "eager launches, one block per tile, 16 px tiles",
                     "speedup": value / world / plain_value},
           "stage_ms": {k: round(v, 5) for k, v in stages.items()},
           "e2e": e2e, "roofline": roof, "cpu_baseline": cpu, "clocks": clk.summary(),
           "gpu_launches": info["kernels_per_iter"] * args.steps,
           "wall_s": t_wall}
    out.update(extra)
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
