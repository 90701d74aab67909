#!/usr/bin/env python
"""Benchmark of the decoupled Fourier pose search (Fast-MbyM Alg. 1) on one GB300 per rank.

Workload (default): 32 scan pairs at 512 x 512 (polar grid 400 x 256), synthetic radar-like scans
from paper_2203_00459_gb300.synth.  One step = one pass of the search over the batch: forward, and
with --mode fwdbwd (default) the adjoint of the L2 pose loss as well.  Inputs stay resident in HBM;
L2 is flushed (a 256 MB write) between timed steps, outside the timed events.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "scan-pairs/s (fwd, fwd+bwd) at 512^2 vs plain per-pair path, pose err <=1e-3px vs FP64"
WORKLOAD = "batch512"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="fwdbwd", choices=["fwd", "fwdbwd"])
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "batch256", "batch511", "batch255", "batch127", "mixed", "masked256",
                             "masked256_tab2"])
    ap.add_argument("--conv-path", type=int, default=0, choices=[0, 1],
                    help="masked workloads: the mask network's flat-GEMM convolutions on mma.sync (0) or tcgen05 (1)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="for profilers: W + K training calls of --pairs pairs of the workload, launched directly "
                         "with the default schedules, and nothing else")
    ap.add_argument("--pairs", type=int, default=0, help="with --profile: pairs per call (default: the workload's)")
    ap.add_argument("--schedule", default="",
                    help="with --profile: launch schedules as knob=value,... (default: the library's defaults)")
    return ap.parse_args()


def run_profile(args):
    """W + K training calls (or forwards, --mode fwd) of the workload, launched kernel by kernel
    with the default launch schedules (or --schedule's), for a profiler to capture; prints one
    short line.  The pairs' offsets are passed explicitly, which keeps one grid per kernel over all
    pairs (a packed call of one size would run as two concurrent halves), as in the traced region
    that the roofline is measured on."""
    import numpy as np
    import torch
    from paper_2203_00459_gb300 import build, synth
    build.build()
    from paper_2203_00459_gb300.search import PoseSearch, size_cfg
    spec = synth.WORKLOADS[args.workload]
    B = args.pairs or spec["pairs"]
    f, g, gt = synth.make_batch(args.workload, pairs=B)
    s = PoseSearch([size_cfg(spec["n"], spec["n_theta"], spec["n_r"])], max_pairs=B)
    if args.schedule:
        s.set_tuning(0, **{k: int(v) for k, v in (kv.split("=") for kv in args.schedule.split(","))})
    F, G = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    GT = torch.from_numpy(gt.astype(np.float32)).cuda()
    offs = np.arange(B, dtype=np.int64) * spec["n"] * spec["n"]
    for _ in range(args.warmup + args.steps):
        if args.mode == "fwdbwd":
            out = s.pose_train(F, G, GT, kind=2, offsets=offs)
        else:
            out = (s.pose(F, G, offsets=offs)["pose"],)
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.workload, "pairs": B, "calls": args.warmup + args.steps, "mode": args.mode,
                      "schedule": s.tuning(0)}))
    s.close()


# ---------------------------------------------------------------------------------------------
# algorithmic bytes and FLOPs per pair of each kernel (what the kernel must read and write)
# ---------------------------------------------------------------------------------------------

def kernel_model(n, p, nt, nr, chunks):
    """Compulsory HBM bytes and nominal FFT FLOPs per pair of every kernel of the training step
    (each input read once, each output written once; the training call's forward also writes the
    arrays it keeps for the adjoint: phasors, angle spectra, column spectra)."""
    w, wp = n // 2, p // 2
    c = 8  # bytes of a complex float
    fft = lambda L: 5.0 * L * math.log2(L)  # nominal FLOPs of one complex length-L FFT
    half = (w + 1) * n                      # elements of a half plane
    m = {
        "s1_rows": (2 * n * n * 4 + 2 * n * w * c, 2 * (n // 2) * fft(n)),
        "s1_cols": (2 * n * w * c + 2 * half * 4 + 2 * half * c, 2 * w * fft(n)),
        "angle": (2 * half * 4 + chunks * nt * c + nt * nr * c, nr * fft(nt)),
        "theta": (chunks * nt * c + nt * 4, fft(nt)),
        "s2_rows": (2 * n * n * 4 + 2 * n * wp * c, 2 * (n // 2) * fft(p)),
        "s2_cols": (2 * n * wp * c + n * wp * c + 2 * p * wp * c, 3 * wp * fft(p)),
        "s2_c2r": (n * wp * c + n * n * 4, (n // 2) * fft(p)),
        "sxy": (n * n * 4, 0.0),
        "b_rows": (n * n * 4 + n * wp * c, (n // 2) * fft(p)),
        "b_cols": (n * wp * c + 2 * p * wp * c + 2 * n * wp * c, 3 * wp * fft(p)),
        "b_c2r": (2 * n * wp * c + 2 * n * n * 4, n * fft(p)),
        "b_rot": (3 * n * n * 4, 0.0),
        "b_theta": (nt * 4 + nt * c, fft(nt)),
        "b_angle": (nt * nr * c + nt * nr * c, nr * fft(nt)),
        "b_polT": (nt * nr * c + 2 * half * 4, 0.0),
        "b_s1cols": (2 * half * c + 2 * half * 4 + 2 * n * w * c, 2 * w * fft(n)),
        "b_s1rows": (2 * n * w * c + 4 * n * n * 4, n * fft(n)),
    }
    return m


# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of a kernel:
# (bytes, hash of the search sources it was taken on, pairs in that launch, column tile and radix
# order of the variant).  Reported, scaled to the launch's pairs, only while the sources are unchanged and the
# autotuner picked the same variant.  k_b_cols<512, 768, 4, 1> over 32 pairs at 512^2 (the third of
# three training calls; ncu flushes the caches before the launch):
#   S=col_tile=4,angle_radii=8,rot_pixels=8,col_plan=1
#   python bench.py --profile --pairs 32 --steps 2 --warmup 1 --schedule $S &&
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none \
#       -k regex:k_b_cols -s 2 -c 1 --csv python bench.py --profile --pairs 32 --steps 2 --warmup 1 --schedule $S
#   -> 201,415,168 read + 71,079,680 written, 85.7 us
TRAFFIC = {"b_cols": (201415168 + 71079680, "4cb11e25804106d3", 32, 4, 1)}


# the sources that define, plan and launch the adjoint kernels (k_b_cols among them)
SEARCH_SOURCES = ("api.cu", "bwd.cu", "common.cuh", "dev_util.cuh", "fft.cuh")


def src_hash():
    """Hash of the sources the adjoint kernels are built and launched from."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2203_00459_gb300", "csrc")
    for name in SEARCH_SOURCES:
        h.update(open(os.path.join(d, name), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "25"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# CPU oracle arm
# ---------------------------------------------------------------------------------------------

def _oracle_pair(args):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy as np
    import oracle as O
    f, g, cfg, dpose = args
    r = O.pose(f, g, cfg)
    if dpose is not None:
        O.pose_backward(f, g, cfg, np.asarray(dpose, np.float64))
    return r["theta"]


def oracle_rate(f, g, gt, spec, mode, pairs, pool):
    """Pairs per second of the FP64 oracle over the first `pairs` pairs, spread over the pool."""
    import numpy as np
    import oracle as O
    cfg = O.make_cfg(spec["n"], spec["n_theta"], spec["n_r"])
    jobs = []
    for i in range(pairs):
        dpose = None
        if mode == "fwdbwd":
            dpose = [1.0, 0.5, -0.5]
        jobs.append((f[i].astype(np.float64), g[i].astype(np.float64), cfg, dpose))
    t0 = time.perf_counter()
    list(pool.map(_oracle_pair, jobs))
    return pairs / (time.perf_counter() - t0)


def make_pool():
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    return mp.get_context("spawn").Pool(cores), cores


def run_reference(args, spec, rank):
    """The FP64 oracle on the host cores, on this arm's workload, metric and unit.  The pairs of a
    step run one after another in this process, each with numpy's BLAS on every core.  Each step
    is a bounded sample: the number of pairs is sized from a first timed pair so that the K + W
    steps end within about two and a half minutes; when even one pair per step would take longer
    with the oracle's direct DFT sums, the steps time its FFT route (the same sums, evaluated
    faster, pinned against the direct route), and the line says so."""
    from paper_2203_00459_gb300 import synth
    if rank != 0:
        return
    import numpy as np
    import oracle as O
    cores = os.cpu_count() or 1
    f, g, gt = synth.make_batch(args.workload, pairs=min(spec["pairs"], 16))
    steps = max(1, args.steps)
    budget = 150.0
    dpose = np.array([1.0, 0.5, -0.5])

    def one(i, cfg):
        fi, gi = f[i].astype(np.float64), g[i].astype(np.float64)
        O.pose(fi, gi, cfg)
        if args.mode == "fwdbwd":
            O.pose_backward(fi, gi, cfg, dpose)

    route = "direct"
    cfg = O.make_cfg(spec["n"], spec["n_theta"], spec["n_r"])
    t0 = time.perf_counter()
    one(0, cfg)
    t_pair = time.perf_counter() - t0
    if (steps + args.warmup) * t_pair > budget:
        route = "fft"
        cfg = O.make_cfg(spec["n"], spec["n_theta"], spec["n_r"], route="fft")
        t0 = time.perf_counter()
        one(0, cfg)
        t_pair = time.perf_counter() - t0
    pairs = max(1, min(f.shape[0], int(budget / ((steps + args.warmup) * t_pair))))

    def step():
        for i in range(pairs):
            one(i, cfg)

    for _ in range(max(0, args.warmup)):
        step()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    dt = time.perf_counter() - t0
    v = pairs * steps / dt
    unit = "scan-pairs/s"
    sample = (f"{pairs} pairs of {args.workload} per step ({args.mode}), one after another in one process with "
              f"numpy's BLAS on {cores} cores, the oracle's {route} DFT route")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": unit, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "mode": args.mode,
            "config": {"workload": args.workload, "n": spec["n"], "n_theta": spec["n_theta"], "n_r": spec["n_r"],
                       "pairs_per_step": pairs, "oracle_route": route},
            "cpu_baseline": {"value": v, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------

def run_mixed(args):
    """The uneven batch: 512 pairs (256 at 128^2, 179 at 256^2, 77 at 512^2, shuffled) in one call;
    a step is mask inference (one U-Net per resolution, evaluation statistics) then the search
    forward, the L1 pose loss and the search adjoint over all pairs (graph replay, concurrent
    size groups)."""
    import numpy as np
    import torch
    from paper_2203_00459_gb300 import build, synth
    build.build()
    from paper_2203_00459_gb300 import _lib, masknet, train
    from paper_2203_00459_gb300.search import PoseSearch, size_cfg
    names = ["single128", "batch256", "batch512"]
    counts = [256, 179, 77]
    cfgs = [size_cfg(128, 128, 64), size_cfg(256, 400, 128), size_cfg(512, 400, 256)]
    levels = [(8, 16, 32), (8, 16, 32, 64), (8, 16, 32, 64)]
    order = np.concatenate([np.full(c, s) for s, c in enumerate(counts)])
    np.random.default_rng(5).shuffle(order)
    per = [np.flatnonzero(order == s) for s in range(3)]
    sizes = [cfgs[s]["n"] ** 2 for s in range(3)]
    offs = np.zeros(len(order), np.int64)
    # pairs of one size are stored contiguously (the U-Net works per size); the search sees the
    # shuffled order through offsets
    base = 0
    for s in range(3):
        offs[per[s]] = base + np.arange(len(per[s])) * sizes[s]
        base += len(per[s]) * sizes[s]
    F = torch.empty(base, device="cuda")
    G = torch.empty(base, device="cuda")
    FM = torch.empty(base, device="cuda")
    GM = torch.empty(base, device="cuda")
    gt = torch.empty((len(order), 3), device="cuda")
    nets = []
    start = 0
    for s in range(3):
        n = cfgs[s]["n"]
        f, g, pz = synth.make_batch(names[s], pairs=len(per[s]), spec=dict(synth.WORKLOADS[names[s]], pairs=len(per[s])))
        F[start:start + f.size] = torch.from_numpy(f.ravel()).cuda()
        G[start:start + g.size] = torch.from_numpy(g.ravel()).cuda()
        gt[torch.from_numpy(per[s]).cuda()] = torch.from_numpy(pz.astype(np.float32)).cuda()
        net = masknet.MaskNet(levels[s], n, n, max_batch=len(per[s]))
        net.load(train.init_params(levels[s], seed=1 + s).cuda())
        nets.append((net, start, len(per[s]), n))
        start += f.size
    search = PoseSearch(cfgs, max_pairs=len(order), flags=_lib.FLAG_GRAPH)
    pose = torch.empty((len(order), 3), device="cuda")
    dpose = torch.empty_like(pose)
    loss = torch.empty(1, device="cuda")
    dF, dG = torch.empty_like(F), torch.empty_like(G)
    L = _lib.lib()
    si = np.ascontiguousarray(order.astype(np.int32))

    def step():
        for net, st, cnt, n in nets:
            view = lambda t: t[st:st + cnt * n * n].view(cnt, n, n)
            net.forward(view(F), view(G), training=False, f_out=view(FM), g_out=view(GM))
        search.pose_train(FM, GM, gt, kind=1, size_idx=si, offsets=offs, out=(pose, loss, dpose, dF, dG))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # the same step for one size group at a time (its mask inference and its search call alone),
    # to see what running the groups concurrently on forked streams gains over running them
    # back to back: the sum of the lone groups against the mixed call
    def group_step(s):
        net, st, cnt, n = nets[s]
        view = lambda t: t[st:st + cnt * n * n].view(cnt, n, n)
        net.forward(view(F), view(G), training=False, f_out=view(FM), g_out=view(GM))
        idx = per[s]
        k = len(idx)
        search.pose_train(FM, GM, gt, kind=1, size_idx=np.full(k, s, np.int32), offsets=offs[idx],
                          out=(pose[:k], loss, dpose[:k], dF, dG))

    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda")
    alone = {}
    gt_full = gt
    for s in range(3):
        gt = gt_full[torch.from_numpy(per[s]).cuda()].contiguous()
        for _ in range(2):
            group_step(s)
        ms_s = []
        for _ in range(max(3, args.steps // 2)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            group_step(s)
            b.record()
            torch.cuda.synchronize()
            ms_s.append(a.elapsed_time(b))
        alone[str(cfgs[s]["n"])] = sum(ms_s) / len(ms_s)
    gt = gt_full
    l0 = L.fmbym_launch_count(search.handle) + sum(net.launch_count() for net, *_ in nets)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record()
        step()
        evs[k][1].record()
    torch.cuda.synchronize()
    launches = L.fmbym_launch_count(search.handle) + sum(net.launch_count() for net, *_ in nets) - l0
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    concurrency = {"alone_ms_per_size": {k: round(v, 4) for k, v in alone.items()},
                   "sum_alone_ms": round(sum(alone.values()), 4), "mixed_ms": round(ms, 4),
                   "gain_of_concurrent_groups": round(sum(alone.values()) / ms, 3),
                   "note": "each size group's step timed alone (mask inference + pose_train of its pairs) "
                           "against the mixed call that runs the three groups on forked streams"}
    line = {"metric": "scan-pairs/s, uneven batch with mask inference, search fwd+bwd", "value": len(order) / (ms * 1e-3),
            "unit": "scan-pairs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 search, bf16 mask",
            "data": "synthetic", "gpu_launches": int(launches),
            "config": {"workload": "mixed", "pairs": {"128": counts[0], "256": counts[1], "512": counts[2]},
                       "mask_levels": {"128": 3, "256": 4, "512": 4}, "l2": "flushed between timed steps"},
            "concurrency": concurrency}
    print(json.dumps(line), flush=True)


def exhaustive_comparison(pairs=64, steps=3, warmup=1):
    """The exhaustive rotate-then-correlate search against the decoupled search's forward on the
    same 256^2 pairs of the batch256 workload: pairs/s of both (CUDA events, L2 flushed before each
    timed call) and their mean absolute pose errors against the generator's ground truth.  The
    exhaustive search runs once with 360 candidate headings 1 degree apart and once at equal
    accuracy: a grid of step 4 e (e the decoupled search's mean heading error; a uniform grid of
    step d errs by d / 4 on average), rounded to whole degrees."""
    import numpy as np
    import torch
    from paper_2203_00459_gb300 import _lib, synth
    from paper_2203_00459_gb300.search import PoseSearch, size_cfg
    f, g, gt = synth.make_batch("batch256", pairs=pairs, start=1000)
    cfg = size_cfg(256, 400, 128)
    s = PoseSearch([cfg], max_pairs=pairs, flags=_lib.FLAG_GRAPH)
    fd, gd = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda")
    pe = torch.empty((pairs, 3), device="cuda")
    pd = torch.empty((pairs, 3), device="cuda")

    def timed(fn, reps):
        for _ in range(warmup):
            fn()
        ms = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return sum(ms) / len(ms)

    def err(p):
        e = np.mean(np.abs(p.cpu().numpy().astype(np.float64) - gt), axis=0)
        return {"theta_deg": float(np.degrees(e[0])), "tx_px": float(e[1]), "ty_px": float(e[2])}

    ms_d = timed(lambda: s.pose(fd, gd, out=pd), max(10, steps))
    out = {"workload": f"batch256, {pairs} pairs", "decoupled_fwd_pairs_per_s": pairs / (ms_d * 1e-3),
           "mean_abs_err_decoupled": err(pd)}
    step_eq = max(1, int(round(4.0 * out["mean_abs_err_decoupled"]["theta_deg"])))
    for label, step in (("grid_1deg", 1), ("equal_accuracy", step_eq)):
        angles = np.radians(np.arange(-180, 180, step, dtype=np.float64)).astype(np.float32)
        ms_e = timed(lambda: s.pose_exhaustive(fd, gd, angles, out=pe), steps)
        out[label] = {"step_deg": step, "candidates": int(angles.size),
                      "exhaustive_pairs_per_s": pairs / (ms_e * 1e-3), "speedup_of_decoupled": ms_e / ms_d,
                      "mean_abs_err_exhaustive": err(pe)}
    s.close()
    return out


def angle_count_comparison(fma_peak, pairs=64, steps=10, warmup=3):
    """Alg. 1's own angle count n_theta = 733 (no FFT plan: the angle correlation and its adjoint
    as direct circular sums) beside n_theta = 400 (FFT route) on the same 256^2 pairs of the
    batch256 workload, n_r = 128: pairs/s of the forward and of the training step (CUDA events,
    L2 flushed before each timed call), and the device time of the angle stage from the library's
    tracer.  The direct sums are bound by FP32 multiply-adds: n_theta^2 n_r per pair forward,
    twice that in the adjoint, against fma_peak, the FP32 multiply-add rate measured on this GPU
    in the same run (fmbym_fp32_fma_rate)."""
    import ctypes
    import torch
    from paper_2203_00459_gb300 import _lib, synth
    from paper_2203_00459_gb300.search import PoseSearch, size_cfg
    L = _lib.lib()
    f, g, gt = synth.make_batch("batch256", pairs=pairs, start=2000)
    fd, gd = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    gtd = torch.from_numpy(gt.astype("float32")).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda")
    pose = torch.empty((pairs, 3), device="cuda")
    dpose = torch.empty((pairs, 3), device="cuda")
    loss = torch.empty(1, device="cuda")
    df, dg = torch.empty_like(fd), torch.empty_like(gd)
    out = {"workload": f"batch256, {pairs} pairs, n_r 128"}

    def fwd(srch):
        st = torch.cuda.current_stream().cuda_stream
        _lib.check(L.fmbym_pose(srch.handle, st, pairs, None, None, fd.data_ptr(), gd.data_ptr(), pose.data_ptr(),
                                None, None), srch.handle)

    def train(srch):
        st = torch.cuda.current_stream().cuda_stream
        _lib.check(L.fmbym_pose_train(srch.handle, st, pairs, None, None, fd.data_ptr(), gd.data_ptr(),
                                      gtd.data_ptr(), 2, pose.data_ptr(), loss.data_ptr(), dpose.data_ptr(),
                                      df.data_ptr(), dg.data_ptr()), srch.handle)

    def timed(fn):
        for _ in range(warmup):
            fn()
        ms = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return sum(ms) / len(ms)

    for nt in (400, 733):
        cfg = size_cfg(256, nt, 128)
        srch = PoseSearch([cfg], max_pairs=pairs, flags=_lib.FLAG_GRAPH)
        ms_f = timed(lambda: fwd(srch))
        ms_t = timed(lambda: train(srch))
        srch.close()
        traced = PoseSearch([cfg], max_pairs=pairs)
        for _ in range(warmup):
            train(traced)
        torch.cuda.synchronize()
        _lib.check(L.fmbym_set_tracing(traced.handle, 1), traced.handle)
        for _ in range(steps):
            flush.zero_()
            train(traced)
        torch.cuda.synchronize()
        K = 32
        tot, cnt, nk = (ctypes.c_double * K)(), (ctypes.c_longlong * K)(), ctypes.c_int()
        _lib.check(L.fmbym_trace_summary(traced.handle, K, tot, cnt, ctypes.byref(nk)), traced.handle)
        kern = {L.fmbym_trace_kind_name(k).decode(): tot[k] / cnt[k] for k in range(nk.value) if cnt[k]}
        traced.close()
        row = {"fwd_pairs_per_s": pairs / (ms_f * 1e-3), "step_pairs_per_s": pairs / (ms_t * 1e-3),
               "angle_ms": kern.get("angle"), "b_angle_ms": kern.get("b_angle"),
               "route": "fft" if nt == 400 else "direct sums"}
        if nt != 400 and kern.get("angle") and kern.get("b_angle"):
            fmas = nt * nt * 128 * pairs
            row["direct_roofline"] = {
                "bound": "alu", "unit": "TFMA/s", "peak": round(fma_peak / 1e12, 2), "peak_source": "measured",
                "achieved_fwd": round(fmas / (kern["angle"] * 1e-3) / 1e12, 2),
                "achieved_adjoint": round(2 * fmas / (kern["b_angle"] * 1e-3) / 1e12, 2),
                "frac_fwd": round(fmas / (kern["angle"] * 1e-3) / fma_peak, 4),
                "frac_adjoint": round(2 * fmas / (kern["b_angle"] * 1e-3) / fma_peak, 4),
                "note": "angle_ms includes the Cart2Pol gather launched with it"}
        out[f"n_theta_{nt}"] = row
    return out


def mixed_concurrency(counts=(64, 45, 19), steps=10, warmup=3):
    """The uneven mix's size groups in one training call (concurrent groups on forked streams,
    graph replay) against each group's training call alone, back to back: 128 pairs in the
    proportions of the 512-pair mixed workload (50 / 35 / 15 % at 128^2, 256^2, 512^2), search
    only.  If the groups left SMs idle at their tails, the mixed call would beat the sum of the
    lone calls by the idle time."""
    import numpy as np
    import torch
    from paper_2203_00459_gb300 import _lib, synth
    from paper_2203_00459_gb300.search import PoseSearch, size_cfg
    names = ["single128", "batch256", "batch512"]
    cfgs = [size_cfg(128, 128, 64), size_cfg(256, 400, 128), size_cfg(512, 400, 256)]
    order = np.concatenate([np.full(c, k) for k, c in enumerate(counts)])
    np.random.default_rng(5).shuffle(order)
    per = [np.flatnonzero(order == k) for k in range(3)]
    sizes = [c["n"] ** 2 for c in cfgs]
    offs = np.zeros(len(order), np.int64)
    base = 0
    F = []
    G = []
    gts = np.zeros((len(order), 3), np.float32)
    for k in range(3):
        offs[per[k]] = base + np.arange(len(per[k])) * sizes[k]
        base += len(per[k]) * sizes[k]
        f, g, gt = synth.make_batch(names[k], pairs=len(per[k]), spec=dict(synth.WORKLOADS[names[k]], pairs=len(per[k])))
        F.append(f.ravel())
        G.append(g.ravel())
        gts[per[k]] = gt
    Ft, Gt = torch.from_numpy(np.concatenate(F)).cuda(), torch.from_numpy(np.concatenate(G)).cuda()
    GT = torch.from_numpy(gts).cuda()
    s = PoseSearch(cfgs, max_pairs=len(order), flags=_lib.FLAG_GRAPH)
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda")
    n = len(order)
    pose, dpose = torch.empty((n, 3), device="cuda"), torch.empty((n, 3), device="cuda")
    loss, dF, dG = torch.empty(1, device="cuda"), torch.empty_like(Ft), torch.empty_like(Gt)

    def call(idx, si):
        k = len(idx)
        s.pose_train(Ft, Gt, GT[torch.from_numpy(idx).cuda()].contiguous() if k < n else GT, kind=1, size_idx=si,
                     offsets=offs[idx], out=(pose[:k], loss, dpose[:k], dF, dG))

    def timed(fn):
        for _ in range(warmup):
            fn()
        ms = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return sum(ms) / len(ms)

    allidx = np.arange(n)
    mixed = timed(lambda: call(allidx, order.astype(np.int32)))
    alone = {str(cfgs[k]["n"]): timed(lambda k=k: call(per[k], np.full(len(per[k]), k, np.int32))) for k in range(3)}
    s.close()
    return {"pairs": {str(cfgs[k]["n"]): int(counts[k]) for k in range(3)}, "mixed_ms": round(mixed, 4),
            "alone_ms": {k: round(v, 4) for k, v in alone.items()}, "sum_alone_ms": round(sum(alone.values()), 4),
            "gain_of_concurrent_groups": round(sum(alone.values()) / mixed, 3),
            "note": "search training calls only; each group alone vs the three groups in one call"}


def odd_side_rates(steps=10, warmup=3):
    """The paper's odd side 511 (Sec. IV-B's 0.2 m cells: stage-1 DFTs by Bluestein through 1024-point
    FFTs, stage 2 in the even frame 512) beside 512 on the same scene generator, 32 pairs each,
    n_theta 400: pairs/s of the forward and of the training step (graph replay, CUDA events, L2
    flushed before each timed call)."""
    import numpy as np
    import torch
    from paper_2203_00459_gb300 import _lib, synth
    from paper_2203_00459_gb300.search import PoseSearch, size_cfg
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda")
    out = {}
    for name in ("batch511", "batch512"):
        spec = synth.WORKLOADS[name]
        B = spec["pairs"]
        f, g, gt = synth.make_batch(name, pairs=B)
        fd, gd = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
        gtd = torch.from_numpy(gt.astype(np.float32)).cuda()
        srch = PoseSearch([size_cfg(spec["n"], spec["n_theta"], spec["n_r"])], max_pairs=B, flags=_lib.FLAG_GRAPH)
        pose = torch.empty((B, 3), device="cuda")
        outs = (pose, torch.empty(1, device="cuda"), torch.empty((B, 3), device="cuda"), torch.empty_like(fd),
                torch.empty_like(gd))

        def timed(fn):
            for _ in range(warmup):
                fn()
            ms = []
            for _ in range(steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn()
                b.record()
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            return sum(ms) / len(ms)

        ms_f = timed(lambda: srch.pose(fd, gd, out=pose))
        ms_t = timed(lambda: srch.pose_train(fd, gd, gtd, kind=2, out=outs))
        err = np.mean(np.abs(pose.cpu().numpy().astype(np.float64) - gt), axis=0)
        out[name] = {"n": spec["n"], "pairs": B, "fwd_pairs_per_s": B / (ms_f * 1e-3),
                     "step_pairs_per_s": B / (ms_t * 1e-3),
                     "mean_abs_err": {"theta_deg": float(np.degrees(err[0])), "tx_px": float(err[1]), "ty_px": float(err[2])}}
        srch.close()
    # Alg. 1's own settings at the paper's 511 (the f-raw rows of Tab. IIIa): n_theta 733 (direct
    # angle sums), T_theta 2, delta_xy 0.4, the radial-mean angle score and Alg. 1's stage 2; one
    # pair per call (the paper's batch of 1) and 32 pairs per call
    f, g, gt = synth.make_batch("batch511", pairs=32)
    fd, gd = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    cfg = size_cfg(511, 733, 255, temp_theta=2.0, delta_xy=0.4, angle_score=1, rotate_target=1)
    lit = {}
    for B in (1, 32):
        srch = PoseSearch([cfg], max_pairs=B, flags=_lib.FLAG_GRAPH)
        pose = torch.empty((B, 3), device="cuda")
        for _ in range(warmup):
            srch.pose(fd[:B], gd[:B], out=pose)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            srch.pose(fd[:B], gd[:B], out=pose)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        lit[f"batch{B}_fwd_pairs_per_s"] = B / (sum(ms) / len(ms) * 1e-3)
        srch.close()
    out["alg1_literal_511"] = dict(lit, config="n 511, n_theta 733, n_r 255, T_theta 2, delta_xy 0.4, radial-mean "
                                               "score, g turned back (Alg. 1 stage 2); forward, graph replay")
    return out


def frontend_rate(scans=64, n=256, delta_xy=0.4, steps=20, warmup=3):
    """Radar front end (fmbym_polar_to_cartesian) on Navtech-sized synthetic scans (400 azimuths x
    3768 range bins of 0.0438 m) to n x n Cartesian scans of delta_xy metres: scans/s (CUDA events,
    L2 flushed before each timed call) and its HBM roofline.  The compulsory bytes of a scan are
    the scan cells its bilinear taps touch, read once, plus the image written once."""
    import numpy as np
    import torch
    from paper_2203_00459_gb300 import synth
    from paper_2203_00459_gb300.search import polar_to_cartesian
    n_az, n_range, res = 400, 3768, 0.0438
    polar = torch.from_numpy(synth.make_polar_scans(scans, seed=9)).cuda()
    out = torch.empty((scans, n, n), device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda")
    for _ in range(warmup):
        polar_to_cartesian(polar, n, delta_xy, res, out=out)
    ms = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        polar_to_cartesian(polar, n, delta_xy, res, out=out)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = sum(ms) / len(ms)
    # cells touched by the taps (the same for every scan)
    idx = (np.arange(n) - n // 2) * delta_xy
    Y, X = np.meshgrid(idx, idx, indexing="ij")
    fa = np.mod(np.arctan2(Y, X), 2 * np.pi) * n_az / (2 * np.pi)
    fk = np.maximum(np.hypot(X, Y) / res - 0.5, 0.0)
    ok = fk <= n_range - 1
    a0 = np.floor(fa[ok]).astype(np.int64) % n_az
    k0 = np.minimum(np.floor(fk[ok]).astype(np.int64), n_range - 1)
    cells = np.unique(np.concatenate([((a0 + da) % n_az) * n_range + np.minimum(k0 + dk, n_range - 1)
                                      for da in (0, 1) for dk in (0, 1)])).size
    byts = scans * (cells * 4 + n * n * 4)
    peaks, src = measured_peaks()
    gbs = byts / (t * 1e-3) / 1e9
    return {"workload": f"{scans} polar scans {n_az} x {n_range} (0.0438 m) -> {n}^2 at {delta_xy} m",
            "scans_per_s": scans / (t * 1e-3), "ms": round(t, 4),
            "roofline": {"bound": "hbm", "alg_bytes_per_launch": int(byts), "achieved": round(gbs, 1),
                         "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(gbs / peaks["hbm_gbs"], 4),
                         "peak_source": src}}


def run_masked256(args):
    """The learned-mask training step at 256^2, batch 64: U-Net forward, masked search, L1 pose loss,
    search adjoint, U-Net adjoint and Adam.  `masked256` uses the 4-level 8..64-channel net,
    `masked256_tab2` the paper's 6-level 8..256-channel net of Tab. II."""
    import numpy as np
    import torch
    from paper_2203_00459_gb300 import build
    build.build()
    from paper_2203_00459_gb300 import train
    F, G, P = train.trajectory_data(2, 33, 20220304)
    channels = (8, 16, 32, 64, 128, 256) if args.workload == "masked256_tab2" else (8, 16, 32, 64)
    ms = train.MaskedSearch(batch=64, channels=channels)
    ms.net.set_conv_path(args.conv_path)
    Ft, Gt = torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda()
    Pt = torch.from_numpy(P.astype(np.float32)).cuda()
    for _ in range(args.warmup):
        ms.train_step(Ft, Gt, Pt)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        evs[k][0].record()
        ms.train_step(Ft, Gt, Pt)
        evs[k][1].record()
    torch.cuda.synchronize()
    ms_step = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    line = {"metric": "scan-pairs/s, learned-mask training step (U-Net fwd+bwd, search fwd+bwd, Adam)",
            "value": 64 / (ms_step * 1e-3), "unit": "scan-pairs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 mask, f32 search", "data": "synthetic",
            "config": {"workload": args.workload, "n": 256, "batch": 64, "mask_channels": list(channels),
                       "conv_path": ["mma.sync", "tcgen05"][args.conv_path]}}
    ms.close()
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.profile:
        return run_profile(args)
    from paper_2203_00459_gb300 import synth
    if args.workload == "mixed" and args.impl == "ours":
        return run_mixed(args)
    if args.workload in ("masked256", "masked256_tab2") and args.impl == "ours":
        return run_masked256(args)
    spec = dict(synth.WORKLOADS[args.workload if args.workload in synth.WORKLOADS else "batch256"])
    from paper_2203_00459_gb300 import replicas
    world, rank, local = replicas.world()
    if args.impl == "reference":
        if args.workload not in synth.WORKLOADS:
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the FP64 oracle arm times the search "
                                  f"workloads (batch512, batch256); {args.workload} has no timed oracle arm"}))
            return
        run_reference(args, spec, rank)
        return

    # the CPU pool for the oracle baseline is spawned before the first CUDA call
    pool = cores = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool, cores = make_pool()

    import numpy as np
    import torch
    from paper_2203_00459_gb300 import build
    build.build()
    from paper_2203_00459_gb300 import _lib
    from paper_2203_00459_gb300.search import PoseSearch, size_cfg

    torch.cuda.set_device(local)
    dist = replicas.init("nccl")

    B = spec["pairs"]
    n, nt, nr = spec["n"], spec["n_theta"], spec["n_r"]
    first, _ = replicas.shard(B, rank)
    f, g, gt = synth.make_batch(args.workload, pairs=B, start=first)
    cfg = size_cfg(n, nt, nr)
    # production path: graph replays, launch schedules picked by the library's autotuner
    search = PoseSearch([cfg], max_pairs=B, flags=_lib.FLAG_GRAPH | _lib.FLAG_AUTOTUNE)
    traced = PoseSearch([cfg], max_pairs=B)                          # direct launches, per-kernel events
    traced.set_tuning(0, **search.tuning(0))
    L = _lib.lib()
    fd = torch.from_numpy(f).cuda()
    gd = torch.from_numpy(g).cuda()
    gtd = torch.from_numpy(gt.astype(np.float32)).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    pose = torch.empty((B, 3), device="cuda")
    dpose = torch.empty((B, 3), device="cuda")
    loss = torch.empty(1, device="cuda")
    df = torch.empty_like(fd)
    dg = torch.empty_like(gd)

    def run_step(srch, fx, gx, gtx, px, dpx, lx, dfx, dgx, nb, separate=False):
        """One step through the library only.  fwd: the search.  fwdbwd: the search, the L2 pose loss
        (the 512^2 configuration's loss) and its adjoint in one training call, whose adjoint reads
        the forward's intermediates; separate=True makes the same step from the three separate
        calls, the adjoint then recomputing the forward."""
        st = torch.cuda.current_stream().cuda_stream
        if args.mode == "fwdbwd" and not separate:
            _lib.check(L.fmbym_pose_train(srch.handle, st, nb, None, None, fx.data_ptr(), gx.data_ptr(),
                                          gtx.data_ptr(), 2, px.data_ptr(), lx.data_ptr(), dpx.data_ptr(),
                                          dfx.data_ptr(), dgx.data_ptr()), srch.handle)
            return
        _lib.check(L.fmbym_pose(srch.handle, st, nb, None, None, fx.data_ptr(), gx.data_ptr(), px.data_ptr(), None,
                                None), srch.handle)
        if args.mode == "fwdbwd":
            _lib.check(L.fmbym_pose_loss(srch.handle, st, nb, px.data_ptr(), gtx.data_ptr(), 2, lx.data_ptr(),
                                         dpx.data_ptr()), srch.handle)
            _lib.check(L.fmbym_pose_backward(srch.handle, st, nb, None, None, fx.data_ptr(), gx.data_ptr(),
                                             dpx.data_ptr(), dfx.data_ptr(), dgx.data_ptr()), srch.handle)

    def step():
        run_step(search, fd, gd, gtd, pose, dpose, loss, df, dg, B)

    def traced_step():
        run_step(traced, fd, gd, gtd, pose, dpose, loss, df, dg, B)

    for _ in range(args.warmup):
        step()
        traced_step()
    torch.cuda.synchronize()

    # ---- timed region: K steps (CUDA-graph replays), per-step CUDA events, L2 flushed between ----
    launches0 = L.fmbym_launch_count(search.handle)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    replicas.barrier(dist)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record()
        step()
        evs[k][1].record()
    torch.cuda.synchronize()
    replicas.barrier(dist)
    clk = clocks.stop()
    launches = L.fmbym_launch_count(search.handle) - launches0
    ms = [a.elapsed_time(b) for a, b in evs]
    ms_step = replicas.max_over_ranks(sum(ms) / len(ms), dist, device="cuda")

    # ---- second timed region, same K steps launched directly with the library's tracer on: the
    # event before each launch gives every kernel's device time on the launching stream ----
    import ctypes
    _lib.check(L.fmbym_set_tracing(traced.handle, 1), traced.handle)
    tms = []
    for k in range(args.steps):
        flush.zero_()
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record()
        traced_step()
        b_.record()
        tms.append((a_, b_))
    torch.cuda.synchronize()
    ms_traced = sum(a_.elapsed_time(b_) for a_, b_ in tms) / len(tms)
    K = 32
    tot = (ctypes.c_double * K)()
    cnt = (ctypes.c_longlong * K)()
    nk = ctypes.c_int()
    _lib.check(L.fmbym_trace_summary(traced.handle, K, tot, cnt, ctypes.byref(nk)), traced.handle)
    _lib.check(L.fmbym_set_tracing(traced.handle, 0), traced.handle)
    kernels = {}
    for k in range(nk.value):
        if cnt[k]:
            kernels[L.fmbym_trace_kind_name(k).decode()] = (tot[k], cnt[k])

    value = replicas.job_rate(world, B, ms_step)

    # ---- dominant kernel roofline ----
    chunks = (nr + 15) // 16
    model = kernel_model(n, 3 * (n + (n & 1)) // 2, nt, nr, chunks)   # zero padding to P = 1.5 N (its even frame)
    total_ms = sum(v[0] for v in kernels.values())
    dom = max(kernels, key=lambda k: kernels[k][0]) if kernels else None
    peaks, peak_src = measured_peaks()
    roof = None
    shares = {k: round(v[0] / total_ms, 4) for k, v in kernels.items()} if total_ms else {}
    if dom and dom in model:
        avg_ms = kernels[dom][0] / kernels[dom][1]
        byts = model[dom][0] * B
        flops = model[dom][1] * B
        achieved = byts / (avg_ms * 1e-3) / 1e9
        tr = TRAFFIC.get(dom)
        tun = search.tuning(0)
        same = tr and tr[1] == src_hash() and (tr[3], tr[4]) == (tun["col_tile"], tun["col_plan"])
        traffic = tr[0] * B / tr[2] if same else None
        roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                "peak_source": peak_src, "alg_bytes_per_launch": byts, "avg_launch_ms": round(avg_ms, 5),
                "fp32_tflops": round(flops / (avg_ms * 1e-3) / 1e12, 2)}

    # the whole step against the same roofline: every kernel's compulsory bytes over the step time
    step_roof = None
    if args.mode == "fwdbwd":
        step_bytes = sum(model[k][0] for k in model if k in kernels) * B
        step_roof = {"alg_bytes_per_step": step_bytes, "achieved_gbs": round(step_bytes / (ms_step * 1e-3) / 1e9, 1),
                     "peak_gbs": peaks["hbm_gbs"], "frac": round(step_bytes / (ms_step * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)}

    # ---- end to end with host buffers ----
    e2e = None
    if rank == 0:
        fh = torch.from_numpy(f).pin_memory()
        gh = torch.from_numpy(g).pin_memory()
        if args.mode == "fwd":
            for _ in range(2):
                search.pose_host(fh, gh)
            t0 = time.perf_counter()
            reps = max(3, args.steps)
            for _ in range(reps):
                search.pose_host(fh, gh)
            dt = (time.perf_counter() - t0) / reps
            e2e = {"value": B / dt, "unit": "scan-pairs/s", "h2d_bytes_per_step": 2 * f.nbytes,
                   "d2h_bytes_per_step": B * 12, "mode": "fwd", "api": "fmbym_pose_host"}
        else:
            # the public host-buffer training call: H2D of f, g and gt, the training call, D2H of
            # pose, loss, df and dg, all inside fmbym_pose_train_host (which synchronises)
            gth = torch.from_numpy(gt.astype(np.float32)).pin_memory()
            outs = (torch.empty((B, 3), pin_memory=True), torch.empty(1, pin_memory=True),
                    torch.empty(fh.shape, pin_memory=True), torch.empty(gh.shape, pin_memory=True))
            for _ in range(2):
                search.pose_train_host(fh, gh, gth, kind=2, out=outs)
            reps = max(3, args.steps)
            t0 = time.perf_counter()
            for _ in range(reps):
                search.pose_train_host(fh, gh, gth, kind=2, out=outs)
            dt = (time.perf_counter() - t0) / reps
            e2e = {"value": B / dt, "unit": "scan-pairs/s", "h2d_bytes_per_step": 2 * f.nbytes + B * 12,
                   "d2h_bytes_per_step": B * 12 + 4 + 2 * f.nbytes, "mode": "fwdbwd",
                   "api": "fmbym_pose_train_host (pinned host f, g, gt in; pose, loss, df, dg out)"}

    # ---- forward-only rate and the plain one-pair-per-call path ----
    extra = {}
    if rank == 0:
        fwd_ms = []
        for _ in range(max(3, args.steps // 2)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            search.pose(fd, gd, out=pose)
            b.record()
            torch.cuda.synchronize()
            fwd_ms.append(a.elapsed_time(b))
        extra["fwd_pairs_per_s"] = B / (statistics.mean(fwd_ms) * 1e-3)
        if args.mode == "fwdbwd":
            # the same step as three calls (pose, loss, backward with its forward recompute)
            sep_ms = []
            for _ in range(max(3, args.steps // 2)):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                run_step(search, fd, gd, gtd, pose, dpose, loss, df, dg, B, separate=True)
                b.record()
                torch.cuda.synchronize()
                sep_ms.append(a.elapsed_time(b))
            extra["separate_calls_pairs_per_s"] = B / (statistics.mean(sep_ms[1:]) * 1e-3)
        if not args.no_plain:
            one = PoseSearch([cfg], max_pairs=1)
            for label, mode in (("fwd", "fwd"), ("step", args.mode)):
                plain = []
                for _ in range(3):
                    flush.zero_()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    for i in range(B):
                        if mode == "fwd":
                            one.pose(fd[i:i + 1], gd[i:i + 1], out=pose[i:i + 1])
                        else:
                            run_step(one, fd[i:i + 1], gd[i:i + 1], gtd[i:i + 1], pose[i:i + 1], dpose[i:i + 1],
                                     loss, df[i:i + 1], dg[i:i + 1], 1)
                    b.record()
                    torch.cuda.synchronize()
                    plain.append(a.elapsed_time(b))
                extra[f"plain_{label}_pairs_per_s"] = B / (statistics.mean(plain[1:]) * 1e-3)
            extra["batched_vs_plain_fwd"] = extra["fwd_pairs_per_s"] / extra["plain_fwd_pairs_per_s"]
            extra["batched_vs_plain_step"] = value / extra["plain_step_pairs_per_s"]
            one.close()

    # ---- the FP32 ceiling, measured on this GPU in this run, and the path-level floor ----
    from paper_2203_00459_gb300.search import fp32_fma_rate
    fp32_peak = 2.0 * fp32_fma_rate()          # FLOP/s
    if roof is not None:
        roof["fp32_peak_tflops_measured"] = round(fp32_peak / 1e12, 2)
        roof["fp32_frac"] = round(model[dom][1] * B / (roof["avg_launch_ms"] * 1e-3) / fp32_peak, 4)
    step_flop = sum(model[k][1] for k in model if k in kernels) * B
    io_bytes = (28 if args.mode == "fwdbwd" else 12) * n * n * B   # scans in, scores / gradients out
    t_floor = max(io_bytes / (peaks["hbm_gbs"] * 1e9), step_flop / fp32_peak)
    extra["step_floor"] = {
        "io_bytes_per_step": io_bytes, "fft_flop_per_step": step_flop,
        "fp32_peak_tflops_measured": round(fp32_peak / 1e12, 2), "hbm_gbs": peaks["hbm_gbs"],
        "t_floor_ms": round(t_floor * 1e3, 5), "bound": "fp32" if step_flop / fp32_peak > io_bytes / (peaks["hbm_gbs"] * 1e9) else "hbm",
        "frac": round(t_floor / (ms_step * 1e-3), 4),
        "note": "T_floor = max(inputs+outputs / HBM, nominal 5 L log2 L FFT FLOPs of the step / measured FP32 peak)"}

    if rank == 0 and args.workload == WORKLOAD:
        extra["exhaustive_256"] = exhaustive_comparison()
        extra["alg1_n_theta_733"] = angle_count_comparison(fp32_peak / 2.0)
        extra["radar_frontend"] = frontend_rate()
        extra["odd_side_511"] = odd_side_rates()
        extra["mixed_concurrency"] = mixed_concurrency()

    cpu = None
    if pool is not None:
        sample = min(B, cores)   # one pair per core: a bounded sample of the batch
        rate = oracle_rate(f, g, gt, spec, args.mode, sample, pool)
        pool.close()
        cpu = {"value": rate, "unit": "scan-pairs/s", "cores": cores, "kind": "oracle",
               "sample": f"the first {sample} of the {B} pairs of {args.workload} ({args.mode}), one pair per "
                         f"process, spawn pool"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "scan-pairs/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "mode": args.mode,
                "config": {"workload": args.workload, "n": n, "n_theta": nt, "n_r": nr, "pairs_per_gpu": B,
                           "pad": "zero to 1.5N (same lags as 2N)", "l2": "flushed (256 MB write) between timed steps",
                           "schedules": search.tuning(0)},
                "roofline": roof, "step_roofline": step_roof, "kernel_shares": shares,
                "ms_per_step_direct_launch": ms_traced,
                "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clk, **extra}
        print(json.dumps(line), flush=True)
    search.close()
    traced.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
