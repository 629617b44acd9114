#!/usr/bin/env python3
"""Throughput of PlanarSplatting's forward + backward plane splatting on GB300.

Workload (the paper-scale single-scene configuration): a synthetic 8x10x3 m
room with furniture, 2,000 ground-truth rectangles, 64 views at 640x480
(fx = fy = 500) on a smooth trajectory; 3,000 planes initialised at random
surface points with random orientation and radii 0.2 m; one step renders
8 views (rotating through the 64), computes the Eq. 14 loss against the exact
ground-truth depth/normal maps, back-propagates to the planes and takes an
Adam step -- every call a libps kernel.  Inputs are synthetic (the paper's
ScanNet scenes are not available) and resident in HBM.

Metric: Mpixel-views/s = 8 * 640 * 480 / (time of one step) / 1e6, device
time by CUDA events on the launching stream, L2 flushed (256 MB write) between
steps outside the timed events.  `e2e` repeats it through host buffers (the
step's ground-truth maps copied from pinned host memory and the loss sums
read back, inside the timed region).  `roofline` reports the dominant kernel
against the FP32 ALU peak, with its algorithmic work counted exactly by
ps_count_pairs.  `cpu_baseline` times the FP64 oracle on a bounded sample.

`--impl reference` times the oracle (the CPU definition of the method) on a
bounded sample per step and prints the same line with "impl": "reference".
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

from paper_2412_03451_gb300 import ranks as RK  # noqa: E402

METRIC = "fwd+bwd splat Mpixel-views/s & time-to-depth-err≤2cm vs plain, 1×GB300"
UNIT = "Mpixel-views/s"
CAPACITY_BIT = 1 << 3          # PS_ERR_CAPACITY in the device status word
H, W, F = 480, 640, 500.0
N_VIEWS, VIEWS_PER_STEP, N_GT, N_INIT = 64, 8, 2000, 3000

# FP32 operation counts of the method's formulas (FMA = 2, MUFU op = 1), used
# for the algorithmic work of the roofline:
#   per candidate pair (Eq. 4, 6-9): d.n 4, t 2, d.v^x d.v^y 8, P_X P_Y 4,
#     margins 2, min 1, weight 6                                       = 27
#   per composited pair, forward (Eq. 11-13): T w 1, D 2, N 6, alpha 1,
#     T(1 - w) 2                                                        = 12
#   per composited pair, backward: T(1 - w) 2 + adjoint of Eq. 11-13 16
#     + A, B updates 12 + Eq. 7-9 chain 5 + Eq. 6 chain 7 + Eq. 4 chain 8
#     + record accumulation 16                                         = 66
FLOP_CAND, FLOP_COMP_FWD, FLOP_COMP_BWD = 27, 12, 66
# special-function (MUFU) operations of the same formulas: per candidate pair a
# reciprocal for t (Eq. 4), an exponential and a reciprocal for the sigmoid (Eq. 7-8);
# per composited pair, backward: those three again plus the reciprocal of d.n (Eq. 4)
MUFU_CAND, MUFU_COMP_BWD = 3, 4
MUFU_PER_SM_CLK = 16           # special-function results per SM per clock
SM_COUNT, FP32_LANES = 152, 128
# kernels of one step: schedule advance 1 (graphs); project 1; bin: record counts 1, scans
# (record and tile scans in one launch when both fit one CTA, 49,152 elements; beyond, the
# record scan takes three launches plus the chunk table 1 and the tile scan six), scatter 1,
# sorts 2; fused splat 1 + chain 1 (split: fwd 1, loss 1, bwd 1 + chain 1); Adam 2
ONE_CTA_SCAN = 48 * 1024


def roofline_entry(counts, stages, K, clocks, sha, peaks, regime=0):
    """Roofline of the dominant splat kernel from the exact work counts of K launches
    (tested, candidate, composited pairs), the per-stage CUDA-event times (ms lists),
    the sampled clocks, the kernel source hash (profile-derived constants apply only
    to the source they were taken on) and the measured peaks.  FP32 work of the
    formulas against the FP32 peak; special functions, instruction issue and DRAM
    as the other roofs."""
    tested, cand, comp = counts
    sm_clock = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = SM_COUNT * FP32_LANES * 2 * sm_clock * 1e6 / 1e12
    if "splat_fused" in stages:
        # one walk: candidates evaluated once, composited pairs forward + adjoint
        dom, dom_ms = "splat_fused", statistics.mean(stages["splat_fused"])
        flops = (cand * FLOP_CAND + comp * (FLOP_COMP_FWD + FLOP_COMP_BWD)) / K
    else:
        fwd_ms = statistics.mean(stages["splat_fwd"])
        bwd_ms = statistics.mean(stages["splat_bwd"])
        dom = "splat_bwd" if bwd_ms >= fwd_ms else "splat_fwd"
        dom_ms = max(fwd_ms, bwd_ms)
        flops = ((cand * FLOP_CAND + comp * FLOP_COMP_BWD) if dom == "splat_bwd"
                 else (cand * FLOP_CAND + comp * FLOP_COMP_FWD)) / K
    achieved = flops / (dom_ms / 1e3) / 1e12
    cap = CAPTURES.get(dom, {}).get(regime) if CAPTURES.get("src_sha") == sha else None
    traffic = cap["dram_bytes"] if cap else None
    roofline = {"bound": "alu", "kernel": dom, "achieved": round(achieved, 4), "peak": round(peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_basis": "152 SMs x 128 FP32 lanes x 2 (FMA) x %.0f MHz" % sm_clock,
                "per_launch": {"candidate_pairs": cand // K, "composited_pairs": comp // K,
                               "tested_pairs": tested // K, "ms": round(dom_ms, 4)}}
    mufu = (cand * MUFU_CAND + (comp * MUFU_COMP_BWD if dom != "splat_fwd" else 0)) / K
    mufu_peak = SM_COUNT * MUFU_PER_SM_CLK * sm_clock * 1e6 / 1e12
    roofline["other_roofs"] = {
        "mufu": {"achieved": round(mufu / (dom_ms / 1e3) / 1e12, 4), "peak": round(mufu_peak, 3),
                 "unit": "Tops/s", "frac": round(mufu / (dom_ms / 1e3) / 1e12 / mufu_peak, 4),
                 "peak_basis": "152 SMs x 16 per clock x %.0f MHz" % sm_clock}}
    instr = cap["warp_instructions"] if cap else None
    if instr:
        ips = instr / (dom_ms / 1e3) / 1e9
        ipeak = SM_COUNT * SCHEDULERS_PER_SM * sm_clock * 1e6 / 1e9
        roofline["other_roofs"]["issue"] = {
            "achieved": round(ips, 1), "peak": round(ipeak, 1), "unit": "G warp instructions/s",
            "frac": round(ips / ipeak, 4),
            "peak_basis": "152 SMs x 4 schedulers x %.0f MHz; instructions from the ncu capture of one "
                          "launch of the same kernel source" % sm_clock}
    if traffic and (peaks or {}).get("hbm_gbs"):
        gbs = traffic / (dom_ms / 1e3) / 1e9
        roofline["other_roofs"]["hbm"] = {"achieved": round(gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                          "frac": round(gbs / peaks["hbm_gbs"], 4),
                                          "peak_basis": "measured copy bandwidth (ncu DRAM bytes of the launch)"}
    return roofline


def measured_peaks() -> dict:
    """The copy bandwidth and GEMM rates measured on the GPUs this runs on (MEASURED_PEAKS.json
    at the repository root), or {} if the file is absent."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def scan_launches(n: int, twice: bool = False) -> int:
    if n <= ONE_CTA_SCAN:
        return 1
    return 6 if twice else 3


def step_launches(n_records: int, n_tiles: int, fused: bool, graph: bool = True) -> int:
    """Kernels of libps per optimisation step: schedule advance (graph only), projection,
    binning (counts, scans, scatter, two sorts), splat (+ chain), Adam (one launch for all
    parameters in the graph step, two eagerly)."""
    if 0 < n_records <= ONE_CTA_SCAN and n_tiles <= ONE_CTA_SCAN:
        scans = 1
    else:
        scans = (scan_launches(n_records) + 1 if n_records > 0 else 0) + scan_launches(n_tiles, True)
    binning = 1 + scans + 3
    adam = 1 if graph else 2
    return (int(graph) + 1 + binning + 2 + adam) if fused else (int(graph) + 1 + binning + 4 + adam)

# DRAM bytes (read + write) and warp instructions (smsp__inst_executed.sum) per launch
# of the fused splat kernel from the ncu captures summarised in
# profiles/k_splat_fused_room640_8x8_ite3.md (the benchmark's first lambda) and
# .._ite1000.md, .._ite2000.md, .._ite4000.md (later points of the fit), keyed by the
# regime's iteration; reported only while the kernel source is the one they were taken
# on.  The issue roof is 152 SMs x 4 schedulers x one warp instruction per clock.
CAPTURES = {"src_sha": "f57b7307b034ad09",
            "splat_fused": {0: {"dram_bytes": 51238656, "warp_instructions": 392692133},
                            1000: {"dram_bytes": 44233728, "warp_instructions": 152681978},
                            2000: {"dram_bytes": 42898176, "warp_instructions": 122084604},
                            4000: {"dram_bytes": 42422784, "warp_instructions": 109970373}}}
SCHEDULERS_PER_SM = 4


def src_hash() -> str:
    p = os.path.join(ROOT, "paper_2412_03451_gb300", "csrc", "ps_splat.cu")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", default="auto", choices=["auto", "16x16", "8x8", "32x8"])
    ap.add_argument("--warps", type=int, default=0, choices=[0, 2, 4, 8],
                    help="warps per CTA of the splat kernels when --tile is given (0: library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ttd", type=int, default=0,
                    help="also fit up to this many iterations and report time to depth error <= 2 cm")
    ap.add_argument("--fit-iters", type=int, default=2000,
                    help="also run the single-scene fit of the benchmark room for this many iterations "
                         "from its initial planes, replayed from graphs (0: skip)")
    ap.add_argument("--start-ite", type=int, default=0, help="iteration (lambda schedule) to start at")
    ap.add_argument("--no-graphs", action="store_true", help="time eager launches instead of graph replays")
    ap.add_argument("--regimes", default="1000,2000,4000",
                    help="iterations of a real fit of the same room at which stage times and the roofline "
                         "are measured again (lambda 20, 54, 300); empty: none")
    ap.add_argument("--batched", type=int, default=32,
                    help="rooms in the batched-vs-plain time-to-2cm comparison (0: skip)")
    ap.add_argument("--batched-iters", type=int, default=5000)
    ap.add_argument("--ablation", type=int, default=0,
                    help="rooms of the Sec. 4.3 ablation (init variants, single radii); 0 = skip")
    ap.add_argument("--ablation-variants", default="plain,mono,sphere,single_radii,split,split_low,gaussian")
    ap.add_argument("--profile-ite", type=int, default=0,
                    help="with --profile-case: fit this many iterations before the profiled step")
    ap.add_argument("--profile-case", action="store_true",
                    help="for ncu: set up, warm up 3 steps, run one step inside a profiler range, exit")
    ap.add_argument("--stress", action="store_true",
                    help="time the differentiation-stress room (10,000 planes, 256 views) and exit")
    ap.add_argument("--profile-gemm", action="store_true",
                    help="the seed network's tcgen05 GEMM (65,536 x 64 x 576): time it, then run one "
                         "inside a profiler range (for ncu), exit")
    return ap.parse_args()


def workload_config(args, world):
    return {"workload": "synthetic room 8x10x3 m, %d GT rectangles, %d planes, %d of %d views "
                        "per step at %dx%d" % (N_GT, N_INIT, VIEWS_PER_STEP, N_VIEWS, W, H),
            "views_per_step": VIEWS_PER_STEP, "image": [H, W], "planes": N_INIT,
            "M": 30, "l2": "flushed between steps (256 MB write, outside the timed events)",
            "start_iteration": args.start_ite, "replicas": world,
            "seed": "scene 1000 + rank, init 2000 + rank"}


# ---------------------------------------------------------------------------
# Clock sampling during the timed region.

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, path=None):
        self.index = index
        self.proc = None
        self.path = path

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        if self.path:
            try:
                with open(self.path, "w") as f:
                    f.write(out)
            except OSError:
                pass
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# Our arm.

class Workload:
    def __init__(self, rank: int, tile, device, warps=0):
        import numpy as np
        import torch
        from paper_2412_03451_gb300 import binding as B
        from paper_2412_03451_gb300 import scenes as S
        from paper_2412_03451_gb300 import splat as SP
        self.torch, self.B, self.SP = torch, B, SP
        seeds = RK.rank_seeds(rank)
        self.room = S.large_room(seeds["scene"], n_rect=N_GT, n_views=N_VIEWS, H=H, W=W, f=F)
        self.init = S.surface_init(self.room, N_INIT, seeds["init"])
        cams = self.room.cams
        # ground truth: exact ray casting of the GT rectangles with the library's hard mode
        gtr = SP.Renderer([H] * N_VIEWS, [W] * N_VIEWS, [0] * N_VIEWS, [0, N_GT], tile=tile,
                          device=device, flags=B.PS_HARD)
        gtr.set_cameras(cams.w2c, cams.intr)
        gflat = SP.planes_to_flat(self.room.gt.center, self.room.gt.quat, self.room.gt.radii,
                                  device)
        gtr.ensure_capacity(gflat, 300.0)
        gtr.forward(gflat, 300.0)
        torch.cuda.synchronize()
        self.gt_depth = gtr.depth.clone()
        self.gt_normal = gtr.normal.clone()
        del gtr
        self.r = SP.Renderer([H] * VIEWS_PER_STEP, [W] * VIEWS_PER_STEP, [0] * VIEWS_PER_STEP,
                             [0, N_INIT], tile=tile, device=device, warps=warps)
        nb = N_VIEWS // VIEWS_PER_STEP
        self.r.preplan([cams.w2c[b * VIEWS_PER_STEP:(b + 1) * VIEWS_PER_STEP] for b in range(nb)],
                       [cams.intr[b * VIEWS_PER_STEP:(b + 1) * VIEWS_PER_STEP] for b in range(nb)])
        self.flat = SP.planes_to_flat(self.init.center, self.init.quat, self.init.radii, device)
        self.fit = SP.Fitter(self.r, self.flat)
        self.hw = H * W
        self.np = np

    def reset(self, ite=0):
        SP = self.SP
        self.flat.copy_(SP.planes_to_flat(self.init.center, self.init.quat, self.init.radii,
                                          self.flat.device))
        self.fit.m.zero_()
        self.fit.v.zero_()
        self.fit.ite = ite

    def gt_slice(self, s):
        b = (s % (N_VIEWS // VIEWS_PER_STEP)) * VIEWS_PER_STEP
        n = VIEWS_PER_STEP * self.hw
        return (self.gt_depth[b * self.hw:b * self.hw + n],
                self.gt_normal[b * self.hw:b * self.hw + n])

    def step(self, s, marks=None, gt=None):
        self.r.select(s % (N_VIEWS // VIEWS_PER_STEP))
        gd, gn = self.gt_slice(s) if gt is None else gt
        return self.fit.step(gd, gn, marks=marks)

    def grow_if_needed(self, s) -> bool:
        """Checks the tile-list capacity for step s's views at the current state."""
        self.r.select(s % (N_VIEWS // VIEWS_PER_STEP))
        lam = self.B.lambda_schedule(self.fit.ite)
        return self.r.ensure_capacity(self.flat, lam, headroom=1.6)


def time_steps(wl, first, K, flush, counts_out=None):
    """Times K steps starting at step index `first`; returns per-stage ms lists."""
    torch = wl.torch
    stages = {}
    per_step = []
    counts = torch.zeros(3, dtype=torch.int64, device=wl.flat.device)
    tot = torch.zeros(3, dtype=torch.int64, device=wl.flat.device)
    pairs = []
    for i in range(K):
        flush.zero_()
        marks = []
        wl.step(first + i, marks=marks)
        pairs.append(marks)
        if counts_out is not None:
            wl.r.count_pairs(counts)
            tot += counts
    torch.cuda.synchronize()
    for marks in pairs:
        t0 = marks[0][1]
        per_step.append(t0.elapsed_time(marks[-1][1]))
        for (a, ea), (b, eb) in zip(marks[:-1], marks[1:]):
            stages.setdefault(b, []).append(ea.elapsed_time(eb))
    if counts_out is not None:
        counts_out.extend(int(x) for x in tot.cpu().tolist())
    return per_step, stages


def autotune_tile(rank, device):
    """Picks the tile shape and the warps per CTA (the planes staged per
    shared-memory batch) for this workload by timing each pair on its first
    camera batch (outside every timed region)."""
    from paper_2412_03451_gb300 import autotune
    from paper_2412_03451_gb300 import splat as SP
    wl = Workload(rank, (16, 16), device)
    gd, gn = wl.gt_slice(0)
    cams = wl.room.cams

    def make(tile, warps):
        r = SP.Renderer([H] * VIEWS_PER_STEP, [W] * VIEWS_PER_STEP, [0] * VIEWS_PER_STEP,
                        [0, N_INIT], tile=tile, device=device, warps=warps)
        r.set_cameras(cams.w2c[:VIEWS_PER_STEP], cams.intr[:VIEWS_PER_STEP])
        return r

    key = autotune.key_for([(H, W)], VIEWS_PER_STEP, N_INIT)
    tile, warps, times = autotune.pick_launch(make, wl.flat, gd, gn, wl.B.lambda_schedule(0), key)
    del wl
    return tile, warps, times


def time_replays(wl, first, K, flush):
    """Times K graph replays (one optimisation step each) from step index `first`."""
    torch = wl.torch
    nb = N_VIEWS // VIEWS_PER_STEP
    evs = []
    for i in range(K):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        wl.fit.replay((first + i) % nb)
        e1.record()
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def run_ours(args, rank, world, local_rank):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    device = "cuda:%d" % local_rank
    torch.cuda.set_device(local_rank)
    tuning = None
    warps = args.warps
    if args.tile == "auto":
        tile, warps, tuning = autotune_tile(rank, device)
    else:
        tile = tuple(int(x) for x in args.tile.split("x"))
    wl = Workload(rank, tile, device, warps)
    wl.reset(args.start_ite)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)
    nb = N_VIEWS // VIEWS_PER_STEP

    # warm-up (capacity checks happen here, never inside the timed region)
    W0 = max(args.warmup, 3)
    for i in range(W0):
        wl.grow_if_needed(i)
        wl.step(i)
    torch.cuda.synchronize()
    first = W0
    for s in range(first, first + args.steps):
        wl.grow_if_needed(s)   # state at the start of timing: make room for every view batch
    wl.r.status.zero_()
    saved = (wl.flat.clone(), wl.fit.m.clone(), wl.fit.v.clone(), wl.fit.ite)
    # clocks are sampled from here to the end of the timed pass (both passes keep the GPU busy)
    # the raw samples are also written out when PS_CLOCKS_DIR names a directory
    cdir = os.environ.get("PS_CLOCKS_DIR")
    clk = ClockSampler(local_rank, os.path.join(cdir, "clocks_r%d.csv" % rank)
                       if cdir and os.path.isdir(cdir) else None)
    clk.start()

    # pass 1 (eager launches): per-stage CUDA events and exact work counts
    counts = []
    per_step_eager, stages = time_steps(wl, first, args.steps, flush, counts_out=counts)
    status = int(wl.r.status.item())
    if status & CAPACITY_BIT:
        raise RuntimeError("tile-list capacity overflow inside the timed region")

    use_graphs = not args.no_graphs
    if use_graphs:
        # pass 2 (headline): the same iterations replayed from captured CUDA graphs
        wl.flat.copy_(saved[0]); wl.fit.m.copy_(saved[1]); wl.fit.v.copy_(saved[2])
        wl.fit.ite = saved[3]
        wl.fit.enable_graphs(first + args.steps + 8, list(range(nb)),
                             [wl.gt_slice(b) for b in range(nb)])
        wl.r.status.zero_()
    RK.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    if use_graphs:
        per_step = time_replays(wl, first, args.steps, flush)
    else:
        wl.flat.copy_(saved[0]); wl.fit.m.copy_(saved[1]); wl.fit.v.copy_(saved[2])
        wl.fit.ite = saved[3]
        per_step, _ = time_steps(wl, first, args.steps, flush)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clocks = clk.stop()
    status = int(wl.r.status.item())
    if status & CAPACITY_BIT:
        raise RuntimeError("tile-list capacity overflow inside the timed region")

    # slowest rank's device time; units summed over ranks (each renders its own room)
    dev_ms = RK.max_over_ranks(sum(per_step), device)
    RK.barrier()
    pix = VIEWS_PER_STEP * H * W
    value = RK.job_throughput(RK.sum_over_ranks(pix * args.steps, device), dev_ms / 1e3) / 1e6

    tested, cand, comp = counts
    roofline = roofline_entry(counts, stages, args.steps, clocks, src_hash(), measured_peaks())

    cfg = workload_config(args, world)
    cfg["tile"] = "%dx%d" % tile
    cfg["warps_per_cta"] = warps or 4
    if tuning:
        cfg["autotune_ms"] = {k: round(v, 4) for k, v in tuning.items()}
    cfg["launch"] = "captured CUDA graph per step" if use_graphs else "eager launches"
    result = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dev_ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": cfg,
        "stage_ms": {k: round(statistics.mean(v), 4) for k, v in stages.items()},
        "eager_ms_per_step": round(sum(per_step_eager) / args.steps, 4),
        "wall_s_timed": round(wall, 4),
        "roofline": roofline, "clocks": clocks,
        "gpu_launches": step_launches(int(wl.r.frame.n_records), int(wl.r.frame.n_tiles),
                                      wl.fit.fused, graph=use_graphs) * args.steps,
        "culling": {"tested_per_candidate": round(tested / max(cand, 1), 2)},
    }

    if not args.no_e2e:
        # the same iterations as the headline, from the same state
        wl.flat.copy_(saved[0]); wl.fit.m.copy_(saved[1]); wl.fit.v.copy_(saved[2])
        wl.fit.ite = saved[3]
        result["e2e"] = run_e2e(wl, args, first, world)
    cps = [int(x) for x in args.regimes.split(",") if x.strip()]
    if cps:
        result["regimes"] = run_regimes(wl, cps, args.steps, clocks, measured_peaks())
    if args.fit_iters > 0:
        result["fit"] = run_fit(wl, args.fit_iters)
        # the paper's own figure, quoted with the hardware it states (context: another dataset,
        # GPU and per-iteration batch; no ratio is formed from it)
        result["paper_context"] = {
            "paper_per_scene_s": 180, "paper_hardware": "one GPU, model not stated",
            "paper_workload": "ScanNetV2 scene, 480x640 images, 5,000 Adam iterations, about 2,000 initial planes",
            "ours_single_scene_fit_s": result["fit"]["device_s"],
            "ours_workload": "the synthetic room above, %d iterations of %d views" % (args.fit_iters, VIEWS_PER_STEP)}
    if args.ttd:
        result["time_to_2cm"] = run_ttd(wl, args.ttd)
    if args.batched > 0:
        del wl
        torch.cuda.empty_cache()
        result["time_to_2cm_vs_plain"] = run_batched(args, rank, device)
    if args.ablation > 0:
        from paper_2412_03451_gb300 import ablation
        torch.cuda.empty_cache()
        result["ablation_time_to_2cm"] = ablation.run(n_rooms=args.ablation, iters=args.batched_iters,
                                                      seed0=7000 + 100 * rank, device=device,
                                                      variants=tuple(args.ablation_variants.split(",")))
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        from paper_2412_03451_gb300 import scenes as S
        room = S.large_room(1000 + rank, n_rect=N_GT, n_views=N_VIEWS, H=H, W=W, f=F)
        result["cpu_baseline"] = cpu_baseline(room, S.surface_init(room, N_INIT, 2000 + rank),
                                              args.start_ite)
        result["cpu_baseline"]["tiny_room"] = tiny_room_timing(device)
    return result


def run_batched(args, rank, device):
    """Time to mean depth error <= 2 cm of uneven rooms (plane counts U{200..3000},
    views U{16..96}, resolutions 320x240 / 480x360 / 640x480): every room to
    2 cm or the iteration cap, GPU seconds by CUDA events (convergence checks
    and frame rebuilds excluded).
      plain:           plain initialisation (random surface points and
                       orientations, radii half the nearest-neighbour spacing,
                       Sec. 3.1), rooms fitted one by one;
      batched:         the same initialisation, all rooms in one launch per
                       kernel per step, rooms leaving the batch when done;
      batched_offset:  the plain initialisation batched, with Eq. 10 started
                       at the learned arm's offset (control: what the later
                       lambda start alone gains);
      batched_learned: network-proposed initialisation (inference time
                       included), batched.
    Besides the totals (capped rooms stop at the cap), every arm reports the
    rooms it brings to 2 cm; then the rooms that every arm reaches are fitted
    again by each batched arm on their own (the batch's clock would otherwise
    include the rooms that never converge), against the sum of their one-by-one
    fit times, with their mean iterations to 2 cm."""
    import torch
    from paper_2412_03451_gb300 import autotune
    from paper_2412_03451_gb300 import batch as BT
    from paper_2412_03451_gb300 import scenes as S
    from paper_2412_03451_gb300 import seed_train as ST
    n = args.batched
    rooms = S.batch_rooms(n, seed0=3000 + 100 * rank)
    inits = [S.surface_init_nn(room, K, 4000 + 100 * rank + i) for i, (room, K) in enumerate(rooms)]
    ss = BT.SceneSet([r for r, _ in rooms], inits, device=device)

    def make(tile, warps):
        ss.tile, ss.warps = tile, warps
        r = ss.renderer()
        r.select(0)
        return r

    key = autotune.key_for([(rm.cams.H, rm.cams.W) for rm in ss.rooms], ss.vps * n, sum(ss.K))
    tile, warps, tuning = autotune.pick_launch(make, ss.flat_init(), ss.gt_depth, ss.gt_normal,
                                               20.0 / 2.718281828459045, key)
    ss.tile, ss.warps = tile, warps
    plain = [BT.fit_until(ss, [s], max_iters=args.batched_iters) for s in range(n)]
    bat = BT.fit_until(ss, list(range(n)), max_iters=args.batched_iters)
    off = BT.fit_until(ss, list(range(n)), max_iters=args.batched_iters,
                       lam_offset=ST.LEARNED_LAM_OFFSET)
    arms = {"plain": [p["done_at"][0] for p in plain], "batched": bat["done_at"],
            "batched_offset": off["done_at"]}
    t_plain = sum(p["gpu_ms"] for p in plain) / 1e3
    t_bat = bat["gpu_ms"] / 1e3
    out = {"rooms": n, "what": "GPU seconds to fit every room to mean depth error <= 2 cm "
                               "(rooms that have not reached it by the iteration cap stop there)",
           "plain_s": round(t_plain, 3), "batched_s": round(t_bat, 3),
           "speedup_batched": round(t_plain / t_bat, 3) if t_bat > 0 else None,
           "reached_plain": sum(p["done_at"][0] is not None for p in plain),
           "reached_batched": sum(d is not None for d in bat["done_at"]),
           "iteration_cap": args.batched_iters, "tile": "%dx%d" % tile, "warps_per_cta": warps,
           "autotune_ms": {k: round(v, 4) for k, v in tuning.items()},
           "batched_offset_s": round(off["gpu_ms"] / 1e3, 3),
           "reached_batched_offset": sum(d is not None for d in off["done_at"]),
           "init_plain": "random surface points, random orientation, radii 0.5 x nearest-neighbour distance"}
    net = ST.load(device=device)
    if net is None:
        out["batched_learned"] = "no trained weights"
        return out
    # warm the network's kernels once (first-call set-up is not inference)
    r0 = ss.rooms[0]
    c0 = r0.cams
    ST.propose_planes(net, r0, ss.gt_depth[:c0.H * c0.W].view(1, c0.H, c0.W),
                      ss.gt_normal[:c0.H * c0.W].view(1, c0.H, c0.W, 3), [0], max_planes=100)
    learned, infer_ms, infer_room = [], 0.0, []
    for i, room in enumerate(ss.rooms):
        c = room.cams
        off = int(ss.gt_off[i][0])
        m = c.V * c.H * c.W
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        P, _, _ = ST.propose_planes(net, room, ss.gt_depth[off:off + m].view(c.V, c.H, c.W),
                                    ss.gt_normal[off:off + m].view(c.V, c.H, c.W, 3), range(c.V),
                                    seed=5000 + i, max_planes=ss.K[i])
        e1.record()
        torch.cuda.synchronize()
        infer_ms += e0.elapsed_time(e1)
        infer_room.append(e0.elapsed_time(e1))
        learned.append(P)
    ss_l = BT.SceneSet(ss.rooms, learned, device=device, tile=tile, warps=warps)
    bl = BT.fit_until(ss_l, list(range(n)), max_iters=args.batched_iters,
                      lam_offset=ST.LEARNED_LAM_OFFSET)
    t_bl = bl["gpu_ms"] / 1e3 + infer_ms / 1e3
    out.update({"batched_learned_s": round(t_bl, 3), "learned_inference_s": round(infer_ms / 1e3, 3),
                "speedup_batched_learned": round(t_plain / t_bl, 3) if t_bl > 0 else None,
                "reached_batched_learned": sum(d is not None for d in bl["done_at"]),
                "learned_lambda_start_iteration": ST.LEARNED_LAM_OFFSET})
    arms["batched_learned"] = bl["done_at"]
    common, cr = common_rooms(arms)
    if common:
        cap = args.batched_iters
        refit = {"plain": sum(plain[s]["gpu_ms"] for s in common)}
        rb = BT.fit_until(ss, common, max_iters=cap)
        ro = BT.fit_until(ss, common, max_iters=cap, lam_offset=ST.LEARNED_LAM_OFFSET)
        rl = BT.fit_until(ss_l, common, max_iters=cap, lam_offset=ST.LEARNED_LAM_OFFSET)
        refit.update({"batched": rb["gpu_ms"], "batched_offset": ro["gpu_ms"],
                      "batched_learned": rl["gpu_ms"] + sum(infer_room[s] for s in common)})
        for a, ms in refit.items():
            cr[a]["seconds"] = round(ms / 1e3, 3)
        for a in ("batched", "batched_offset", "batched_learned"):
            cr[a]["speedup_vs_plain"] = round(refit["plain"] / max(refit[a], 1e-9), 3)
        cr["refit_reached"] = {"batched": sum(d is not None for d in rb["done_at"]),
                               "batched_offset": sum(d is not None for d in ro["done_at"]),
                               "batched_learned": sum(d is not None for d in rl["done_at"])}
    out["common_rooms"] = cr
    return out


def common_rooms(arms):
    """The rooms every arm brings to 2 cm, and per arm how many it reaches and the
    mean iterations to 2 cm on the common rooms (done_at entries are (iteration,
    GPU ms) or None)."""
    names = list(arms)
    n = len(arms[names[0]])
    common = [s for s in range(n) if all(arms[a][s] is not None for a in names)]
    out = {"rooms": len(common), "reached": {a: sum(d is not None for d in arms[a]) for a in names}}
    for a in names:
        if common:
            its = [arms[a][s][0] for s in common]
            out[a] = {"mean_iterations": round(sum(its) / len(its), 1)}
    return common, out


def run_e2e(wl, args, first, world):
    """Same metric through host buffers: every step's ground-truth depth/normal
    maps come from pinned host memory and its loss sums go back to pinned host
    memory, inside the timed region.  The step's CUDA graph copies the next
    step's supervision into the other of two device buffers on a parallel branch
    (overlapping the step) and its loss sums to the host (Fitter.enable_graphs
    with host_stream); the first step's supervision is copied in the timed
    region before the first replay.  The caller restores the state at `first`,
    so the same iterations as the device-resident measurement are timed."""
    import torch
    dev = wl.flat.device
    nb = N_VIEWS // VIEWS_PER_STEP
    n = VIEWS_PER_STEP * wl.hw
    host_d = wl.gt_depth.cpu().pin_memory()
    host_n = wl.gt_normal.cpu().pin_memory()
    bufs = [(torch.empty(n, dtype=torch.float32, device=dev),
             torch.empty((n, 3), dtype=torch.float32, device=dev)) for _ in range(2)]
    K = args.steps
    sums_host = torch.zeros((nb, VIEWS_PER_STEP, 4), dtype=torch.float64).pin_memory()
    for s in range(first, first + K):
        wl.grow_if_needed(s)
    wl.fit.ite = first
    # batch b always reads buffer b % 2 (the batch count is even)
    offsets = [b * n for b in range(nb)]
    wl.fit.enable_graphs(first + K + 8, list(range(nb)), [bufs[b % 2] for b in range(nb)],
                         host_stream={"host_depth": host_d, "host_normal": host_n, "offsets": offsets,
                                      "sums_host": sums_host})
    wl.r.status.zero_()
    main = torch.cuda.current_stream()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ev0.record(main)
    b0 = first % nb
    bufs[b0 % 2][0].copy_(host_d[offsets[b0]:offsets[b0] + n], non_blocking=True)
    bufs[b0 % 2][1].copy_(host_n[offsets[b0]:offsets[b0] + n], non_blocking=True)
    for i in range(K):
        wl.fit.replay((first + i) % nb)
    ev1.record(main)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if int(wl.r.status.item()) & CAPACITY_BIT:
        raise RuntimeError("tile-list capacity overflow inside the e2e region")
    if not bool(torch.isfinite(sums_host).all()):
        raise RuntimeError("non-finite loss sums in the e2e region")
    ms = ev0.elapsed_time(ev1)
    t = RK.max_over_ranks(max(ms / 1e3, wall), dev)
    value = RK.job_throughput(RK.sum_over_ranks(VIEWS_PER_STEP * H * W * K, dev), t) / 1e6
    return {"value": round(value, 3), "unit": UNIT,
            "h2d_bytes_per_step": int(n * 4 + n * 12), "d2h_bytes_per_step": VIEWS_PER_STEP * 4 * 8,
            "ms_per_step": round(t * 1e3 / K, 4),
            "pipeline": "each step's graph copies the next step's supervision from pinned host memory "
                        "(parallel branch, two device buffers) and its loss sums back to pinned memory",
            "l2": "not flushed: every step's supervision arrives from host memory"}


def run_regimes(wl, checkpoints, K, clocks, peaks):
    """Stage times and the roofline at later points of a real fit of the benchmark
    room (Eq. 10 sharpens the weight: the lists shrink and more pairs are opaque).
    The room is fitted from its initial planes with eager steps; at each checkpoint
    K more steps are timed with per-stage CUDA events (L2 flushed between steps)
    and their work counted exactly, then K more are replayed from CUDA graphs
    captured there (the step time a fit sees at that point)."""
    import torch
    wl.reset(0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=wl.flat.device)
    nb = N_VIEWS // VIEWS_PER_STEP
    out = []
    for cp in checkpoints:
        while wl.fit.ite < cp:
            s = wl.fit.ite
            if s % 100 == 0:
                for b in range(nb):
                    wl.grow_if_needed(s + b)
            wl.step(s)
        for b in range(nb):
            wl.grow_if_needed(wl.fit.ite + b)
        wl.r.status.zero_()
        first = wl.fit.ite
        counts = []
        per_step, stages = time_steps(wl, first, K, flush, counts_out=counts)
        if int(wl.r.status.item()) & CAPACITY_BIT:
            raise RuntimeError("tile-list capacity overflow in the regime measurement")
        vs = wl.r.view_sums.cpu().numpy()
        # the next K steps replayed from graphs captured at this point of the fit
        for b in range(nb):
            wl.grow_if_needed(wl.fit.ite + b)
        wl.fit.enable_graphs(wl.fit.ite + K + 8, list(range(nb)), [wl.gt_slice(b) for b in range(nb)])
        wl.r.status.zero_()
        g_ms = statistics.mean(time_replays(wl, wl.fit.ite, K, flush))
        if int(wl.r.status.item()) & CAPACITY_BIT:
            raise RuntimeError("tile-list capacity overflow in the regime measurement")
        out.append({"iteration": first, "lambda": round(wl.B.lambda_schedule(first), 3),
                    "ms_per_step_graph": round(g_ms, 4),
                    "mpixel_views_per_s_graph": round(VIEWS_PER_STEP * H * W / g_ms / 1e3, 1),
                    "ms_per_step_eager": round(statistics.mean(per_step), 4),
                    "stage_ms": {k: round(statistics.mean(v), 4) for k, v in stages.items()},
                    "mean_abs_depth_err_m": round(float(vs[:, 2].sum() / max(vs[:, 3].sum(), 1.0)), 5),
                    "roofline": roofline_entry(counts, stages, K, clocks, src_hash(), peaks, regime=cp)})
    return out


def depth_error_all_views(wl):
    """Mean |D - D*| over the supervised pixels of all views (forward-only render)."""
    from paper_2412_03451_gb300 import splat as SP
    ev = SP.Renderer([H] * N_VIEWS, [W] * N_VIEWS, [0] * N_VIEWS, [0, N_INIT],
                     tile=wl.r.tile, device=wl.flat.device)
    ev.set_cameras(wl.room.cams.w2c, wl.room.cams.intr)
    lam = SP.B.lambda_schedule(wl.fit.ite)
    ev.ensure_capacity(wl.flat, lam)
    ev.forward(wl.flat, lam, alpha=False)
    valid = wl.gt_depth > 0
    return float((ev.depth - wl.gt_depth).abs()[valid].mean().item())


def run_fit(wl, n_iters):
    """The single-scene fit of the benchmark room as a user runs it: n_iters
    optimisation steps from the initial planes (Eq. 10 from iteration 0), each
    replayed from its camera batch's CUDA graph, timed by CUDA events around the
    whole fit (no L2 flush).  Tile-list capacity is sized before the fit with
    headroom; if the status word reports an overflow the fit is run again with
    more room.  Reports the mean depth error over all views after the fit."""
    import torch
    nb = N_VIEWS // VIEWS_PER_STEP
    for headroom in (1.6, 2.5, 4.0):
        wl.reset(0)
        for b in range(nb):
            wl.r.select(b)
            wl.r.ensure_capacity(wl.flat, wl.B.lambda_schedule(0), headroom=headroom)
        wl.fit.enable_graphs(n_iters + 8, list(range(nb)), [wl.gt_slice(b) for b in range(nb)])
        wl.r.status.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0.record()
        for s in range(n_iters):
            wl.fit.replay(s % nb)
        e1.record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if not int(wl.r.status.item()) & CAPACITY_BIT:
            ms = e0.elapsed_time(e1)
            return {"iterations": n_iters, "device_s": round(ms / 1e3, 4), "wall_s": round(wall, 4),
                    "ms_per_step": round(ms / n_iters, 4),
                    "mpixel_views_per_s": round(VIEWS_PER_STEP * H * W * n_iters / ms / 1e3, 1),
                    "capacity_headroom": headroom,
                    "depth_err_m_after": round(depth_error_all_views(wl), 5)}
    raise RuntimeError("tile-list capacity overflow in the single-scene fit")


def run_ttd(wl, max_iters):
    """Wall time of the plain single-scene fit (from the initial planes, lambda
    schedule from 0) until the mean |D - D_gt| over all 64 views is <= 2 cm,
    checked every 8 steps (one pass over the views) with a forward-only render
    of all views; evaluation time is excluded."""
    import torch
    from paper_2412_03451_gb300 import splat as SP
    wl.reset(0)
    ev = SP.Renderer([H] * N_VIEWS, [W] * N_VIEWS, [0] * N_VIEWS, [0, N_INIT],
                     tile=wl.r.tile, device=wl.flat.device)
    ev.set_cameras(wl.room.cams.w2c, wl.room.cams.intr)
    nb = N_VIEWS // VIEWS_PER_STEP
    spent = 0.0
    err = float("nan")
    hist = []
    for it in range(0, max_iters, nb):
        for s in range(it, it + nb):
            wl.grow_if_needed(s)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(it, it + nb):
            wl.step(s)
        torch.cuda.synchronize()
        spent += time.perf_counter() - t0
        if (it // nb) % 4 == 3 or it + nb >= max_iters:
            lam = SP.B.lambda_schedule(wl.fit.ite)
            ev.ensure_capacity(wl.flat, lam)
            ev.forward(wl.flat, lam, alpha=False)
            e = (ev.depth - wl.gt_depth).abs()
            valid = wl.gt_depth > 0
            err = float(e[valid].mean().item())
            hist.append((wl.fit.ite, round(err, 5), round(spent, 3)))
            if err <= 0.02:
                return {"seconds": round(spent, 3), "iterations": wl.fit.ite, "depth_err_m": err,
                        "reached": True, "history": hist}
    return {"seconds": round(spent, 3), "iterations": wl.fit.ite, "depth_err_m": err,
            "reached": False, "history": hist}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm).

def oracle_sample_step(room, planes, views, rows, lam):
    """One forward + loss + backward of the FP64 oracle on `rows` of `views`."""
    import numpy as np
    from oracle import oracle as O
    cams = room.cams.subset(views)
    z32 = float(np.float32(0.01))
    gd, gn, _ = O.raycast(room.gt.center, room.gt.quat, room.gt.radii, cams.w2c, cams.intr, H, W,
                          z_near=z32, rows=rows)
    t0 = time.perf_counter()
    o = O.render(planes.center, planes.quat, planes.radii, cams.w2c, cams.intr, H, W,
                 float(np.float32(lam)), z_near=z32, rows=rows)
    _, dD, dN, _ = O.loss(o["depth"], o["normal"], gd, gn)
    keep = np.zeros(dD.shape, bool)
    keep[:, rows[0]:rows[1]] = True
    dD[~keep] = 0
    dN[~keep] = 0
    O.backward(planes.center, planes.quat, planes.radii, cams.w2c, cams.intr, H, W,
               float(np.float32(lam)), dD, dN, z_near=z32)
    return time.perf_counter() - t0, len(views) * (rows[1] - rows[0]) * W


def cpu_baseline(room, init, ite, target_s=20.0):
    from oracle import oracle as O
    lam = O.lambda_schedule(ite)
    views = list(range(VIEWS_PER_STEP))
    r0 = H // 2
    # two short samples give the per-row time apart from the fixed set-up cost
    t2, _ = oracle_sample_step(room, init, views, (r0, r0 + 2), lam)
    t6, _ = oracle_sample_step(room, init, views, (r0, r0 + 6), lam)
    per_row = max((t6 - t2) / 4.0, 1e-4)
    fixed = max(t2 - 2 * per_row, 0.0)
    rows = max(2, min(H, int((target_s - fixed) / per_row)))
    r0 = max(0, H // 2 - rows // 2)
    t, npx = oracle_sample_step(room, init, views, (r0, r0 + rows), lam)
    return {"value": round(npx / t / 1e6, 6), "unit": UNIT, "cores": O.num_threads(),
            "kind": "oracle",
            "sample": "rows %d-%d of the first %d views (%d pixel-views), forward + loss + backward "
                      "of the FP64 brute-force oracle over all %d planes; %.1f s" %
                      (r0, r0 + rows, len(views), npx, N_INIT, t)}


def tiny_room_timing(device, n_steps=50):
    """The 64-plane room (8 views of 128x96) fitted for n_steps Adam steps, every
    view in every step: on the GPU (eager steps, CUDA events, tile-list capacity
    sized once at the first step's lambda, whose widening is the largest) and by
    the FP64 oracle on the host cores (forward, loss, backward and Adam per step);
    the oracle's step is also timed on one core."""
    import numpy as np
    import torch
    from oracle import oracle as O
    from paper_2412_03451_gb300 import binding as B
    from paper_2412_03451_gb300 import scenes as S
    from paper_2412_03451_gb300 import splat as SP
    room = S.tiny_room(0)
    init = S.perturb_planes(room.gt, 1)
    cams = room.cams
    V, Ht, Wt, K = cams.V, cams.H, cams.W, init.K
    z32 = float(np.float32(0.01))
    D, N, _ = O.raycast(room.gt.center, room.gt.quat, room.gt.radii, cams.w2c, cams.intr, Ht, Wt,
                        z_near=z32)
    r = SP.Renderer([Ht] * V, [Wt] * V, [0] * V, [0, K], device=device)
    r.set_cameras(cams.w2c, cams.intr)
    gd = torch.from_numpy(D.astype(np.float32).reshape(-1)).to(device)
    gn = torch.from_numpy(N.astype(np.float32).reshape(-1, 3)).to(device)
    r.ensure_capacity(SP.planes_to_flat(init.center, init.quat, init.radii, device),
                      B.lambda_schedule(0), headroom=2.0)

    def gpu_fit():
        fit = SP.Fitter(r, SP.planes_to_flat(init.center, init.quat, init.radii, device))
        for it in range(n_steps):
            fit.step(gd, gn, lam=B.lambda_schedule(it))
        return fit

    gpu_fit()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r.status.zero_()
    e0.record()
    gpu_fit()
    e1.record()
    torch.cuda.synchronize()
    gpu_s = e0.elapsed_time(e1) / 1e3
    ok = int(r.status.item()) == 0

    def oracle_steps(n):
        p = np.concatenate([init.center.ravel(), init.quat.ravel(), init.radii.ravel()]).astype(np.float64)
        m, v = np.zeros_like(p), np.zeros_like(p)
        t0 = time.perf_counter()
        for it in range(n):
            lam = float(np.float32(O.lambda_schedule(it)))
            c, q, rr = p[:3 * K].reshape(K, 3), p[3 * K:7 * K].reshape(K, 4), p[7 * K:].reshape(K, 4)
            o = O.render(c, q, rr, cams.w2c, cams.intr, Ht, Wt, lam, z_near=z32)
            _, dD, dN, _ = O.loss(o["depth"], o["normal"], D, N)
            gc, gq, gr = O.backward(c, q, rr, cams.w2c, cams.intr, Ht, Wt, lam, dD, dN, z_near=z32)
            g = np.concatenate([gc.ravel(), gq.ravel(), gr.ravel()])
            a = O.adam(p[:7 * K], g[:7 * K], m[:7 * K], v[:7 * K], it + 1)
            b = O.adam(p[7 * K:], g[7 * K:], m[7 * K:], v[7 * K:], it + 1, clamp_min=1e-3)
            p, m, v = (np.concatenate([a[i], b[i]]) for i in range(3))
        return time.perf_counter() - t0

    cores = O.num_threads()
    oracle_s = oracle_steps(n_steps)
    O.set_num_threads(1)
    try:
        one_core = oracle_steps(2) / 2
    finally:
        O.set_num_threads(cores)
    return {"workload": "64 planes, 8 views of 128x96, %d Adam steps over all views" % n_steps,
            "gpu_s": round(gpu_s, 4), "gpu_launch": "eager steps", "gpu_status_ok": ok,
            "oracle_s": round(oracle_s, 3), "oracle_cores": cores,
            "oracle_single_core_s_per_step": round(one_core, 4),
            "gpu_vs_oracle": round(oracle_s / gpu_s, 1)}


def run_reference(args):
    """The oracle as it stands, on the same workload and metric: each step
    renders, scores and back-propagates a bounded sample of the step's views."""
    import numpy as np
    from oracle import oracle as O
    from paper_2412_03451_gb300 import scenes as S
    room = S.large_room(1000, n_rect=N_GT, n_views=N_VIEWS, H=H, W=W, f=F)
    init = S.surface_init(room, N_INIT, 2000)
    lam = O.lambda_schedule(args.start_ite)
    total_steps = args.steps + args.warmup
    # size the sample so the whole run takes about two minutes
    t, npx = oracle_sample_step(room, init, list(range(VIEWS_PER_STEP)), (H // 2, H // 2 + 1), lam)
    per_row = t
    rows = int(max(1, min(H, 120.0 / max(total_steps, 1) / max(per_row, 1e-3))))
    times, pix = [], 0
    for s in range(total_steps):
        b = (s % (N_VIEWS // VIEWS_PER_STEP)) * VIEWS_PER_STEP
        r0 = (37 * s) % (H - rows + 1)
        t, npx = oracle_sample_step(room, init, list(range(b, b + VIEWS_PER_STEP)), (r0, r0 + rows),
                                    lam)
        if s >= args.warmup:
            times.append(t)
            pix += npx
    value = pix / sum(times) / 1e6
    sample = ("per step: %d rows x %d px of the step's %d views (%d pixel-views of %d), forward + "
              "loss + backward of the FP64 brute-force oracle over all %d planes" %
              (rows, W, VIEWS_PER_STEP, rows * W * VIEWS_PER_STEP, VIEWS_PER_STEP * H * W, N_INIT))
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * statistics.mean(times), 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(args, 1), l2="host CPU run (no GPU cache to flush)"),
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": O.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def profile_case(args):
    """One eager optimisation step of the workload inside cudaProfilerStart/Stop
    (for `ncu --profile-from-start off`), after 3 warm-up steps, or, with
    --profile-ite N, after a real fit of N iterations (eager steps, outside the
    profiled range)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    tile = (16, 16) if args.tile == "auto" else tuple(int(x) for x in args.tile.split("x"))
    wl = Workload(0, tile, "cuda:0", args.warps)
    wl.reset(args.start_ite)
    last = max(3, args.profile_ite)
    nb = N_VIEWS // VIEWS_PER_STEP
    for i in range(last):
        if i < 3 or i % 100 == 0:
            for b in range(nb):
                wl.grow_if_needed(i + b)
        wl.step(i)
    wl.grow_if_needed(last)
    wl.r.status.zero_()
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    wl.step(last)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    status = int(wl.r.status.item())
    print(json.dumps({"profile_case": "step %d" % last, "lambda": wl.B.lambda_schedule(last),
                      "tile": "%dx%d" % tile, "status": status}))
    return 0 if status == 0 else 1


def run_stress(args):
    """The differentiation-stress configuration: one room with 10,000 planes and 256
    views of 640x480 (78.6 M pixel-views) in one fused forward + loss + backward launch
    per step, supervision from a hard-mode render of the ground-truth rectangles.
    Times K fused steps (project, bin, fused kernel, by CUDA events, L2 flushed) at the
    first lambda and at lambda 20, for 8x8 and 16x16 tiles."""
    import statistics
    import torch
    import __graft_entry__
    from paper_2412_03451_gb300 import binding as B
    from paper_2412_03451_gb300 import scenes as S
    from paper_2412_03451_gb300 import splat as SP
    __graft_entry__.build()
    dev = "cuda:0"
    room = S.large_room(1300, n_rect=2000, n_views=256)
    init = S.surface_init(room, 10000, seed=1301)
    cams = room.cams
    V = cams.V
    gtr = SP.Renderer([H] * V, [W] * V, [0] * V, [0, room.gt.center.shape[0]], tile=(16, 16),
                      device=dev, flags=B.PS_HARD)
    gtr.set_cameras(cams.w2c, cams.intr)
    gflat = SP.planes_to_flat(room.gt.center, room.gt.quat, room.gt.radii, dev)
    gtr.ensure_capacity(gflat, 300.0)
    gtr.forward(gflat, 300.0)
    gd, gn = gtr.depth.clone(), gtr.normal.clone()
    del gtr
    flat = SP.planes_to_flat(init.center, init.quat, init.radii, dev)
    g = torch.zeros_like(flat)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    out = []
    for tile in ((8, 8), (16, 16)):
        r = SP.Renderer([H] * V, [W] * V, [0] * V, [0, init.K], tile=tile, device=dev)
        r.set_cameras(cams.w2c, cams.intr)
        for lam in (B.lambda_schedule(0), 20.0):
            r.ensure_capacity(flat, lam)
            r.status.zero_()
            ts = []
            for i in range(args.steps + 1):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                r.project_bin(flat, lam)
                r.fused(flat, g, gd, gn)
                e1.record()
                torch.cuda.synchronize()
                if i > 0:
                    ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            out.append({"tile": "%dx%d" % tile, "lambda": round(lam, 3), "ms_per_step": round(ms, 3),
                        "mpixel_views_per_s": round(V * H * W / ms / 1e3, 1),
                        "tile_entries": int(r.required), "status": int(r.status.item())})
        del r
        torch.cuda.empty_cache()
    print(json.dumps({"stress": "10,000 planes, 256 views of %dx%d, fused forward + loss + backward" % (W, H),
                      "runs": out}), flush=True)
    return 0 if all(o["status"] == 0 for o in out) else 1


def profile_gemm(args):
    """The seed network's inner-layer GEMM (im2col rows of 64 patches' 32x32
    outputs, 64 channels, K = 9 x 64): bf16 operands, FP32 output; 50 timed
    launches (CUDA events), then one inside cudaProfilerStart/Stop."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2412_03451_gb300 import binding as B
    M, N, K = 65536, 64, 576
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn(M, K, device="cuda", generator=g).bfloat16()
    Bm = torch.randn(N, K, device="cuda", generator=g).bfloat16()
    C = torch.empty(M, N, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(3):
        B.ps_gemm_bf16(A, Bm, None, C, None, err=err)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(50):
        B.ps_gemm_bf16(A, Bm, None, C, None, err=err)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 50
    torch.cuda.cudart().cudaProfilerStart()
    B.ps_gemm_bf16(A, Bm, None, C, None, err=err)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    ok = bool(torch.allclose(C, A.float() @ Bm.float().T, rtol=1e-4, atol=1e-3 * K ** 0.5))
    nbytes = (M * K + N * K) * 2 + M * N * 4
    print(json.dumps({"profile_gemm": "%dx%dx%d" % (M, N, K), "us": round(ms * 1e3, 2),
                      "TFLOP/s": round(2 * M * N * K / ms / 1e9, 1), "GB/s": round(nbytes / ms / 1e6, 0),
                      "matches_fp32_matmul": ok, "error_word": int(err.item())}))
    return 0 if ok and int(err.item()) == 0 else 1


def main():
    args = parse()
    if args.profile_case:
        return profile_case(args)
    if args.profile_gemm:
        return profile_gemm(args)
    if args.stress:
        return run_stress(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args)), flush=True)
        return 0
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
