#!/usr/bin/env python
"""Benchmark of the TileGS forward path on GB300.

A step is one whole frame of the hot path -- projection, tile intersection,
ordering (binned: depth range, bin count/scan/scatter, repair; baseline: global
radix sort) and rasterisation -- of the 1M-Gaussian mixture scene at
1920x1080 (fx = fy = 1100), inputs resident in HBM.  The headline `value` is
the binned (EXACT) path's frame throughput in Mpix/s; the plain global-sort
path is timed beside it on the same GPU, with per-stage and raster-kernel
times for both.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Timing: W untimed warm-up frames, then K frames, each preceded by an L2 flush
(a 256 MiB write outside the timed events) and bracketed by CUDA events on
the stream the library launches on; barrier + synchronize around the loop,
max over ranks.  Multi-GPU: independent replicas, one frame per rank per step
(no data-path collective; the method does not shard a frame).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "raster ms/frame & Mpix/s at 1080p: binned vs global-sort, same GB300, err≤1e-5"
WORKLOAD = "mid"
WORKLOAD_DESC = ("1M Gaussians (90% 64-component anisotropic mixture + 10% background shell, "
                 "log-scales N(-5,1), SH degree 3 N(0,0.3), opacity sigmoid(N(0,1.5)), seed 1); "
                 "camera (0,0,3) -> origin, 1920x1080, fx=fy=1100")
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 300; the reference arm, whose steps are CPU frames: 10)")
    ap.add_argument("--warmup", type=int, default=None, help="warm-up steps (default 10; reference arm: 3)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-train", action="store_true", help="skip the forward+backward training-step leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the 16-view batched-render leg")
    ap.add_argument("--no-spatial", action="store_true", help="skip the raster-order-aware storage leg")
    ap.add_argument("--no-heavy", action="store_true", help="skip the 3M / 6M-Gaussian depth-complexity leg")
    ap.add_argument("--profile-frame", action="store_true",
                    help="for ncu: two warm-up frames, then one frame of each path, no timing")
    ap.add_argument("--modes", default="exact,global", help="paths run by --profile-frame")
    ap.add_argument("--backward", action="store_true", help="--profile-frame: also one saved frame + backward")
    ap.add_argument("--spatial", action="store_true",
                    help="--profile-frame: render the scene in raster-order-aware (Morton) storage")
    ap.add_argument("--workload", default="mid", choices=["mid", "heavy3m", "heavy6m_4k"],
                    help="--profile-frame: the workload rendered")
    a = ap.parse_args()
    if a.steps is None:
        a.steps = 10 if a.impl == "reference" else 300
    if a.warmup is None:
        a.warmup = 3 if a.impl == "reference" else 10
    return a


# --------------------------------------------------------------------- dist
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(backend):
    import torch.distributed as dist
    ws, rank, _ = dist_env()
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if ws > 1 else None


def max_over_ranks(x: float, dist, device=None) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(ws: int, units_per_rank: float, local_ms: float, dist, device=None) -> tuple:
    """Whole-job throughput of N independent replicas: the slowest rank's time
    (max over ranks) bounds the step; every rank processed units_per_rank.
    Returns (units per second, max ms)."""
    ms = max_over_ranks(local_ms, dist, device)
    return ws * units_per_rank / (ms * 1e-3), ms


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


# --------------------------------------------------------------------- oracle timing (cpu_baseline / reference arm)
def bench_config(ws: int) -> dict:
    """The workload both arms report (identical dicts, so the two JSON lines
    name the same configuration)."""
    return {"workload": WORKLOAD_DESC, "gaussians": 1000000, "resolution": "1920x1080", "tile": 16,
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
            "l2": "GPU steps: flushed between timed steps (256 MiB write outside the timed events)"}


def oracle_frame(scene, cam, threads: int) -> dict:
    """One whole frame of the CPU oracle, measured, nothing extrapolated:
    projection, emission and the per-tile (depth, gid) sort (single-threaded
    code in the oracle), then the compositing of every tile on `threads`
    OpenMP threads.  Wall-clock seconds of each part."""
    import oracle as O
    O.set_threads(threads)
    t0 = time.perf_counter()
    proj = O.project(scene, cam)
    ent = O.emit(proj, cam.width, cam.height)
    tx, ty = O.tiles_xy(cam.width, cam.height)
    off, stream = O.sort_tiles(ent, tx * ty)
    t1 = time.perf_counter()
    O.composite(proj, off, stream, cam.width, cam.height)
    t2 = time.perf_counter()
    return dict(frame_s=t2 - t0, setup_s=t1 - t0, composite_s=t2 - t1, threads=threads,
                entries=int(ent[0].shape[0]))


def host_cores() -> int:
    return len(os.sched_getaffinity(0))


def cpu_baseline_block(scene, cam):
    """The oracle on the full 1080p frame, once on all host cores and once on
    one thread (the compositing is the part the oracle runs in parallel)."""
    P = cam.width * cam.height
    ncores = host_cores()
    allc = oracle_frame(scene, cam, ncores)
    one = oracle_frame(scene, cam, 1)
    return {"value": round(P / allc["frame_s"] / 1e6, 6), "unit": "Mpix/s", "cores": ncores, "kind": "oracle",
            "sample": (f"one full frame ({allc['entries']} entries, all {cam.width}x{cam.height} pixels), "
                       f"measured, not extrapolated: projection + emission + per-tile sort single-threaded "
                       f"(the oracle's code), compositing on {ncores} threads; the same frame is also timed "
                       f"on 1 thread"),
            "frame_s_allcores": round(allc["frame_s"], 3),
            "frame_s_1thread": round(one["frame_s"], 3),
            "setup_s": round(allc["setup_s"], 3),
            "composite_s_allcores": round(allc["composite_s"], 3),
            "composite_s_1thread": round(one["composite_s"], 3),
            "value_1thread": round(P / one["frame_s"] / 1e6, 6)}


def run_reference(args):
    """The oracle as the reference arm (rank 0 only): every step, warm-up
    included, is one whole frame of the oracle on all host cores, and its
    wall-clock time is the step time."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2609_03613_gb300 import scenes
    scene, cam = scenes.workload(WORKLOAD)
    P = cam.width * cam.height
    ncores = host_cores()
    times = []
    for i in range(args.warmup + args.steps):
        f = oracle_frame(scene, cam, ncores)
        if i >= args.warmup:
            times.append(f["frame_s"])
    frame_s = sum(times) / len(times)
    value = P / frame_s / 1e6
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Mpix/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(frame_s * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic", "config": bench_config(ws),
           "path": "CPU oracle (plain C, float32 in the definition's operation order)",
           "step_s": [round(t, 3) for t in times],
           "cpu_baseline": {"value": round(value, 6), "unit": "Mpix/s", "cores": ncores, "kind": "oracle",
                            "sample": ("each step one whole frame, measured: projection + emission + per-tile "
                                       f"sort single-threaded, compositing of every tile on {ncores} threads")},
           "e2e": {"value": round(value, 6), "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------- ours
def kernel_hash() -> str:
    """Hash of the source the binned raster kernel compiles from: its files and
    the device part of internal.cuh (the host-side context struct after the
    context marker does not change the kernel)."""
    h = hashlib.sha256()
    for f in ("raster.cu", "raster_common.cuh", "internal.cuh", "device.cuh"):
        b = open(os.path.join(ROOT, "paper_2609_03613_gb300", "csrc", f), "rb").read()
        if f == "internal.cuh":
            b = b.split(b"// ------------------------------------------------------------------ context")[0]
        h.update(b)
    return h.hexdigest()[:16]


def load_traffic():
    """ncu DRAM traffic of the binned raster kernel for this workload, if the
    profile was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "raster_binned_mid.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None, None
    if d.get("kernel_hash") != kernel_hash():
        return None, d
    return d.get("dram_bytes_per_launch"), d


def run_ours(args):
    import numpy as np
    import torch

    from paper_2609_03613_gb300 import scenes, tilegs as G

    ws, rank, local = dist_env()
    dist = dist_init("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scene, cam = scenes.workload(WORKLOAD)
    P = cam.width * cam.height
    ds = G.DeviceScene.from_numpy(scene, dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    bg = (0.0, 0.0, 0.0)
    H, W = cam.height, cam.width

    side = torch.cuda.Stream(device=dev)  # graphs cannot be captured on the legacy stream

    def make(mode, sc_dev=ds, **kw):
        ctx = G.Context(mode, **kw)
        out = (torch.empty((H, W, 3), device=dev), torch.empty((H, W), device=dev),
               torch.empty((H, W), dtype=torch.int32, device=dev))
        with torch.cuda.stream(side):
            ctx.render(sc_dev, cam, bg, out)  # sizes the scratch (one read of M)
        torch.cuda.synchronize()
        m = ctx.last_entry_count()
        ctx.reserve(sc_dev.n, int(m * 1.25) + 1024, W, H)
        return ctx, out, m

    def timed(ctx, out, steps, warmup, flags=G.RENDER_NO_SYNC | G.RENDER_GRAPH, sc_dev=ds, stages=None):
        # stage events only outside graphs (their records inside a captured
        # graph do not time the stages)
        staged = not (flags & G.RENDER_GRAPH) if stages is None else stages
        ctx.enable_timing(staged)
        with torch.cuda.stream(side):
            for _ in range(warmup):
                ctx.render(sc_dev, cam, bg, out, flags=flags)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        stage = {s: [] for s in G.STAGES}
        l0 = ctx.launch_count()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        with torch.cuda.stream(side):
            for i in range(steps):
                flush.zero_()
                ev[i][0].record()
                ctx.render(sc_dev, cam, bg, out, flags=flags)
                ev[i][1].record()
                if staged:
                    st = ctx.stage_times()  # events on the library's stream; synchronises
                    for s in G.STAGES:
                        stage[s].append(st[s])
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        wall = time.perf_counter() - w0
        ms = [a.elapsed_time(b) for a, b in ev]
        launches = ctx.launch_count() - l0
        return ms, stage, wall, launches

    ctx_b, out_b, m_b = make("exact")
    ctx_g, out_g, m_g = make("global")
    assert ctx_b.error() == 0 and ctx_g.error() == 0

    with ClockSampler(local) as clk:
        ms_b, _, wall_b, launches = timed(ctx_b, out_b, args.steps, args.warmup)
        ms_g, _, wall_g, _ = timed(ctx_g, out_g, args.steps, args.warmup)
        # the same frames issued launch by launch (no graph), with per-stage
        # events on the library's stream: the stage and raster-kernel times
        ms_b_ng, st_b, _, _ = timed(ctx_b, out_b, max(50, args.steps // 2), 3, flags=G.RENDER_NO_SYNC)
        ms_g_ng, st_g, _, _ = timed(ctx_g, out_g, max(50, args.steps // 2), 3, flags=G.RENDER_NO_SYNC)
    clocks = clk.summary()

    # launch overlap: the frame's kernels with programmatic dependent launch
    # (the default) against ordinary launches, graph-replayed and issued
    # launch by launch without stage events
    n_l = max(50, args.steps // 2)
    ms_u, _, _, _ = timed(ctx_b, out_b, n_l, 3, flags=G.RENDER_NO_SYNC, stages=False)
    ctx_o, out_o, _ = make("exact", pdl=0)
    ms_og, _, _, _ = timed(ctx_o, out_o, n_l, 3)
    ms_ou, _, _, _ = timed(ctx_o, out_o, n_l, 3, flags=G.RENDER_NO_SYNC, stages=False)
    del ctx_o, out_o
    launch_overlap = {"frame_graph_ms": round(sum(ms_b) / len(ms_b), 4),
                      "frame_uncaptured_ms": round(sum(ms_u) / len(ms_u), 4),
                      "ordinary_launches": {"frame_graph_ms": round(sum(ms_og) / len(ms_og), 4),
                                            "frame_uncaptured_ms": round(sum(ms_ou) / len(ms_ou), 4)},
                      "note": "EXACT frame, CUDA events, L2 flushed; un-captured frames without stage events"}

    value_pix_s, frame_b = replica_throughput(ws, P, sum(ms_b) / len(ms_b), dist, dev)
    value_g_pix_s, frame_g = replica_throughput(ws, P, sum(ms_g) / len(ms_g), dist, dev)
    mean = lambda v: sum(v) / len(v)
    raster_b = mean(st_b["raster"])
    raster_g = mean(st_g["raster"])

    # images of both paths must agree (EXACT reproduces the global order)
    with torch.cuda.stream(side):
        ctx_b.render(ds, cam, bg, out_b)
        ctx_g.render(ds, cam, bg, out_g)
    torch.cuda.synchronize()
    err_vs_global = float((out_b[0] - out_g[0]).abs().max().item())
    last_equal = bool(torch.equal(out_b[2], out_g[2]))

    # library comparator for the baseline's sort: torch's stable sort of the
    # same M 64-bit (tile << 32 | depth bits) keys, L2 flushed, CUDA events
    sort_lib_ms = None
    try:
        gen = torch.Generator(device=dev)
        gen.manual_seed(0)
        keys = torch.randint(0, 1 << 62, (m_g,), dtype=torch.int64, device=dev, generator=gen)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
        with torch.cuda.stream(side):
            for _ in range(2):
                torch.sort(keys, stable=True)
            for i in range(10):
                flush.zero_()
                ev[i][0].record()
                torch.sort(keys, stable=True)
                ev[i][1].record()
        torch.cuda.synchronize()
        sort_lib_ms = statistics.median(a.elapsed_time(b) for a, b in ev)
        del keys
    except Exception as e:  # pragma: no cover
        print(f"library sort comparator failed: {e}", file=sys.stderr)

    # the paper's approximate policy, for the repair ablation
    ctx_p = G.Context("paper")
    out_p = (torch.empty((H, W, 3), device=dev), torch.empty((H, W), device=dev),
             torch.empty((H, W), dtype=torch.int32, device=dev))
    with torch.cuda.stream(side):
        ctx_p.render(ds, cam, bg, out_p)
    ms_p, st_p, _, _ = timed(ctx_p, out_p, max(3, args.steps // 4), 2, flags=G.RENDER_NO_SYNC)
    with torch.cuda.stream(side):
        ctx_p.render(ds, cam, bg, out_p)
    torch.cuda.synchronize()
    err_paper = float((out_p[0] - out_b[0]).abs().max().item())

    # roofline of the dominant kernel (binned raster): float32 ops of the
    # compositing definition it executed, counted by its instrumented twin
    ops = None
    try:
        proj = ctx_b.project(ds, cam)
        isect, m_cap, m_dev, m = ctx_b.tile_intersect(proj, ds.n, cam)
        words, offsets, _ = ctx_b.sort_or_bin(proj, ds.scales, ds.n, cam, isect, m_cap, m_dev)
        _, _, _, nt = ctx_b.rasterize_fwd(proj, ds.n, cam, words, offsets, count_tests=True)
        ops = ctx_b.last_raster_ops()
        tests = int(nt.sum().item())
        del proj, isect, words, offsets, nt
    except Exception as e:  # pragma: no cover
        tests = None
        print(f"op count failed: {e}", file=sys.stderr)
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    # FP32 roofline of the dominant kernel as the measurement plan defines it:
    # 20 FP32 flops per Gaussian test (the exp counted as its FP32 work),
    # against SMs x 128 FMA lanes x 2 flops x the sampled SM clock
    flops_per_test = 20
    peak_flops = n_sm * 128 * 2 * sm_mhz * 1e6
    flops = flops_per_test * tests if tests else None
    achieved = flops / (raster_b * 1e-3) if flops else None
    traffic, prof = load_traffic()
    roofline = {"kernel": "k_raster<16,binned>", "bound": "alu",
                "achieved": round(achieved / 1e12, 4) if achieved else None,
                "peak": round(peak_flops / 1e12, 4), "unit": "TFLOP/s",
                "frac": round(achieved / peak_flops, 4) if achieved else None,
                "traffic": traffic,
                "peak_source": (f"{n_sm} SMs x 128 FP32 FMA lanes x 2 flops x {sm_mhz:.0f} MHz (median SM clock "
                                "sampled during the timed region)"),
                "flops_per_test": flops_per_test, "tests_per_launch": tests,
                "achieved_source": "20 flops x Gaussian tests counted by the raster's instrumented twin, over the "
                                   "raster's CUDA-event time in un-captured frames"}
    # the same kernel against the FP32 lanes' instruction rate, with the
    # compositing definition's own operation count (8 per visit, +17 with
    # exp, +3 when alpha passes, +4 when applied), and against the warp
    # schedulers' issue rate (warp instructions per launch from the ncu
    # capture, only while the source is unchanged)
    if ops:
        lane_peak = n_sm * 128 * sm_mhz * 1e6
        roofline["lane_issue"] = {"achieved": round(ops / (raster_b * 1e-3) / 1e12, 4),
                                  "peak": round(lane_peak / 1e12, 4), "unit": "T FP32 inst/s",
                                  "frac": round(ops / (raster_b * 1e-3) / lane_peak, 4), "ops_per_launch": ops}
    winst = prof.get("warp_inst_per_launch") if (prof and traffic is not None) else None
    if winst:
        issue_peak = n_sm * 4 * sm_mhz * 1e6
        issue = winst / (raster_b * 1e-3)
        roofline["issue"] = {"achieved": round(issue / 1e9, 2), "peak": round(issue_peak / 1e9, 2),
                             "unit": "G warp-inst/s", "frac": round(issue / issue_peak, 4),
                             "warp_inst_per_launch": winst}

    # what each part of the binned frame buys, stage by stage, on this frame:
    # the same images from (1) the plain global-sort frame, (2) the global
    # stream rastered by the binned kernel (tile cull at staging, colour
    # staging, per-warp masks, early-out), (3) only the culled entries, one
    # bin per tile, sorted before the raster (their global order), (4) one
    # bin per tile with the repair in the raster, and (5) the EXACT frame
    ablation = {"global_plain": {"frame_ms": round(frame_g, 4), "raster_ms": round(raster_g, 4),
                                 "stages_ms": {k: round(mean(v), 4) for k, v in st_g.items() if mean(v) > 0},
                                 "entries_sorted": m_g}}
    for label, mode, kw in (("global_binned_raster", "global", {"tile_cull": 1}),
                            ("culled_global_order", "exact", {"K": 1, "repair_in_raster": 0}),
                            ("culled_one_bin_lazy", "exact", {"K": 1})):
        ctx_a, out_a, m_a = make(mode, **kw)
        ms_a, _, _, _ = timed(ctx_a, out_a, args.steps, args.warmup)
        _, st_a, _, _ = timed(ctx_a, out_a, max(20, args.steps // 4), 3, flags=G.RENDER_NO_SYNC)
        with torch.cuda.stream(side):
            ctx_a.render(ds, cam, bg, out_a)
        torch.cuda.synchronize()
        ablation[label] = {"frame_ms": round(mean(ms_a), 4), "raster_ms": round(mean(st_a["raster"]), 4),
                           "stages_ms": {k: round(mean(v), 4) for k, v in st_a.items() if mean(v) > 0},
                           "entries": m_a,
                           "image_equal_exact": bool(torch.equal(out_a[0], out_b[0])
                                                     and torch.equal(out_a[2], out_b[2]))}
        ctx_a.close()
        del out_a
    ablation["binned_exact"] = {"frame_ms": round(frame_b, 4), "raster_ms": round(raster_b, 4),
                                "stages_ms": {k: round(mean(v), 4) for k, v in st_b.items() if mean(v) > 0},
                                "entries": m_b}

    # end to end through the C-ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()
        hs = G.DeviceScene(pin(scene.means), pin(scene.scales), pin(scene.quats), pin(scene.opacities),
                           pin(scene.sh), scene.sh_degree)
        hout = (torch.empty((H, W, 3)).pin_memory(), torch.empty((H, W)).pin_memory(),
                torch.empty((H, W), dtype=torch.int32).pin_memory())
        ctx_e = G.Context("exact")
        flags = G.RENDER_HOST_INPUTS | G.RENDER_HOST_OUTPUTS
        for _ in range(args.warmup):
            ctx_e.render(hs, cam, bg, hout, flags=flags)

        def e2e_run(step_flags):
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                # the warm-up sized the entry buffers: no mid-frame entry-count
                # read-back (a capacity overflow raises GS_ERR_CAPACITY)
                ctx_e.render(hs, cam, bg, hout, flags=step_flags)
            ctx_e.render_wait()  # every step's outputs are in host memory
            torch.cuda.synchronize()
            if dist is not None:
                dist.barrier()
            return max_over_ranks((time.perf_counter() - t0) / args.steps, dist, dev)

        # pipelined calls (each still uploads its scene and downloads its
        # image; the upload of one overlaps the frame and download of the
        # one before), then calls that each return after their outputs landed
        e2e_s = e2e_run(flags | G.RENDER_PIPELINE)
        e2e_sync_s = e2e_run(flags | G.RENDER_NO_SYNC)
        assert ctx_e.error() == 0
        h2d = sum(int(t.numel()) * 4 for t in (hs.means, hs.scales, hs.quats, hs.opacities, hs.sh))
        d2h = sum(int(t.numel()) * 4 for t in hout)
        e2e = {"value": round(ws * P / e2e_s / 1e6, 4), "unit": "Mpix/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_s * 1e3, 3),
               "call": "gs_render, host scene in and host image out every step, GS_RENDER_PIPELINE",
               "one_call_at_a_time": {"value": round(ws * P / e2e_sync_s / 1e6, 4),
                                      "ms_per_step": round(e2e_sync_s * 1e3, 3)}}

    # training step on the same workload: the frame (graph replay, saving the
    # backward's state), the L1 loss gradient against a fixed U[0,1] target,
    # and the raster backward
    train = None
    if not args.no_train:
        target = torch.from_numpy(scenes.random_target(H, W, 5)).to(dev)
        grad = torch.empty(int(G.lib().gs_grad2d_bytes(ds.n)), dtype=torch.uint8, device=dev)
        dl = torch.empty((H, W, 3), device=dev)
        flags_t = G.RENDER_NO_SYNC | G.RENDER_GRAPH | G.RENDER_SAVE
        ctx_b.enable_timing(False)

        def train_step(ev=None):
            ctx_b.render(ds, cam, bg, out_b, flags=flags_t)
            torch.sub(out_b[0], target, out=dl)
            dl.sign_().mul_(1.0 / dl.numel())
            if ev is not None:
                ev[0].record()
            ctx_b.render_bwd(dl, None, grad=grad)
            if ev is not None:
                ev[1].record()

        n_t = max(20, args.steps // 3)
        with torch.cuda.stream(side):
            for _ in range(args.warmup):
                train_step()
        torch.cuda.synchronize()
        ev_s = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_t)]
        ev_b = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_t)]
        l0 = ctx_b.launch_count()
        with ClockSampler(local) as clk_t:
            with torch.cuda.stream(side):
                for i in range(n_t):
                    flush.zero_()
                    ev_s[i][0].record()
                    train_step(ev_b[i])
                    ev_s[i][1].record()
            torch.cuda.synchronize()
        assert ctx_b.error() == 0
        step_ms = max_over_ranks(mean([a.elapsed_time(b) for a, b in ev_s]), dist, dev)
        bwd_ms = mean([a.elapsed_time(b) for a, b in ev_b])
        train = {"ms_per_step": round(step_ms, 4), "mpix_s": round(ws * P / (step_ms * 1e-3) / 1e6, 3),
                 "raster_bwd_ms": round(bwd_ms, 4), "steps": n_t,
                 "launches_per_step": (ctx_b.launch_count() - l0) / n_t,
                 "step": "frame (CUDA graph, RENDER_SAVE) + L1 loss gradient vs a U[0,1] target + gs_render_bwd",
                 "clocks": clk_t.summary()}

    # the learned bin planner on the same frame: per-tile chunk plan against
    # the fixed chunk size (images compared bit for bit)
    planner = None
    wpath = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2609_03613_gb300",
                         "planner_weights.npy")
    if os.path.exists(wpath):
        ctx_pl = G.Context("exact", planner=1)
        ctx_pl.set_planner_weights(torch.from_numpy(np.load(wpath).astype(np.float32)))
        out_pl = (torch.empty((H, W, 3), device=dev), torch.empty((H, W), device=dev),
                  torch.empty((H, W), dtype=torch.int32, device=dev))
        with torch.cuda.stream(side):
            ctx_pl.render(ds, cam, bg, out_pl)
        torch.cuda.synchronize()
        ctx_pl.reserve(ds.n, int(ctx_pl.last_entry_count() * 1.25) + 1024, W, H)
        ms_pl, _, _, _ = timed(ctx_pl, out_pl, args.steps, args.warmup)
        _, st_pl, _, _ = timed(ctx_pl, out_pl, max(50, args.steps // 2), 3, flags=G.RENDER_NO_SYNC)
        with torch.cuda.stream(side):
            ctx_pl.render(ds, cam, bg, out_pl)
        torch.cuda.synchronize()
        planner = {"frame_ms": round(mean(ms_pl), 4), "frame_ms_fixed": round(frame_b, 4),
                   "frame_gain": round(1.0 - mean(ms_pl) / frame_b, 4),
                   "stages_ms": {k: round(mean(v), 4) for k, v in st_pl.items() if mean(v) > 0},
                   "stages_ms_fixed": {k: round(mean(v), 4) for k, v in st_b.items() if mean(v) > 0},
                   "tiles_to_second_pass": ctx_pl.flagged_tiles(),
                   "quantile": float(ctx_pl.cfg.planner_quantile),
                   "image_equal_fixed": bool(torch.equal(out_pl[0], out_b[0]) and torch.equal(out_pl[2], out_b[2]))}

    # raster-order-aware storage: the same scene with its Gaussians in the
    # Morton order of their means (a per-scene step, timed once, outside the
    # frames); the frame on it against the frame on the scene as generated
    spatial = None
    if not args.no_spatial:
        ctx_o = G.Context("exact")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(side):
            ctx_o.reorder_scene(ds)  # sizes the scratch
            e0.record()
            rs, _ = ctx_o.reorder_scene(ds)
            e1.record()
        torch.cuda.synchronize()
        reorder_ms = e0.elapsed_time(e1)
        ctx_s, out_s, m_s = make("exact", rs)
        ms_s, _, _, _ = timed(ctx_s, out_s, args.steps, args.warmup, sc_dev=rs)
        _, st_s, _, _ = timed(ctx_s, out_s, max(50, args.steps // 2), 3, flags=G.RENDER_NO_SYNC, sc_dev=rs)
        with torch.cuda.stream(side):
            ctx_s.render(rs, cam, bg, out_s)
            ctx_b.render(ds, cam, bg, out_b)
        torch.cuda.synchronize()
        diff = (out_s[0] - out_b[0]).abs()
        spatial = {"frame_ms": round(mean(ms_s), 4), "raster_ms": round(mean(st_s["raster"]), 4),
                   "stages_ms": {s: round(mean(v), 4) for s, v in st_s.items() if mean(v) > 0},
                   "frame_ms_as_generated": round(frame_b, 4), "raster_ms_as_generated": round(raster_b, 4),
                   "frame_gain": round(1.0 - mean(ms_s) / frame_b, 4),
                   "reorder_ms_once_per_scene": round(reorder_ms, 4), "entries_per_frame": m_s,
                   "max_abs_err_vs_as_generated": float(diff.max().item()),
                   "pixels_differing": int((diff.amax(dim=2) > 0).sum().item())}
        del ctx_s, out_s, rs, ctx_o

    batch = None
    if not args.no_batch:
        batch = batch_leg(args, dev, side, flush, dist)

    heavy = None
    if not args.no_heavy:
        heavy = heavy_leg(dev, side, flush)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_block(scene, cam)

    if rank != 0:
        return
    value = value_pix_s / 1e6
    res = {
        "metric": METRIC, "value": round(value, 4), "unit": "Mpix/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(frame_b, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(ws),
        "path": "binned EXACT, K=64, 16x16 tiles, frame replayed as one CUDA graph",
        "entries_per_frame": m_b,
        "raster_ms": round(raster_b, 4),
        "raster_ms_source": "CUDA events around the raster kernel on the library stream, un-captured frames",
        "raster_mpix_s": round(P / (raster_b * 1e-3) / 1e6, 3),
        "stages_ms": {s: round(mean(v), 4) for s, v in st_b.items() if mean(v) > 0},
        "global_sort": {"frame_ms": round(frame_g, 4), "raster_ms": round(raster_g, 4),
                        "torch_sort_same_keys_ms": None if sort_lib_ms is None else round(sort_lib_ms, 4),
                        "value": round(value_g_pix_s / 1e6, 4),
                        "stages_ms": {s: round(mean(v), 4) for s, v in st_g.items() if mean(v) > 0}},
        "speedup_raster_vs_global": round(raster_g / raster_b, 4),
        "speedup_frame_vs_global": round(frame_g / frame_b, 4),
        "max_abs_err_vs_global": err_vs_global, "last_id_equal_vs_global": last_equal,
        "paper_policy": {"frame_ms": round(mean(ms_p), 4), "raster_ms": round(mean(st_p["raster"]), 4),
                         "max_abs_err_vs_exact": err_paper},
        "frame_ms_min": round(min(ms_b), 4), "frame_ms_median": round(statistics.median(ms_b), 4),
        "frame_ms_without_graph": {"binned": round(mean(ms_b_ng), 4), "global_sort": round(mean(ms_g_ng), 4)},
        "wall_s_timed": round(wall_b, 3),
        "ablation": ablation,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "train_step": train,
        "planner": planner, "spatial_order": spatial, "batch16": batch, "heavy": heavy,
        "launch_overlap": launch_overlap,
        "gpu_launches": int(launches),
    }
    print(json.dumps(res), flush=True)


def heavy_leg(dev, side, flush, frames=10):
    """The depth-complexity sweep: 3M Gaussians at 1920x1080 and 6M at
    3840x2160 with the camera inside a dense cluster (per-tile ranges of
    ~18k-70k).  Graph-replayed frames of the binned EXACT path, the same path
    with the trained bin planner and the global-sort baseline; raster ms from
    the library's stage events in one un-captured frame; images compared."""
    import numpy as np
    import torch

    from paper_2609_03613_gb300 import planner_train as PT, scenes, tilegs as G

    weights = np.load(PT.WEIGHTS).astype(np.float32) if os.path.exists(PT.WEIGHTS) else None
    res = {}
    for name in ("heavy3m", "heavy6m_4k"):
        sc, cam = scenes.workload(name)
        ds = G.DeviceScene.from_numpy(sc, dev)
        H, W = cam.height, cam.width
        r = {"gaussians": sc.n, "resolution": f"{W}x{H}"}
        ref = None
        rs = None
        for label, mode, kw in (("exact", "exact", {}), ("exact_morton_storage", "exact", {}),
                                ("planner", "exact", {"planner": 1}), ("global_sort", "global", {})):
            if label == "planner" and weights is None:
                continue
            scene_dev = ds
            if label == "exact_morton_storage":
                # raster-order-aware storage (the scene permuted once; ties in
                # depth may order differently, so its image is not compared)
                rs, _ = G.Context("exact").reorder_scene(ds)
                scene_dev = rs
            ctx = G.Context(mode, **kw)
            if label == "planner":
                ctx.set_planner_weights(torch.from_numpy(weights))
            out = (torch.empty((H, W, 3), device=dev), torch.empty((H, W), device=dev),
                   torch.empty((H, W), dtype=torch.int32, device=dev))
            with torch.cuda.stream(side):
                ctx.render(scene_dev, cam, (0, 0, 0), out)
            torch.cuda.synchronize()
            m = ctx.last_entry_count()
            ctx.reserve(ds.n, int(m * 1.05) + 1024, W, H)
            fl = G.RENDER_NO_SYNC | G.RENDER_GRAPH
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(frames)]
            with torch.cuda.stream(side):
                for _ in range(3):
                    ctx.render(scene_dev, cam, (0, 0, 0), out, flags=fl)
                for i in range(frames):
                    flush.zero_()
                    ev[i][0].record()
                    ctx.render(scene_dev, cam, (0, 0, 0), out, flags=fl)
                    ev[i][1].record()
                ctx.enable_timing(True)
                ctx.render(scene_dev, cam, (0, 0, 0), out, flags=G.RENDER_NO_SYNC)
            torch.cuda.synchronize()
            st = ctx.stage_times()
            assert ctx.error() == 0
            frame = sum(a.elapsed_time(b) for a, b in ev) / frames
            r[label] = {"frame_ms": round(frame, 4), "raster_ms": round(st["raster"], 4),
                        "stages_ms": {k: round(v, 4) for k, v in st.items() if v > 0}}
            if label == "planner":
                r[label]["tiles_to_second_pass"] = ctx.flagged_tiles()
            if label != "exact_morton_storage":
                r["entries_per_frame"] = m
            if ref is None:
                ref = (out[0].clone(), out[2].clone())
            elif label == "exact_morton_storage":
                r[label]["max_abs_err_vs_exact"] = float((out[0] - ref[0]).abs().max().item())
                del rs
                rs = None
            else:
                r[label]["image_equal_exact"] = bool(torch.equal(out[0], ref[0]) and torch.equal(out[2], ref[1]))
            ctx.close()
            del out
            torch.cuda.empty_cache()
        g, e = r["global_sort"], r["exact"]
        if "planner" in r:
            r["planner_frame_gain_vs_exact"] = round(1.0 - r["planner"]["frame_ms"] / e["frame_ms"], 4)
        r["speedup_frame_vs_global"] = round(g["frame_ms"] / e["frame_ms"], 3)
        r["speedup_raster_vs_global"] = round(g["raster_ms"] / e["raster_ms"], 3)
        res[name] = r
        del ds, ref
        torch.cuda.empty_cache()
    return res


def batch_leg(args, dev, side, flush, dist):
    """16 views of a 2M-Gaussian scene (resolutions 512^2 .. 1080p): one
    gs_render_batch graph (default per-view config, then autotuned) against
    16 single-view graphs issued back to back."""
    import torch

    from paper_2609_03613_gb300 import scenes, tilegs as G
    scene, cams = scenes.workload("batch16")
    ds = G.DeviceScene.from_numpy(scene, dev)
    P = sum(c.width * c.height for c in cams)
    steps = max(10, args.steps // 15)

    def timed(fn, n):
        with torch.cuda.stream(side):
            for _ in range(3):
                fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        with torch.cuda.stream(side):
            for i in range(n):
                flush.zero_()
                ev[i][0].record()
                fn()
                ev[i][1].record()
        torch.cuda.synchronize()
        return max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / n, dist, dev)

    gflags = G.RENDER_NO_SYNC | G.RENDER_GRAPH
    # 16 single-view contexts, each replaying its own frame graph
    singles = []
    for cam in cams:
        c = G.Context("exact")
        out = c.render(ds, cam)
        torch.cuda.synchronize()
        c.reserve(ds.n, int(c.last_entry_count() * 1.25) + 1024, cam.width, cam.height)
        singles.append((c, cam, out))

    def run_singles():
        for c, cam, out in singles:
            c.render(ds, cam, (0.0, 0.0, 0.0), out, flags=gflags)

    ms_single = timed(run_singles, steps)
    del singles
    ctx = G.Context("exact")
    outs = ctx.render_batch(ds, cams)
    torch.cuda.synchronize()
    l0 = ctx.launch_count()
    ms_batch = timed(lambda: ctx.render_batch(ds, cams, (0.0, 0.0, 0.0), outs, flags=gflags), steps)
    launches = (ctx.launch_count() - l0) / (steps + 3)
    t0 = time.perf_counter()
    best = ctx.batch_autotune(ds, cams, tune_tile=True, iters=2)
    tune_s = time.perf_counter() - t0
    outs = ctx.render_batch(ds, cams)
    torch.cuda.synchronize()
    ms_tuned = timed(lambda: ctx.render_batch(ds, cams, (0.0, 0.0, 0.0), outs, flags=gflags), steps)
    assert ctx.error() == 0
    cfgs = [(ctx.batch_view_config(v).tile_size, ctx.batch_view_config(v).K) for v in range(len(cams))]
    return {"views": len(cams), "gaussians": ds.n, "pixels": P, "steps": steps,
            "resolutions": [f"{c.width}x{c.height}" for c in cams],
            "single_view_graphs_ms": round(ms_single, 4), "batch_graph_ms": round(ms_batch, 4),
            "batch_tuned_ms": round(ms_tuned, 4),
            "mpix_s": {"single_view_graphs": round(P / (ms_single * 1e-3) / 1e6, 2),
                       "batch": round(P / (ms_batch * 1e-3) / 1e6, 2),
                       "batch_tuned": round(P / (ms_tuned * 1e-3) / 1e6, 2)},
            "launches_per_batch": launches, "tuned_tile_K": cfgs, "tune_s": round(tune_s, 2),
            "tuned_view_ms": [round(x, 4) for x in best]}


def run_profile_frame(args):
    """Minimal frame sequence for Nsight Compute captures."""
    import torch

    from paper_2609_03613_gb300 import scenes, tilegs as G
    scene, cam = scenes.workload(args.workload)
    ds = G.DeviceScene.from_numpy(scene, "cuda")
    if args.spatial:
        ds, _ = G.Context("exact").reorder_scene(ds)
        torch.cuda.synchronize()
    for mode in args.modes.split(","):
        ctx = G.Context(mode)
        for _ in range(3):
            ctx.render(ds, cam)
        torch.cuda.synchronize()
        assert ctx.error() == 0
        print(mode, "entries", ctx.last_entry_count(), flush=True)
        if args.backward:
            rgb, _, _ = ctx.render(ds, cam, flags=G.RENDER_SAVE)
            target = torch.from_numpy(scenes.random_target(cam.height, cam.width, 5)).cuda()
            dl = (torch.sign(rgb - target) / rgb.numel()).contiguous()
            ctx.render_bwd(dl)
            torch.cuda.synchronize()
            assert ctx.error() == 0


def main():
    args = parse_args()
    if args.profile_frame:
        run_profile_frame(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
    try:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()
    except Exception:
        pass


if __name__ == "__main__":
    main()
