#!/usr/bin/env python
"""Throughput of the fused pyramidal FAST + 3x3 NMS + cell-max detector.

Default workload ("mixed64"): one step = one batched call over 64 frames
(16 each of 640x480, 752x480, 1280x720, 1920x1080; seeds 2..65), 3 levels,
FAST-9, threshold 15, 3x3 NMS, 32x32 cells, SAD-B score.  Inputs rotate over
4 device-resident copies of the batch (4 x 58.6 MB > the 129 MB L2), so no
step starts with its frames in L2.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead, on the host cores.
"""
from __future__ import annotations

import argparse
import csv
import gc
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "frames/s & Mpixel/s detect+grid-NMS (batched/served vs plain), p50/p99 frame latency"

WORKLOADS = {
    "mixed64": dict(levels=3, thresh=15, arc=9, cell=32,
                    desc="64 frames in one batched launch: 16 each of 640x480, 752x480, 1280x720, "
                         "1920x1080 (seeds 2..65, 40 shapes), 3-level pyramid, FAST-9, thresh 15, "
                         "3x3 NMS, 32x32 or 64x64 cells picked by the autotuner, SAD-B"),
    "large4k": dict(levels=4, thresh=10, arc=9, cell=64, sweep=[(t, a) for a in (12, 9) for t in (5, 10, 20, 40)],
                    desc="32 frames of 3840x2160 (seeds 100..131, 400 shapes), 4-level pyramid built once, "
                         "FAST-12 and FAST-9 at thresholds 5, 10, 20, 40 (8 detections per step), 3x3 NMS, "
                         "64x64 cells, SAD-B"),
    "single752": dict(levels=3, thresh=20, arc=9, cell=32,
                      desc="one 752x480 frame (seed 1), 3-level pyramid, FAST-9, thresh 20, 3x3 NMS, "
                           "32x32 cells, SAD-B"),
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="mixed64")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle baseline leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip plain/e2e/profile legs")
    ap.add_argument("--spin", type=float, default=0.5, help="seconds of untimed steps before timing")
    ap.add_argument("--variant", type=int, default=-1, help="pin a tile variant instead of autotuning")
    ap.add_argument("--cell", type=int, default=0, help="pin the cell size instead of the workload's choice")
    ap.add_argument("--no-tracker", action="store_true", help="skip the feature-tracker leg")
    ap.add_argument("--no-large4k", action="store_true", help="skip the 4K sweep leg of the default run")
    ap.add_argument("--tracker-only", action="store_true",
                    help="run only the feature-tracker leg and print its JSON object")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the Poisson serving run (0 skips it)")
    return ap.parse_args()


def make_frames(workload: str):
    from paper_2003_13493_gb300 import synth

    if workload == "mixed64":
        return synth.mixed_batch(first_seed=2, per_size=16)
    if workload == "large4k":
        return [synth.make_frame(3840, 2160, seed=100 + i, n_shapes=400) for i in range(32)]
    return [synth.make_frame(752, 480, seed=1)]


# ---- clocks -------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu=timestamp,{self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def mark(self, which: str):
        setattr(self, which, time.time())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.05)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = []
        for r in csv.reader(io.StringIO(out)):
            if len(r) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(r[0].strip().split(".")[0], "%Y/%m/%d %H:%M:%S"))
                rows.append((ts, [c.strip() for c in r[1:]]))
            except ValueError:
                continue
        inside = [v for ts, v in rows if self.t0 is not None and self.t0 - 1 <= ts <= self.t1 + 1]
        use = inside or [v for _, v in rows]
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(v[1]) for v in use if v[1].replace(".", "").isdigit()]
        mx = [float(v[2]) for v in use if v[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for v in use:
            for name, val in zip(names, v[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(use), "samples_in_window": len(inside)}


# ---- ncu traffic recorded for the current kernel source ------------------------

KERNEL_SOURCES = {
    "fast_nms_cell": ("ptx.cuh", "vio_kernels.cuh"),
    "fast_sweep": ("ptx.cuh", "vio_kernels.cuh", "vio_sweep.cuh"),
}


def kernel_source_hash(kernel: str = "fast_nms_cell") -> str:
    """Hash of the code a detect kernel is compiled from: its sources with
    comments and blank space removed, so that edits of comments alone keep
    a recorded profile valid."""
    import re

    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2003_13493_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def recorded_profile(workload: str, kernel: str = "fast_nms_cell") -> dict:
    """Figures of a detect kernel's committed ncu summary
    (profiles/<kernel>_<workload>.md: `key: value` lines), if it was taken on
    the current kernel source; else {}."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return {}
    vals = {}
    with open(path) as f:
        for line in f:
            for key in ("kernel_source_sha256", "dram_bytes_per_launch", "alu_pipe_pct", "issue_active_pct",
                        "warp_instructions_per_launch"):
                if line.startswith(key + ":"):
                    vals[key] = line.split(":", 1)[1].split()[0].strip()
    if vals.get("kernel_source_sha256") != kernel_source_hash(kernel):
        return {}
    return vals


def recorded_traffic(workload: str, kernel: str = "fast_nms_cell"):
    """dram bytes per launch from the committed ncu summary, or None."""
    v = recorded_profile(workload, kernel).get("dram_bytes_per_launch")
    return float(v) if v is not None else None


def max_over_ranks(value: float) -> float:
    """Largest `value` over all ranks (identity without torch.distributed).
    Uses a CUDA tensor under NCCL and a CPU tensor otherwise (gloo)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_rate(units_per_rank: int, steps: int, ms_max: float, world: int) -> float:
    """Whole-job throughput: every rank did units_per_rank per step; the job
    took the slowest rank's time."""
    return world * units_per_rank * steps / (ms_max / 1e3)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0}, "fallback"


# ---- CPU oracle leg ------------------------------------------------------------

def oracle_rate(frames, wl, seconds: float, cores: int = 0):
    """Frames/s of the plain C oracle over a bounded sample, frame-parallel on
    `cores` threads (all host cores by default; ctypes releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    oracle.build()
    by_size = {}
    for f in frames:
        by_size.setdefault(f.shape, []).append(f)
    sample = [v[i] for v in by_size.values() for i in range(min(2, len(v)))]
    cores = cores or os.cpu_count() or 1
    settings = wl.get("sweep") or [(wl["thresh"], wl["arc"])]

    def one(im):  # a frame is done when every setting of the workload is
        for t, a in settings:
            oracle.detect(im, t, a, wl["cell"], wl["levels"])

    done = 0
    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        while True:
            list(ex.map(one, sample))
            done += len(sample)
            if time.perf_counter() - t0 >= seconds:
                break
    dt = time.perf_counter() - t0
    desc = "+".join(f"{len(v[:2])}x{s[1]}x{s[0]}" for s, v in by_size.items())
    return done / dt, cores, f"{desc} frames of the workload, repeated {done // len(sample)}x ({dt:.1f} s)"


# ---- our implementation ------------------------------------------------------------

def algorithmic_bytes(dims, levels, cell, num_cells, npar=1):
    """Per-step bytes and the detect kernel's bytes per launch.

    A step reads level 0 once, writes and reads each pyramid level once and
    writes 16 bytes per cell.  A sweep of npar settings is one fused pass: the
    levels are read once for all settings, each setting writes its own cells.
    The detect kernel reads every level once and updates 8 bytes of key per
    cell and setting."""
    step = 0.0
    fused = 0.0
    for (w, h) in dims:
        nc = num_cells(w, h, cell)
        pyr_px = sum((w >> k) * (h >> k) for k in range(1, levels))
        all_px = sum((w >> k) * (h >> k) for k in range(levels))
        step += w * h + 2 * pyr_px + npar * 16 * nc
        fused += all_px + 8 * nc * npar
    return step, fused


def run_ours(args, rank, world, local_rank):
    import ctypes

    import torch

    from paper_2003_13493_gb300 import vio

    wl = dict(WORKLOADS[args.workload])
    if args.cell:
        wl["cell"] = args.cell
    # the mixed batch's cell size (32 or 64) is the autotuner's pick: the timed
    # calls pass cell_size 0, everything after the warm-up uses the size it chose
    auto_cell = args.workload == "mixed64" and not args.cell and args.variant < 0
    call_cell = 0 if auto_cell else wl["cell"]
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    frames_np = make_frames(args.workload)
    n = len(frames_np)
    dims = [(f.shape[1], f.shape[0]) for f in frames_np]
    mpx = sum(w * h for w, h in dims) / 1e6
    # enough device copies that the inputs of a step are not in L2 (129 MB)
    sets = max(1, -(-200 // max(1, int(mpx))))
    stream = torch.cuda.Stream(device=dev)
    sh = ctypes.c_void_p(stream.cuda_stream)

    det = vio.Detector(device=local_rank, max_frames=max(64, n), autotune=args.variant < 0)
    if args.variant >= 0:
        det.set_variant(args.variant)
    dev_sets = []
    with torch.cuda.stream(stream):
        for _ in range(sets):
            dev_sets.append([torch.from_numpy(f).to(dev) for f in frames_np])
    sweep = wl.get("sweep")
    npar = len(sweep) if sweep else 1
    outs = [torch.empty((vio.num_cells(w, h, call_cell or 32), 4), dtype=torch.int32, device=dev)
            for _ in range(npar) for w, h in dims]
    counts = torch.empty(npar * n, dtype=torch.int32, device=dev)

    def marshal(frames):
        d = (vio.Dims * n)(*[vio.Dims(f.shape[1], f.shape[0], f.stride(0)) for f in frames])
        fp = (ctypes.c_void_p * n)(*[f.data_ptr() for f in frames])
        return fp, d

    marshalled = [marshal(s) for s in dev_sets]
    optr = (ctypes.c_void_p * (npar * n))(*[o.data_ptr() for o in outs])
    cptr = ctypes.c_void_p(counts.data_ptr())
    if sweep:
        th = (ctypes.c_int * npar)(*[p[0] for p in sweep])
        ar = (ctypes.c_int * npar)(*[p[1] for p in sweep])

    def step(i, d=det):
        fp, dd = marshalled[i % sets]
        if sweep:
            d.detect_sweep_ptrs(fp, dd, n, th, ar, npar, wl["cell"], wl["levels"], optr, cptr, sh)
        else:
            d.detect_ptrs(fp, dd, n, wl["thresh"], wl["arc"], call_cell, wl["levels"], optr, cptr, sh)

    for i in range(max(3, args.warmup)):
        step(i)
    det.sync(stream)
    tune = det.tuning()
    tune_full = det.tuning_full()
    tune_log = det.autotune_log()
    if auto_cell:
        wl["cell"] = tune_full["cell_size"]

    dist = None
    if world > 1:
        import torch.distributed as dist
    clocks = ClockSampler(local_rank)
    clocks.start()
    # bring clocks up before the timed region
    t_spin = time.perf_counter()
    i = 0
    while time.perf_counter() - t_spin < args.spin:
        step(i)
        i += 1
    det.sync(stream)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks.mark("t0")
    e0.record(stream)
    for i in range(args.steps):
        step(i)
    e1.record(stream)
    det.sync(stream)
    torch.cuda.synchronize(dev)
    clocks.mark("t1")
    if dist:
        dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1))
    clk = clocks.stop()
    ms_per_step = ms / args.steps
    fps = weak_scaling_rate(n, args.steps, ms, world)

    res = {
        "metric": METRIC, "value": round(fps, 1), "unit": "frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded value noise + shapes, integer generator)",
        "mpixel_per_s": round(world * mpx * args.steps / (ms / 1e3), 1),
        "config": {"workload": f"{args.workload}: {wl['desc']}", "frames_per_step": n,
                   "detections_per_frame": npar,
                   "mpixel_per_step": round(mpx, 3), "levels": wl["levels"], "thresh": wl["thresh"],
                   "arc_len": wl["arc"], "cell": wl["cell"], "score": "SAD-B",
                   "l2": f"inputs rotate over {sets} device copies of the batch "
                         f"({sets * mpx:.0f} MB > 129 MB L2)",
                   "tile": {"w": tune[0], "h": tune[1], "variant": tune[2],
                            "rows_per_warp": tune[1] // 8 + (1 if tune[1] % 8 else 0),
                            "cta_per_sm": tune_full["cta_per_sm"],
                            "picked_by": ("fixed: the sweep kernel's tile, CTAs per SM from its occupancy" if sweep
                                          else "autotuner" if args.variant < 0 else "--variant")},
                   "cell_picked_by": "autotuner (32 or 64)" if auto_cell else ("--cell" if args.cell else "workload"),
                   "parallelism": f"replicas x{world}, no collective"},
        "clocks": clk,
        # per step: the pyramid, then a detect and a decode kernel per launch
        # (a sweep detects up to 8 settings per launch)
        "gpu_launches": args.steps * ((1 if wl["levels"] > 1 else 0) + 2 * ((npar + 7) // 8 if sweep else 1)),
    }
    if tune_log:
        res["autotune"] = {"chosen": {k: tune_full[k] for k in ("variant", "tile_h", "cta_per_sm", "cell_size")},
                           "alternatives": [{k: e[k] for k in ("variant", "tile_h", "cta_per_sm", "cell_size", "ms")}
                                            for e in tune_log],
                           "what": "ms per call of every configuration the tuner timed on this batch"}
    # later legs reuse the tuned configuration instead of tuning again
    if args.variant < 0:
        det.set_variant(tune_full["variant"], cta_per_sm=tune_full["cta_per_sm"])
    if sweep:
        res["detections_per_s"] = round(world * n * npar * args.steps / (ms / 1e3), 1)
    if not args.no_extras and not sweep:
        res["e2e"] = e2e_leg(args, wl, det, dev, stream, frames_np, dims, n, world)
    if world > 1:
        args.no_cpu_baseline = True  # the oracle baseline is an N = 1 figure
    if rank == 0 and not args.no_extras:
        res.update(extras(args, wl, det, dev, stream, sh, frames_np, dims, marshalled, optr, cptr, n, mpx,
                          ms_per_step))
        alu = res.get("roofline", {}).get("alu", {})
        kern_ms = res.get("stage_ms", {}).get(res["roofline"]["kernel"].replace("_kernel", "")) if alu else None
        if "warp_instructions_per_launch" in alu and kern_ms and (clk or {}).get("sm_mhz"):
            # the issue roofline: warp instructions the kernel executes (ncu, same
            # source) over its live duration, against one instruction per cycle
            # per scheduler (4 per SM) at the SM clock sampled under load
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            ach = alu["warp_instructions_per_launch"] / (kern_ms * 1e-3) / 1e9
            pk = sms * 4 * clk["sm_mhz"] * 1e6 / 1e9
            alu["issue"] = {"achieved": round(ach, 1), "peak": round(pk, 1), "unit": "G warp instructions/s",
                            "frac": round(ach / pk, 4),
                            "peak_from": f"{sms} SMs x 4 schedulers x 1 instruction/cycle x {clk['sm_mhz']:.0f} MHz"}
    det.close()
    return res


def e2e_leg(args, wl, det, dev, stream, frames_np, dims, n, world) -> dict:
    """End to end through the host-buffer entry points (pinned host frames and
    outputs): each step copies its frames in and its records out.  Every rank
    runs it on its own GPU; the whole-job rate divides all ranks' frames by
    the slowest rank's time.  The frames lie back to back in one pinned
    buffer, as a camera ring buffer delivers them (uploaded in one copy); the
    same frames in separate allocations are timed beside it."""
    import torch

    from paper_2003_13493_gb300 import vio

    separate = [torch.from_numpy(f).pin_memory() for f in frames_np]
    arena = torch.empty(sum(f.size for f in frames_np), dtype=torch.uint8).pin_memory()
    packed, o = [], 0
    for f in frames_np:
        v = arena[o:o + f.size].view(f.shape)
        v.copy_(torch.from_numpy(f))
        packed.append(v)
        o += f.size

    def pinned_outs():
        o = [torch.empty((vio.num_cells(w, h, wl["cell"]), 4), dtype=torch.int32).pin_memory().numpy()
             for w, h in dims]
        return o, torch.empty(n, dtype=torch.int32).pin_memory().numpy()

    e2e_det = vio.Detector(device=dev.index, max_frames=max(64, n))
    e2e_det.set_variant(det.tuning()[2])
    esteps = max(3, min(args.steps, 50))
    streams = [torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)]
    bufs = [pinned_outs(), pinned_outs()]

    def rates(host_frames):
        # the buffers are marshalled once (vio.HostBatch), as a camera ring's
        # fixed slots would be; every step is one C call on them
        wk = (wl["thresh"], wl["arc"], wl["cell"], wl["levels"])
        sync_batch = vio.HostBatch(host_frames, *pinned_outs())
        # synchronous: one vio_detect_host call per step
        for _ in range(3):
            e2e_det.detect_host_batch(sync_batch, *wk, stream=stream)
        barrier()
        t0 = time.perf_counter()
        for _ in range(esteps):
            e2e_det.detect_host_batch(sync_batch, *wk, stream=stream)
        dt_sync = max_over_ranks(time.perf_counter() - t0)
        # pipelined: vio_detect_host_async on two alternating streams, so that
        # a step's frame copies overlap the previous step's kernels
        batches = [vio.HostBatch(host_frames, *b) for b in bufs]
        for i in range(4):
            e2e_det.detect_host_batch(batches[i % 2], *wk, stream=streams[i % 2], pipelined=True)
        for st in streams:
            e2e_det.sync(st)
        barrier()
        t0 = time.perf_counter()
        for i in range(esteps):
            e2e_det.detect_host_batch(batches[i % 2], *wk, stream=streams[i % 2], pipelined=True)
        for st in streams:
            e2e_det.sync(st)
        dt = max_over_ranks(time.perf_counter() - t0)
        return round(world * esteps * n / dt, 1), round(world * esteps * n / dt_sync, 1)

    packed_async, packed_sync = rates([v.numpy() for v in packed])
    sep_async, sep_sync = rates([t.numpy() for t in separate])
    e2e_det.close()
    # the host link's rate for one copy of the whole buffer: the bound of the
    # pipelined path
    dst = torch.empty(arena.numel(), dtype=torch.uint8, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    with torch.cuda.stream(stream):
        for _ in range(6):
            e0.record(stream)
            dst.copy_(arena, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
    link_gbs = arena.numel() / (best * 1e-3) / 1e9
    e2e_gbs = packed_async / world * arena.numel() / n / 1e9
    # bytes of one job step: every rank copies its own frames and records
    h2d = world * sum(w * h for w, h in dims)
    d2h = world * (sum(16 * vio.num_cells(w, h, wl["cell"]) for w, h in dims) + 4 * n)
    return {"value": packed_async, "unit": "frames/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": esteps,
            "what": "vio_detect_host_async on two alternating streams, the step's frames back to back in one "
                    "pinned buffer (one copy-engine copy): frames copied in, records written into pinned host "
                    "memory, counts copied back, all inside the timed region; buffers marshalled once "
                    "(vio.HostBatch), one C call per step",
            "sync": {"value": packed_sync, "unit": "frames/s",
                     "what": "vio_detect_host, one synchronous call per step, same buffer"},
            "host_link": {"achieved_gbs": round(e2e_gbs, 1), "one_copy_gbs": round(link_gbs, 1),
                          "frac": round(e2e_gbs / link_gbs, 3),
                          "what": "frame bytes uploaded per second by the pipelined path, against one "
                                  "cudaMemcpyAsync of the same pinned buffer timed alone"},
            "separate_frames": {"value": sep_async, "sync": sep_sync, "unit": "frames/s",
                                "what": "each frame in its own pinned allocation: one copy per frame when "
                                        "pipelined; read by the pyramid kernel through its device mapping "
                                        "when synchronous"}}


def barrier():
    """torch.distributed barrier when a process group is up (no-op otherwise)."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def extras(args, wl, det, dev, stream, sh, frames_np, dims, marshalled, optr, cptr, n, mpx, ms_per_step):
    import ctypes

    import torch

    from paper_2003_13493_gb300 import vio

    out = {}
    # roofline of the fused kernel: stage events captured inside the graph
    prof = vio.Detector(device=dev.index, max_frames=max(64, n), profile=True)
    tf = det.tuning_full()
    prof.set_variant(tf["variant"], cta_per_sm=tf["cta_per_sm"])
    steps = min(args.steps, 200)
    acc = [0.0, 0.0, 0.0]
    sweep = wl.get("sweep")
    npar = len(sweep) if sweep else 1
    if sweep:
        th = (ctypes.c_int * npar)(*[p[0] for p in sweep])
        ar = (ctypes.c_int * npar)(*[p[1] for p in sweep])
        sw_optr = (ctypes.c_void_p * (npar * n))(*([optr[i] for i in range(n)] * npar))
        sw_counts = torch.empty(npar * n, dtype=torch.int32, device=dev)
    for i in range(steps + 3):
        fp, dd = marshalled[i % len(marshalled)]
        # the stage events time each kernel of the step's (last) launch: for a
        # sweep of at most 8 settings that is the one fused launch
        if sweep:
            prof.detect_sweep_ptrs(fp, dd, n, th, ar, npar, wl["cell"], wl["levels"], sw_optr,
                                   ctypes.c_void_p(sw_counts.data_ptr()), sh)
        else:
            prof.detect_ptrs(fp, dd, n, wl["thresh"], wl["arc"], wl["cell"], wl["levels"], optr, cptr, sh)
        st = prof.stage_ms()
        if i >= 3:
            acc = [a + b for a, b in zip(acc, st)]
    prof.close()
    stage = [a / steps for a in acc]
    step_bytes, fused_bytes = algorithmic_bytes(dims, wl["levels"], wl["cell"], vio.num_cells, npar)
    peaks, kind = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = fused_bytes / (stage[1] * 1e-3) / 1e9
    kname = "fast_sweep_kernel" if sweep and npar <= 8 else "fast_nms_cell_kernel"
    traffic = recorded_traffic(args.workload, kname.replace("_kernel", ""))
    out["roofline"] = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                       "frac": round(achieved / peak, 4), "traffic": traffic,
                       "kernel": kname, "peak_kind": f"{kind} hbm_gbs",
                       "algorithmic_bytes_per_launch": int(fused_bytes)}
    # where `traffic` comes from: not measured in this run, but read from the
    # committed ncu summary of the same kernel source (matched by hash); null
    # when the source changed since that capture
    out["roofline"]["traffic_source"] = {
        "profile": f"profiles/{kname.replace('_kernel', '')}_{args.workload}.md",
        "kernel_source_sha256": kernel_source_hash(kname.replace("_kernel", "")),
        "matched": traffic is not None}
    prof_vals = recorded_profile(args.workload, kname.replace("_kernel", ""))
    if "alu_pipe_pct" in prof_vals:
        # what binds instead: integer issue (ncu on the same kernel source)
        out["roofline"]["alu"] = {"pipe_alu_pct": float(prof_vals["alu_pipe_pct"]),
                                  "issue_active_pct": float(prof_vals["issue_active_pct"]),
                                  "binds": "integer issue: the ALU pipe is this busy while DRAM moves the "
                                           "algorithmic bytes at the HBM fraction above",
                                  "source": f"profiles/{kname.replace('_kernel', '')}_{args.workload}.md"}
        if "warp_instructions_per_launch" in prof_vals:
            out["roofline"]["alu"]["warp_instructions_per_launch"] = int(prof_vals["warp_instructions_per_launch"])
    out["stage_ms"] = {"pyramid": round(stage[0], 5), kname.replace("_kernel", ""): round(stage[1], 5),
                       "decode": round(stage[2], 5)}
    step_gbs = step_bytes / (ms_per_step * 1e-3) / 1e9
    out["step_roofline"] = {"algorithmic_bytes_per_step": int(step_bytes), "achieved_gbs": round(step_gbs, 1),
                            "frac": round(step_gbs / peak, 4),
                            "what": "whole step (pyramid + fused detect + decode) against the HBM peak"}

    if sweep:
        return out

    # the other scores of Section II-D on the same batches (same tile variant)
    scores = {}
    for name, mode in (("sad_a", vio.SCORE_SAD_A), ("mt", vio.SCORE_MT)):
        d = vio.Detector(device=dev.index, max_frames=max(64, n), score=mode)
        d.set_variant(det.tuning()[2])
        ssteps = max(5, min(args.steps, 200))
        for i in range(3):
            fp, dd = marshalled[i % len(marshalled)]
            d.detect_ptrs(fp, dd, n, wl["thresh"], wl["arc"], wl["cell"], wl["levels"], optr, cptr, sh)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(ssteps):
            fp, dd = marshalled[i % len(marshalled)]
            d.detect_ptrs(fp, dd, n, wl["thresh"], wl["arc"], wl["cell"], wl["levels"], optr, cptr, sh)
        e1.record(stream)
        d.sync(stream)
        sms = e0.elapsed_time(e1) / ssteps
        d.close()
        scores[name] = {"value": round(n / (sms / 1e3), 1), "unit": "frames/s", "ms_per_step": round(sms, 5)}
    out["scores"] = scores

    # Table III's windows: 3x3 .. 9x9 NMS, on the same batches at 1 level, FAST-10, thresh 10
    wins = {}
    for r in (1, 2, 3, 4):
        d = vio.Detector(device=dev.index, max_frames=max(64, n), nms_radius=r)
        wsteps = max(5, min(args.steps, 200))
        for i in range(3):
            fp, dd = marshalled[i % len(marshalled)]
            d.detect_ptrs(fp, dd, n, 10, 10, 32, 1, optr, cptr, sh)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(wsteps):
            fp, dd = marshalled[i % len(marshalled)]
            d.detect_ptrs(fp, dd, n, 10, 10, 32, 1, optr, cptr, sh)
        e1.record(stream)
        d.sync(stream)
        wms = e0.elapsed_time(e1) / wsteps
        d.close()
        wins[f"{2 * r + 1}x{2 * r + 1}"] = {"value": round(n / (wms / 1e3), 1), "unit": "frames/s",
                                            "ms_per_step": round(wms, 5)}
    out["nms_windows"] = {"what": "the batch at 1 level, FAST-10, thresh 10, 32x32 cells (Table III's setting)",
                          **wins}

    # plain path: one frame per call
    plain = vio.Detector(device=dev.index, max_frames=4)
    plain.set_variant(det.tuning()[2])
    single = [((ctypes.c_void_p * 1)(marshalled[s][0][i]), (vio.Dims * 1)(marshalled[s][1][i]),
               (ctypes.c_void_p * 1)(optr[i])) for s in range(len(marshalled)) for i in range(n)]
    psteps = max(3, min(args.steps, 100))
    for j in range(n * 2):
        fp, dd, op = single[j % len(single)]
        plain.detect_ptrs(fp, dd, 1, wl["thresh"], wl["arc"], wl["cell"], wl["levels"], op, None, sh)
    plain.sync(stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for j in range(psteps * n):
        fp, dd, op = single[j % len(single)]
        plain.detect_ptrs(fp, dd, 1, wl["thresh"], wl["arc"], wl["cell"], wl["levels"], op, None, sh)
    e1.record(stream)
    plain.sync(stream)
    pms = e0.elapsed_time(e1)
    plain.close()
    out["plain"] = {"value": round(psteps * n / (pms / 1e3), 1), "unit": "frames/s",
                    "what": "same frames, one vio_detect call (and graph replay) per frame"}

    out["latency"] = latency_leg(args, dev.index)
    if args.serve_seconds > 0:
        out["serving"] = serving_leg(args, dev.index)
        out["serving_saturation"] = serving_saturation_leg(args, dev.index)
    if args.workload == "mixed64" and not args.no_large4k:
        out["large4k"] = large4k_leg(args, dev.index)
    if not args.no_tracker:
        out["tracker"] = tracker_leg(args, dev.index)

    if not args.no_cpu_baseline:
        rate, cores, sample = oracle_rate(frames_np, wl, args.cpu_seconds)
        rate1, _, sample1 = oracle_rate(frames_np, wl, args.cpu_seconds / 3, cores=1)
        out["cpu_baseline"] = {"value": round(rate, 2), "unit": "frames/s", "cores": cores, "kind": "oracle",
                               "sample": sample,
                               "single_core": {"value": round(rate1, 2), "unit": "frames/s", "cores": 1,
                                               "sample": sample1}}
    return out


def frontend_loop(args, dev_index: int, det) -> dict:
    """The paper's frontend loop on one camera stream: per 752x480 frame,
    detect (3 levels, FAST-9, thresh 10, 32x32 cells, SAD-B) and track the
    previous frame's grid features into it (vio_track_cells, gain and
    offset), one frame after the other on one stream; frames resident on the
    device, a smooth scene moving 0.9 px right and 0.4 px down per frame."""
    import ctypes

    import numpy as np
    import torch

    from paper_2003_13493_gb300 import synth, vio

    w, h, nfr = 752, 480, 48
    dev = torch.device("cuda", dev_index)
    frames = [torch.from_numpy(synth.smooth_frame(w, h, seed=77, dx=0.9 * t, dy=0.4 * t)).to(dev)
              for t in range(nfr)]
    ncell = vio.num_cells(w, h, 32)
    cells = [torch.empty((ncell, 4), dtype=torch.int32, device=dev) for _ in range(2)]
    res = torch.empty((ncell, vio.TRACK_RESULT_WORDS), dtype=torch.float32, device=dev)
    dims = (vio.Dims * 1)(vio.Dims(w, h, w))
    sh = vio._stream_handle(torch.cuda.current_stream(dev))
    tp = vio.TrackParams()
    det.lib.vio_track_params_default(ctypes.byref(tp))
    one = lambda p: (ctypes.c_void_p * 1)(p)  # noqa: E731
    fptr = [one(f.data_ptr()) for f in frames]
    cptr = [one(c.data_ptr()) for c in cells]
    optr = one(res.data_ptr())
    cnt = (ctypes.c_int * 1)(ncell)

    def step(t):
        det.detect_ptrs(fptr[t], dims, 1, 10, 9, 32, 3, cptr[t % 2], None, sh)
        if t > 0:
            det.track_cells_ptrs(fptr[t - 1], fptr[t], dims, 1, cptr[(t - 1) % 2], cnt, tp, optr, sh)

    for t in range(nfr):
        step(t)
    det.sync()
    reps = 3
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    e0.record(stream)
    for _ in range(reps):
        for t in range(nfr):
            step(t)
    e1.record(stream)
    det.sync()
    ms = e0.elapsed_time(e1) / (reps * nfr)
    r = res.cpu().numpy()
    _, _, _, status, _, _ = vio.track_fields(r)

    # the same loop on two streams: the detection of frame t runs beside the
    # tracking into frame t-1 (it needs frame t-2's cells, detected two steps
    # earlier); three cell buffers, ordered by events
    sa, sb = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ha, hb = vio._stream_handle(sa), vio._stream_handle(sb)
    cells3 = [torch.empty((ncell, 4), dtype=torch.int32, device=dev) for _ in range(3)]
    cptr3 = [one(c.data_ptr()) for c in cells3]
    det_ev = [torch.cuda.Event() for _ in range(nfr)]
    trk_ev = [torch.cuda.Event() for _ in range(nfr)]

    def step2(t):
        if t >= 2:
            sa.wait_event(trk_ev[t - 2])  # cells3[t % 3] was last read by the track into frame t-2
        det.detect_ptrs(fptr[t], dims, 1, 10, 9, 32, 3, cptr3[t % 3], None, ha)
        det_ev[t].record(sa)
        if t > 0:
            sb.wait_event(det_ev[t - 1])
            det.track_cells_ptrs(fptr[t - 1], fptr[t], dims, 1, cptr3[(t - 1) % 3], cnt, tp, optr, hb)
            trk_ev[t].record(sb)

    def loop2():
        for t in range(nfr):
            step2(t)
        sa.wait_stream(sb)

    sa.wait_stream(stream)
    sb.wait_stream(stream)
    loop2()
    e0.record(sa)
    sb.wait_stream(sa)
    for _ in range(reps):
        loop2()
    e1.record(sa)
    det.sync(sa)
    ms2 = e0.elapsed_time(e1) / (reps * nfr)
    r2 = res.cpu().numpy()
    same = bool(np.array_equal(r2, r))  # the last track of both loops: same frames, same cells
    return {"value": round(1e3 / ms, 1), "unit": "frames/s", "ms_per_frame": round(ms, 4),
            "features_tracked_last_frame": int((status == 1).sum()),
            "what": "per 752x480 frame: vio_detect, then vio_track_cells of the previous frame's grid features "
                    "into it; one stream, frames resident on the device (the paper reports over 1000 fps for "
                    "detection and tracking on a Jetson TX2)",
            "two_streams": {"value": round(1e3 / ms2, 1), "unit": "frames/s", "ms_per_frame": round(ms2, 4),
                            "same_tracks": same,
                            "what": "the same loop with the detection of frame t on one stream beside the "
                                    "tracking into frame t-1 on another"}}


def tracker_leg(args, dev_index: int) -> dict:
    """Feature tracker (Section II-E): throughput of one vio_track call over
    64 pairs of 752x480 frames x 256 features (a 16 x 16 grid inside a 40-pixel
    margin), and the latency of one pair with 100 features for each model of
    Table VI (both pyramids built inside the call).  Frames: the smooth
    moving scene of synth.smooth_frame with seeded sub-pixel motion and
    intensity change; default parameters (3 levels, 16 x 16 / 8 x 8 patches,
    30 iterations, min_update 0.01)."""
    import numpy as np
    import torch

    from oracle import lk_oracle as lk
    from paper_2003_13493_gb300 import synth, vio

    rng = np.random.default_rng(9)
    w, h, npairs = 752, 480, 64
    ys, xs = np.meshgrid(np.linspace(40, h - 40, 16), np.linspace(40, w - 40, 16), indexing="ij")
    grid = np.stack([xs.ravel(), ys.ravel()], axis=1).astype(np.float32)
    pairs = []
    for i in range(npairs):
        dx, dy = rng.uniform(-4, 4, 2)
        g, o = rng.uniform(0.9, 1.1), rng.uniform(-10, 10)
        pairs.append((synth.smooth_frame(w, h, seed=300 + i),
                      synth.smooth_frame(w, h, seed=300 + i, dx=dx, dy=dy, gain=g, offset=o)))
    dev = torch.device("cuda", dev_index)
    prev = [torch.from_numpy(a).to(dev) for a, _ in pairs]
    nxt = [torch.from_numpy(b).to(dev) for _, b in pairs]
    pts = [torch.from_numpy(grid).to(dev) for _ in pairs]
    det = vio.Detector(device=dev_index, max_frames=npairs)
    outs = det.track(prev, nxt, pts)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        det.track(prev, nxt, pts, outs=outs)
    reps = max(5, min(args.steps, 50))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        det.track(prev, nxt, pts, outs=outs)
    e1.record(stream)
    det.sync()
    ms = e0.elapsed_time(e1) / reps
    res = np.concatenate([o.cpu().numpy() for o in outs])
    _, _, _, status, iters, _ = vio.track_fields(res)
    out = {"value": round(npairs * len(grid) / (ms / 1e3), 1), "unit": "features/s",
           "ms_per_call": round(ms, 4), "features_per_call": npairs * len(grid),
           "tracked_frac": round(float((status == 1).mean()), 4), "mean_iters": round(float(iters.mean()), 2),
           "what": "one vio_track call: 64 pairs of 752x480 x 256 features, pyramids of both frames included"}
    # Table VI: 100 features on one pair, per model
    p100 = [torch.from_numpy(grid[::256 // 100][:100].copy()).to(dev)]
    lat = {}
    for name, model in (("trans", 0), ("trans_offset", vio.TRACK_OFFSET), ("trans_gain", vio.TRACK_GAIN),
                        ("trans_gain_offset", vio.TRACK_GAIN | vio.TRACK_OFFSET)):
        o1 = det.track(prev[:1], nxt[:1], p100, dict(model=model))
        for _ in range(5):
            det.track(prev[:1], nxt[:1], p100, dict(model=model), outs=o1)
        det.sync()
        e0.record(stream)
        for _ in range(reps):
            det.track(prev[:1], nxt[:1], p100, dict(model=model), outs=o1)
        e1.record(stream)
        det.sync()
        lat[name] = round(e0.elapsed_time(e1) / reps * 1e3, 1)
    out["latency_us_100_features"] = lat
    out["frontend"] = frontend_loop(args, dev_index, det)
    out["paper_ms_100_features"] = {"tegra_x2": {"trans": 0.96, "trans_offset": 0.90, "trans_gain": 0.91,
                                                 "trans_gain_offset": 1.01},
                                    "gtx_960m": {"trans": 0.33, "trans_offset": 0.28, "trans_gain": 0.29,
                                                 "trans_gain_offset": 0.38}}
    det.close()
    if not args.no_cpu_baseline:
        # the oracle on a bounded sample: the first 64 features of the first pairs
        t0 = time.perf_counter()
        done = 0
        for a, b in pairs:
            lk.track(a, b, grid[:64].astype(np.float64), levels=3)
            done += 64
            if time.perf_counter() - t0 > min(5.0, args.cpu_seconds):
                break
        out["cpu_baseline"] = {"value": round(done / (time.perf_counter() - t0), 1), "unit": "features/s",
                               "cores": 1, "kind": "oracle",
                               "sample": f"{done} features of the same pairs, fp64 numpy, one thread"}
    return out


def latency_leg(args, dev_index: int) -> dict:
    """Per-frame latency of one 752x480 frame per call, synchronised after
    every call: the single-frame workloads (seed 0: FAST-9, thresh 10, one
    level; seed 1: thresh 20, 3 levels; 32x32 cells).  'device': frame and
    cells in device memory (vio_detect, then vio_sync); 'host': pinned host
    frame in, records into pinned host memory (vio_detect_host, upload and
    download included)."""
    import ctypes

    import numpy as np
    import torch

    from paper_2003_13493_gb300 import synth, vio

    dev = torch.device("cuda", dev_index)
    stream = torch.cuda.current_stream(dev)
    sh = vio._stream_handle(stream)
    w, h, reps = 752, 480, 400
    ncell = vio.num_cells(w, h, 32)
    out = {}
    for name, seed, thresh, levels in (("seed0_1level", 0, 10, 1), ("seed1_3levels", 1, 20, 3)):
        img = synth.make_frame(w, h, seed)
        det = vio.Detector(device=dev_index, max_frames=1)
        g = torch.from_numpy(img).to(dev)
        cells = torch.empty((ncell, 4), dtype=torch.int32, device=dev)
        hf = torch.from_numpy(img).pin_memory()
        hc = torch.empty((ncell, 4), dtype=torch.int32).pin_memory()
        dims = (vio.Dims * 1)(vio.Dims(w, h, w))
        fd = (ctypes.c_void_p * 1)(g.data_ptr())
        od = (ctypes.c_void_p * 1)(cells.data_ptr())
        fh = (ctypes.c_void_p * 1)(hf.data_ptr())
        oh = (ctypes.c_void_p * 1)(hc.data_ptr())
        res = {}
        for kind in ("device", "host"):
            ts = []
            for i in range(reps + 20):
                t0 = time.perf_counter()
                if kind == "device":
                    det.detect_ptrs(fd, dims, 1, thresh, 9, 32, levels, od, None, sh)
                    det.sync(stream)
                else:
                    det._check(det.lib.vio_detect_host(det.ctx, fh, dims, 1, thresh, 9, 32, levels, oh, None, sh))
                if i >= 20:
                    ts.append((time.perf_counter() - t0) * 1e6)
            res[kind] = {"p50_us": round(float(np.percentile(ts, 50)), 1),
                         "p99_us": round(float(np.percentile(ts, 99)), 1)}
        same = bool(np.array_equal(cells.cpu().numpy(), hc.numpy()))
        det.close()
        out[name] = {**res, "same_cells": same}
    out["what"] = ("one 752x480 frame per call, synchronised after every call (host clock): device-resident "
                   "(vio_detect + vio_sync) and host buffers (vio_detect_host, pinned frame in, pinned "
                   "records out); seed 0 at one level (thresh 10), seed 1 at three (thresh 20)")
    return out


def serving_leg(args, dev_index: int) -> dict:
    """Serving workload: 16 camera streams with Poisson arrivals at
    200 + 800 s/15 Hz (stream s), resolutions cycling through the four mixed
    sizes, 4 seeded frames per stream, 3 levels, FAST-9, thresh 15, 32x32
    cells, 4 GiB device budget.  Latency = submit -> cells in host memory.
    The same arrival schedule is replayed against a one-frame-per-launch
    server (1 lane, batch 1) for comparison."""
    import numpy as np
    import torch

    from paper_2003_13493_gb300 import synth, vio

    n_streams, per_stream, T = 16, 4, args.serve_seconds
    pools = []
    for s in range(n_streams):
        w, h = synth.MIXED_SIZES[s % 4]
        pools.append([torch.from_numpy(synth.make_frame(w, h, seed=5000 + 16 * s + j)).pin_memory()
                      for j in range(per_stream)])
    dims = [[vio.Dims(p.shape[1], p.shape[0], p.shape[1]) for p in pool] for pool in pools]
    rng = np.random.default_rng(4)
    events = []
    for s in range(n_streams):
        lam = 200.0 + 800.0 * s / (n_streams - 1)
        t = rng.exponential(1.0 / lam)
        j = 0
        while t < T:
            events.append((t, s, j % per_stream))
            t += rng.exponential(1.0 / lam)
            j += 1
    events.sort()

    def run(**kw):
        det = vio.Detector(device=dev_index, max_frames=max(64, kw.get("max_batch", 1)))
        det.serve_start(thresh=15, arc_len=9, cell_size=32, levels=3, keep_results=0,
                        mem_budget_bytes=4 << 30, queue_capacity=1 << 20, **kw)
        # warm the lanes (graphs, arenas) outside the measured window
        for s in range(n_streams):
            det.submit_raw(s, pools[s][0].data_ptr(), dims[s][0])
        det.drain(120000)
        det.serve_stop()
        det.serve_start(thresh=15, arc_len=9, cell_size=32, levels=3, keep_results=0,
                        mem_budget_bytes=4 << 30, queue_capacity=1 << 20, **kw)
        lag = 0.0
        rejected = 0
        # no garbage-collection pause inside the paced submission loop
        gc_was_on = gc.isenabled()
        gc.disable()
        t0 = time.perf_counter()
        for (t, s, j) in events:
            while True:
                now = time.perf_counter() - t0
                if now >= t:
                    break
            lag = max(lag, now - t)
            st, _ = det.submit_raw(s, pools[s][j].data_ptr(), dims[s][j])
            rejected += st != 0
        det.drain(600000)
        if gc_was_on:
            gc.enable()
        stats = det.serve_stats()
        det.serve_stop()
        det.close()
        stats["max_submit_lag_us"] = round(lag * 1e6, 1)
        stats["rejected"] = rejected
        return stats

    served = run(max_batch=32, lanes=3, max_wait_us=0)
    plain = run(max_batch=1, lanes=1, max_wait_us=0)
    offered = len(events) / T
    out = {"value": round(served["frames_per_s"], 1), "unit": "frames/s", "offered_fps": round(offered, 1),
           "frames": len(events), "p50_us": round(served["p50_us"], 1), "p99_us": round(served["p99_us"], 1),
           "max_us": round(served["max_us"], 1), "mean_batch": round(served["mean_batch"], 2),
           "max_batch_frames": int(served["max_batch_frames"]), "max_lanes_in_flight": int(served["max_lanes_in_flight"]),
           "overlapped_batches": int(served["overlapped_batches"]), "batches": int(served["batches"]),
           "max_submit_lag_us": served["max_submit_lag_us"], "lanes": 3, "max_batch": 32,
           "plain": {"value": round(plain["frames_per_s"], 1), "p50_us": round(plain["p50_us"], 1),
                     "p99_us": round(plain["p99_us"], 1), "max_us": round(plain["max_us"], 1),
                     "what": "same arrivals, one frame per launch on one lane"},
           "what": f"{n_streams} Poisson camera streams (200..1000 Hz) for {T:g} s, 4 GiB budget, "
                   "latency from submit to cells in host memory"}
    return out


def large4k_leg(args, dev_index: int) -> dict:
    """The 4K sweep workload (32 frames of 3840x2160, 4 levels, FAST-12 and
    FAST-9 at thresholds 5..40, 64x64 cells) timed like the main line: its own
    warm-up, timed steps on the device, clocks and the roofline of the fused
    sweep kernel.  The 265 MB batch is larger than L2."""
    import copy

    a = copy.copy(args)
    a.workload, a.cell, a.variant = "large4k", 0, -1
    a.steps, a.warmup, a.spin = max(4, min(args.steps, 12)), 3, 0.3
    a.no_extras, a.no_cpu_baseline, a.no_large4k = False, True, True
    r = run_ours(a, 0, 1, dev_index)
    keep = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "mpixel_per_s", "detections_per_s",
            "config", "clocks", "gpu_launches", "roofline", "stage_ms", "step_roofline")
    return {k: r[k] for k in keep if k in r}


def serving_saturation_leg(args, dev_index: int) -> dict:
    """The serving mix of serving_leg with its Poisson rates scaled up until
    one lane at one frame per launch saturates, and past it.  At each rate
    the batching server (3 lanes, up to 32 frames per launch) and the plain
    one (1 lane, 1 frame per launch) see the same arrivals; each run lasts
    `seconds` of arrivals (the plain server's backlog then drains)."""
    import numpy as np
    import torch

    from paper_2003_13493_gb300 import synth, vio

    n_streams, per_stream = 16, 4
    seconds = max(0.5, min(2.0, args.serve_seconds / 5))
    pools = []
    for s in range(n_streams):
        w, h = synth.MIXED_SIZES[s % 4]
        pools.append([torch.from_numpy(synth.make_frame(w, h, seed=5000 + 16 * s + j)).pin_memory()
                      for j in range(per_stream)])
    dims = [[vio.Dims(p.shape[1], p.shape[0], p.shape[1]) for p in pool] for pool in pools]
    ptrs = [[p.data_ptr() for p in pool] for pool in pools]

    def schedule(scale, seed):
        rng = np.random.default_rng(seed)
        ev = []
        for s in range(n_streams):
            lam = scale * (200.0 + 800.0 * s / (n_streams - 1))
            t = rng.exponential(1.0 / lam)
            j = 0
            while t < seconds:
                ev.append((t, s, j % per_stream))
                t += rng.exponential(1.0 / lam)
                j += 1
        ev.sort()
        return ev

    def run(events, **kw):
        det = vio.Detector(device=dev_index, max_frames=max(64, kw.get("max_batch", 1)))
        cfg = dict(thresh=15, arc_len=9, cell_size=32, levels=3, keep_results=0, mem_budget_bytes=4 << 30,
                   queue_capacity=1 << 22, **kw)
        det.serve_start(**cfg)
        for s in range(n_streams):
            det.submit_raw(s, ptrs[s][0], dims[s][0])
        det.drain(120000)
        det.serve_stop()
        det.serve_start(**cfg)
        lag = 0.0
        rejected = 0
        gc_was_on = gc.isenabled()
        gc.disable()
        t0 = time.perf_counter()
        for (t, s, j) in events:
            while True:
                now = time.perf_counter() - t0
                if now >= t:
                    break
            lag = max(lag, now - t)
            st, _ = det.submit_raw(s, ptrs[s][j], dims[s][j])
            rejected += st != 0
        det.drain(600000)
        if gc_was_on:
            gc.enable()
        st = det.serve_stats()
        det.serve_stop()
        det.close()
        return {"frames_per_s": round(st["frames_per_s"], 1), "p50_us": round(st["p50_us"], 1),
                "p99_us": round(st["p99_us"], 1), "mean_batch": round(st["mean_batch"], 2),
                "max_batch_frames": int(st["max_batch_frames"]), "max_lanes_in_flight": int(st["max_lanes_in_flight"]),
                "overlapped_batches": int(st["overlapped_batches"]), "batches": int(st["batches"]),
                "rejected": rejected, "max_submit_lag_us": round(lag * 1e6, 1)}

    points = []
    for scale in (1, 4, 16, 48):
        ev = schedule(scale, 40 + scale)
        offered = len(ev) / seconds
        served = run(ev, max_batch=32, lanes=3, max_wait_us=0)
        plain = run(ev, max_batch=1, lanes=1, max_wait_us=0)
        points.append({"rate_scale": scale, "offered_fps": round(offered, 1), "frames": len(ev),
                       "served": served, "plain": plain})
    return {"points": points, "seconds_of_arrivals": seconds,
            "what": "the 16-stream serving mix with every stream's Poisson rate multiplied by rate_scale; "
                    "served = 3 lanes, up to 32 frames per launch; plain = 1 lane, 1 frame per launch; "
                    "frames/s = completed frames / (last completion - first submit); latency from submit "
                    "to cells in host memory"}


def run_reference(args, rank, world):
    wl = dict(WORKLOADS[args.workload])
    if args.cell:
        wl["cell"] = args.cell
    frames = make_frames(args.workload)
    if rank != 0:
        return None
    import oracle

    oracle.build()
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps + args.warmup))
    for _ in range(max(0, args.warmup)):
        oracle_rate(frames, wl, 0.0)
    total = 0.0
    t0 = time.perf_counter()
    rates = []
    cores = sample = None
    for _ in range(args.steps):
        r, cores, sample = oracle_rate(frames, wl, per_step)
        rates.append(r)
    dt = time.perf_counter() - t0
    total = sum(rates) / len(rates)
    return {"metric": METRIC, "value": round(total, 2), "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded value noise + shapes, integer generator)", "impl": "reference",
            "config": {"workload": f"{args.workload}: {wl['desc']}", "frames_per_step": len(frames),
                       "detections_per_frame": len(wl.get("sweep") or [0]),
                       "mpixel_per_step": round(sum(f.size for f in frames) / 1e6, 3), "levels": wl["levels"],
                       "thresh": wl["thresh"], "arc_len": wl["arc"], "cell": wl["cell"], "score": "SAD-B"},
            "cpu_baseline": {"value": round(total, 2), "unit": "frames/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(total, 2), "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.tracker_only:
        import torch

        torch.cuda.set_device(local_rank)
        print(json.dumps({"tracker": tracker_leg(args, local_rank)}))
        return
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res))
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
