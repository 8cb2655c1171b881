#!/usr/bin/env python3
"""Throughput of the EVIS event-synthesis hot path on B300.

Headline workload (default): the high-speed batch, the largest configuration that fits one
GPU.  1024 environments at 640x480, K = 32 sub-frames per keyframe gap (8 ms), C = 0.15, five
depth layers of seeded textured disks moving up to 40 px per keyframe (about 10 % of the
target-sub-frames have a disocclusion hole in one warp direction or the other; the line's
`holes` key measures it), fp32 log-intensity inputs, no refractory period.  Synthetic scenes, no dataset.

One step = one keyframe gap of every environment: the input-preparation kernel (motion
bounds, per-source packs) and the synthesis kernel (bidirectional splat, z-buffer, blend,
threshold crossings, event compaction), on keyframes already resident in HBM.  Metric:
Mpixel-substeps/s (sum over environments of H * W * K per step / time); events/s beside it.

The same JSON line carries, as extra keys: the 64-environment 346x260 workload with linear
inputs and a refractory period ("config2"), the uneven 256-environment batch run as one
context per environment, as one batched step and as an autotuned graph replay ("config3"),
and the differentiable surrogate ("soft_surrogate").

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl evis|reference]

Under torchrun each rank runs its own 1024 environments (disjoint seeds, no data exchange:
weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixel-substeps/s"
UNIT = "Mpx-substeps/s"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["evis", "reference"], default="evis")
    ap.add_argument("--workload", choices=["highspeed", "envs64", "batched", "stages", "soft"],
                    default="highspeed",
                    help="highspeed: the headline line (1024 envs at 640x480, K=32) with the "
                         "other workloads as extra keys; envs64: the 64-env 346x260 line alone; "
                         "batched: the uneven 256-env batch alone; stages: sensor noise, colour, "
                         "margin, defocus and the voxel grid; soft: the differentiable surrogate")
    ap.add_argument("--hs-envs", type=int, default=1024,
                    help="environments of the high-speed workload (640x480, K=32)")
    ap.add_argument("--envs", type=int, default=64, help="environments of the 346x260 workload")
    ap.add_argument("--e2e-steps", type=int, default=6)
    ap.add_argument("--e2e-slices", type=int, default=4,
                    help="contexts (one stream each) the end-to-end leg splits the "
                         "environments into")
    ap.add_argument("--tile", default=None,
                    help="WxH: fixed tile shape instead of the autotuner's (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline line only (no config2 / config3 / soft_surrogate keys)")
    ap.add_argument("--stage", choices=["all", "synthesis", "defocus", "voxel"], default="all",
                    help="with --workload stages: the part to run")
    ap.add_argument("--voxel-envs", type=int, default=8,
                    help="environments (640x480) of the voxel-grid stage")
    return ap.parse_args()


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------------------------------
# workloads and their byte models
# ------------------------------------------------------------------------------------------

def highspeed_workload(n_envs, rank=0):
    import scenes
    return scenes.config4(n_envs=n_envs, first_env=rank * n_envs)


def highspeed_config(w, n_envs):
    e = w.envs[0]
    return {"workload": f"high-speed batch: {n_envs} envs at {e.W}x{e.H}, K={e.K}, C={e.c_on}, "
                        "5 depth layers, flows up to 40 px per keyframe (~10 % of target-sub-frames with a hole in one direction), "
                        "log-intensity inputs, no refractory period",
            "envs": n_envs, "width": e.W, "height": e.H, "K": e.K, "C": e.c_on,
            "refractory_ns": 0, "dt_ns": w.dt_ns, "input": "log intensity, fp32",
            "pixel_substeps_per_step": w.pixel_substeps,
            "l2": "each step reads a fresh 5 GB keyframe (inputs far larger than the 126 MB L2); "
                  "a 256 MB L2 flush runs between timed steps as well"}


def config2_workload(n_envs, rank=0):
    import scenes
    return scenes.config2(n_envs=n_envs, first_env=rank * n_envs)


def config2_config(w, n_envs):
    return {"workload": f"{n_envs} envs at 346x260, K=16, C=0.25, refractory 100us, "
                        "3 depth layers, linear-radiance inputs",
            "envs": n_envs, "width": 346, "height": 260, "K": 16, "C": 0.25,
            "refractory_ns": 100_000, "dt_ns": w.dt_ns, "input": "linear luminance (log on path)",
            "pixel_substeps_per_step": w.pixel_substeps,
            "l2": "flushed between timed steps (256 MB write); each step also reads a fresh keyframe"}


def algorithmic_bytes(envs, n_events):
    """Bytes the method must move for one keyframe gap of envs (per pixel: keyframes A and B,
    2 x (4 L + 8 mv + 4 Z) = 32 B; the reference level read and written, 8 B; the last-event
    time read and written, 16 B, where a refractory period is set; the two threshold maps,
    8 B, where they are per pixel) plus 16 B per event written."""
    b = 0
    for e in envs:
        per_px = 32 + 8
        if e.refractory_ns > 0:
            per_px += 16
        if getattr(e, "c_on_map", None) is not None:
            per_px += 8
        b += e.W * e.H * per_px
    return b + 16 * n_events


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "20",
                                       "-i", str(device_index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------------------
# peaks and committed profile records
# ------------------------------------------------------------------------------------------

def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


def traffic_record(workload_key):
    """ncu figures per launch of the synthesis kernel for one workload (DRAM bytes, warp
    instructions), if profiles/step_kernel_traffic.json holds a capture of the current kernel
    source, else None."""
    p = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    src = os.path.join(ROOT, "paper_2607_08098_b300", "csrc", "evis_step.cuh")
    try:
        rec = json.load(open(p))
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if rec.get("kernel_sha256") == h:
            return rec.get("workloads", {}).get(workload_key)
    except (OSError, ValueError):
        pass
    return None


def roofline_block(envs, n_events_per_step, syn_ms, prep_ms, shapes, tuned_ms, workload_key,
                   clk, sms):
    """The synthesis kernel against HBM (algorithmic bytes / its mean CUDA-event duration)
    and against instruction issue (its captured warp instructions / duration)."""
    peak, peak_kind = measured_peak()
    alg = algorithmic_bytes(envs, n_events_per_step)
    achieved = alg / (syn_ms / 1e3) / 1e9
    tr = traffic_record(workload_key)
    r = {"kernel": "step_kernel (splat + z-buffer + blend + crossings + compaction)",
         "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
         "frac": achieved / peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
         "traffic": None if tr is None else tr["dram_bytes_per_launch"],
         "algorithmic_bytes_per_launch": alg, "kernel_ms": syn_ms, "prep_ms": prep_ms,
         "tile_shape": shapes, "autotune_best_ms": tuned_ms,
         "nominal_peak": 7700.0, "frac_of_nominal": achieved / 7700.0}
    if tr is not None:
        dram = tr["dram_bytes_per_launch"] / (syn_ms / 1e3) / 1e9
        r["dram"] = {"achieved": dram, "frac": dram / peak, "unit": "GB/s",
                     "source": tr.get("source", "ncu dram__bytes_read.sum + dram__bytes_write.sum")}
        if "warp_instructions_per_launch" in tr:
            # the kernel's real ceiling: instruction issue, 4 schedulers per SM, one warp
            # instruction per clock each, at the SM clock sampled during the timed region
            mhz = clk.get("sm_mhz") or 2032.0
            peak_issue = sms * 4 * mhz * 1e6
            ach = tr["warp_instructions_per_launch"] / (syn_ms / 1e3)
            r["issue"] = {"bound": "instruction issue", "achieved_warp_inst_per_s": ach,
                          "peak_warp_inst_per_s": peak_issue, "frac": ach / peak_issue,
                          "sm_mhz": mhz, "nominal_peak_warp_inst_per_s": sms * 4 * 2.032e9,
                          "warp_instructions_per_pixel_substep":
                              tr.get("warp_instructions_per_pixel_substep"),
                          "source": "ncu smsp__inst_executed.sum of the committed capture"}
    return r


# ------------------------------------------------------------------------------------------
# device-timed keyframe gaps
# ------------------------------------------------------------------------------------------

def upload_keyframes(w, n_kf, frame_key, world=1):
    """Renders keyframes 0..n_kf-1 (host) and keeps them on the device: (frames, mv, depth).
    Under several ranks on one host each renders with its share of the host's cores."""
    import scenes
    import torch
    threads = max(1, (os.cpu_count() or 1) // max(world, 1))
    dev = []
    for k in range(n_kf):
        kf = scenes.render(w.envs, k, want=(frame_key, "mv", "Z"), threads=threads)
        dev.append(tuple(torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()
                         for a in (getattr(kf, frame_key), kf.mv, kf.Z)))
        del kf
    return dev


def timed_gaps(ev, w, dev, flags, steps, warmup, dist=None, reps_autotune=1, tile=None):
    """Context over w.envs fed dev[0] (reference levels), autotuned on dev[1], warmed up on
    dev[1..warmup], then `steps` timed gaps dev[warmup+1..], each bracketed by CUDA events on
    the context's stream after an L2 flush and an event-buffer clear (the events of a gap
    stay in the buffer until the next gap).  Returns the per-step figures."""
    import torch
    probe = ev.Context(w.envs, eps=1e-4, flags=flags, capacity=1 << 20)
    probe.step(*dev[0], w.dt_ns)
    probe.step(*dev[1], w.dt_ns)
    per_gap = probe.event_count()          # counted beyond the buffer too
    probe.close()
    # later gaps of the moving scenes carry more events than the first (up to ~1.4x over 25
    # gaps of the high-speed batch): room for twice the first gap's
    capacity = int(per_gap * 2.0) + (1 << 20)
    ctx = ev.Context(w.envs, eps=1e-4, flags=flags, capacity=capacity)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    ctx.step(*dev[0], w.dt_ns)
    if tile:
        ctx.set_tile_shape(*(int(v) for v in tile.split("x")))
        tuned_ms = None
    else:
        tuned_ms = ctx.autotune(*dev[1], w.dt_ns, reps=reps_autotune)
    shapes = ctx.tile_shapes()
    for k in range(1, 1 + warmup):
        ctx.clear_events()
        ctx.step(*dev[k], w.dt_ns)
    torch.cuda.synchronize()
    ctx.profile(steps)
    st = torch.cuda.current_stream()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms, events = [], []
    wall0 = time.perf_counter()
    for s_ in range(steps):
        ctx.clear_events()
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        ctx.step(*dev[1 + warmup + s_], w.dt_ns)
        b.record(st)
        b.synchronize()
        ms.append(a.elapsed_time(b))
        n = ctx.event_count()
        if n > capacity:
            raise RuntimeError("event buffer overflow in the timed region")
        events.append(n)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - wall0
    prof = ctx.profile_read()
    ctx.close()
    classes = {}
    for e, sh in zip(w.envs, shapes):
        classes.setdefault(f"{e.W}x{e.H}", f"{sh[0]}x{sh[1]}")
    return {"step_ms": ms, "events": events, "syn_ms": float(prof[:, 1].mean()),
            "prep_ms": float(prof[:, 0].mean()), "shapes": classes, "tuned_ms": tuned_ms,
            "capacity": capacity, "per_gap_probe": per_gap, "wall_s": wall}


def reduce_over_ranks(total_ms, units, events, device):
    """Whole-job figures of a weak-scaling run: the slowest rank's time and the units and
    events summed over ranks (timing only; ranks exchange no data of the path)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms), float(units), float(events)], device=device,
                     dtype=torch.float64)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1]), float(sm[2])


def host_mem_available():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


def hole_fraction_leg(ev, w, dev, n_sample=16, gaps=2):
    """Disocclusion holes of the workload (Sec. 3.3, the blend's hole filling): the first
    n_sample environments over `gaps` keyframe gaps in a context with EVIS_STATS, as fractions
    of their target-sub-frames with no source of A, of B, of both, and of at least one."""
    import torch
    n_px = sum(e.H * e.W for e in w.envs[:n_sample])   # equal sizes: no packing pads between
    ctx = ev.Context(w.envs[:n_sample], flags=ev.IN_LOG | ev.KEEP_INPUTS | ev.STATS,
                     capacity=1 << 27)
    for k in range(gaps + 1):
        L, mv, Z = dev[k]
        ctx.step(L[:n_px], mv[:2 * n_px], Z[:n_px], w.dt_ns)
    st = ctx.env_stats()
    ctx.close()
    torch.cuda.synchronize()
    tot = float(st["target_subframes"].sum())
    a, b, both = (float(st[f].sum()) for f in ("holes_a", "holes_b", "holes_both"))
    return {"sample": f"environments 0-{n_sample - 1}, {gaps} keyframe gaps",
            "target_subframes": int(tot), "no_source_of_A": a / tot, "no_source_of_B": b / tot,
            "no_source_of_either": both / tot, "at_least_one_direction": (a + b - both) / tot}


def link_rates(nbytes=1 << 30, reps=3):
    """Host<->device copy rates of this GPU's link with pinned host memory (GB/s, best of
    reps): host to device alone, device to host alone, and both at once on two streams
    (their sum)."""
    import torch
    d0 = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    d1 = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    h0 = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h1 = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    s0, s1 = torch.cuda.Stream(), torch.cuda.Stream()

    def best(fn):
        t = float("inf")
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            t = min(t, time.perf_counter() - t0)
        return t

    def both():
        with torch.cuda.stream(s0):
            d0.copy_(h0, non_blocking=True)
        with torch.cuda.stream(s1):
            h1.copy_(d1, non_blocking=True)

    out = {"h2d_gbs": nbytes / best(lambda: d0.copy_(h0, non_blocking=True)) / 1e9,
           "d2h_gbs": nbytes / best(lambda: h1.copy_(d1, non_blocking=True)) / 1e9,
           "both_gbs": 2 * nbytes / best(both) / 1e9}
    del d0, d1, h0, h1
    torch.cuda.empty_cache()
    return out


def link_floor_ms(h2d_bytes, d2h_bytes, rates):
    """Least time the link needs for one step's copies: each direction at most at its own
    rate, both together at most at their summed rate."""
    return 1e3 * max(h2d_bytes / (rates["h2d_gbs"] * 1e9), d2h_bytes / (rates["d2h_gbs"] * 1e9),
                     (h2d_bytes + d2h_bytes) / (rates["both_gbs"] * 1e9))


def slice_plan(n_env, slices, capacity):
    """Consecutive environment slices for the end-to-end leg: the cut points (slice q holds
    environments cut[q] .. cut[q+1]-1) and each slice's event capacity.  A slice's buffer is
    its share of the whole launch's capacity with a margin for an uneven split of the events,
    growing as the slice holds fewer environments (their counts differ from scene to scene),
    and never more than the whole capacity."""
    S = max(1, min(slices, n_env))
    cut = [n_env * q // S for q in range(S + 1)]
    if S == 1:
        return cut, [capacity]
    caps = []
    for q in range(S):
        m = cut[q + 1] - cut[q]
        caps.append(min(capacity, int(capacity * m / n_env * (1.2 + 2.0 / m ** 0.5)) + 4096))
    return cut, caps


def slice_planes(planes, px, lo_env, hi_env):
    """Views of packed per-pixel planes (each a flat array of total pixels x its per-pixel
    width, px the pixel prefix sums over environments) restricted to environments
    lo_env .. hi_env-1."""
    total = int(px[-1])
    lo, hi = int(px[lo_env]), int(px[hi_env])
    return tuple(t[lo * (t.numel() // total):hi * (t.numel() // total)] for t in planes)


def e2e_leg(ev, w, dev, n_steps, capacity, flags_host, dist=None, world=1, shapes=None,
            slices=4):
    """Host buffers in, events out, through the public API: pinned host keyframes copied by
    evis_step_host, every gap's events copied to pinned host memory by
    evis_read_events_async, all inside the timed region.

    The environments are split into `slices` contexts, each on its own stream with its own
    event buffers.  A context's synthesis launch is persistent (one wave of resident CTAs),
    so the slices' launches take the GPU in turn.  As soon as a slice is done, the read-back
    of its events starts and its next gap is enqueued: both copies run while the later
    slices compute, and the next gap's launch is ready when they finish.  In one context the
    whole gap's read-back waited for its last tile, and the next keyframe's copy for the
    read-back.  The copy of a slice's gap completes before that slice's next read-back
    starts, so one destination buffer per slice serves.

    Six gaps by default: with two, filling and draining the pipeline (the first gap's input
    copy and compute, the last gap's read-back) was a third of the time.  Each rank pins at
    most 0.6 of the host's available memory divided by the number of ranks (so the ranks of
    one host never pin more than 0.6 of it between them) and the ranks agree on the number
    of gaps, or on skipping; under several ranks the figures are whole-job (the slowest
    rank's time, work and bytes summed).  The contexts take the tile shapes of the timed
    leg (per resolution class); the host link's copy rates, measured beside it, give the
    least time per step that the step's copies need."""
    import torch
    kf = sum(t.numel() * 4 for t in dev[0])
    n_env = len(w.envs) if w is not None else 1
    cut, cap = slice_plan(n_env, slices, capacity)
    S = len(cap)
    out_bytes = sum(cap) * 16
    avail = host_mem_available()
    n = n_steps
    if avail is not None:
        n = min(n, int((0.6 * avail / world - out_bytes) // kf) - 1)
    n = max(n, 0)
    if dist:
        t = torch.tensor([n], device="cuda", dtype=torch.int64)
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        n = int(t.item())
    if n < 1:
        return {"skipped": f"two keyframes ({2 * kf / 2**30:.0f} GiB) and the event buffers "
                           f"({out_bytes / 2**30:.0f} GiB) of pinned host memory per rank do not "
                           f"fit 0.6 of the {(avail or 0) / 2**30:.0f} GiB available over {world} ranks"}
    px = np.cumsum([0] + [e.W * e.H for e in w.envs])
    host = [tuple(t.cpu().pin_memory() for t in dev[k]) for k in range(n + 1)]

    def part(k, q):   # slice q of keyframe k: views of the packed host planes
        return slice_planes(host[k], px, cut[q], cut[q + 1])

    outs = [torch.empty(c * 16, dtype=torch.uint8).pin_memory() for c in cap]
    streams = [torch.cuda.Stream() for _ in range(S)]
    ctxs = [ev.Context(w.envs[cut[q]:cut[q + 1]], eps=1e-4, flags=flags_host, capacity=cap[q],
                       stream=streams[q]) for q in range(S)]
    cnt = ctypes.c_int64()
    L = ev.lib()
    for q, ctx in enumerate(ctxs):
        if shapes:
            ctx.set_env_tile_shapes([tuple(int(v) for v in shapes[f"{e.W}x{e.H}"].split("x"))
                                     for e in w.envs[cut[q]:cut[q + 1]]])
        ctx.step_host(*part(0, q), w.dt_ns)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    d2h = 0
    t0 = time.perf_counter()
    for q, ctx in enumerate(ctxs):
        ctx.step_host(*part(1, q), w.dt_ns)
    for k in range(1, n + 1):
        for q, ctx in enumerate(ctxs):
            # slice q's gap k is done: its read-back starts, and its next gap is enqueued
            # (the input copy then runs while the other slices compute)
            st = L.evis_read_events_async(ctx.handle, outs[q].data_ptr(), cap[q], ctypes.byref(cnt))
            if st != ev.OK:
                raise RuntimeError(f"event read-back: {ev.status_string(st)}")
            d2h += cnt.value * 16 + 16
            if k < n:
                ctx.step_host(*part(k + 1, q), w.dt_ns)
    for ctx in ctxs:
        ctx.read_wait()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    for ctx in ctxs:
        ctx.close()
    del host, outs
    torch.cuda.empty_cache()
    rates = link_rates()
    floor = link_floor_ms(kf, d2h / n, rates)
    units = w.pixel_substeps * n
    ms_rank = ms
    if dist:
        ms, units, d2h = reduce_over_ranks(ms, units, d2h, "cuda")
    return {"value": units / (ms / 1e3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": kf * world,
            "d2h_bytes_per_step": int(d2h) // n, "steps": n, "slices": S,
            "link": dict({k: round(v, 2) for k, v in rates.items()},
                         floor_ms_per_step=round(floor, 2), ms_per_step=round(ms_rank / n, 2),
                         frac=round(floor / (ms_rank / n), 3),
                         note="this rank's link, measured after the leg with 1 GiB pinned "
                              "copies; floor = the step's copies alone at those rates"),
            "path": f"{S} contexts over consecutive environment slices, one stream each: "
                    "evis_step_host (pinned host keyframe -> device) + evis_read_events_async "
                    "(every event -> pinned host, copied while the later slices and the next "
                    "gap run); each slice's next gap enqueued as soon as its gap is done; host "
                    "wall clock over the steps"}


# ------------------------------------------------------------------------------------------
# the oracle: CPU baseline, reference arm, and the parity sample of the benchmarked launch
# ------------------------------------------------------------------------------------------

def _events_of_envs_on_device(ev, ctx, env_ids):
    """Drains the context's events into device memory and returns, on the host, those of
    the given environments (the filter runs on the device)."""
    import torch
    n = ctx.event_count()
    buf = torch.empty((max(n, 1), 2), dtype=torch.int64, device="cuda")
    cnt = ctypes.c_int64()
    st = ev.lib().evis_read_events(ctx.handle, buf.data_ptr(), n, ctypes.byref(cnt))
    if st != ev.OK:
        raise RuntimeError(f"read: {ev.status_string(st)}")
    words = buf[:cnt.value]
    env = (words[:, 1] >> 32) & 0xFFFF
    keep = torch.isin(env, torch.tensor(env_ids, device="cuda"))
    sel = words[keep].cpu().numpy()
    del buf
    return sel.view(ev.EVENT_DTYPE).reshape(-1), cnt.value


def parity_and_cpu_baseline(ev, w, dev, shapes, sample_ids, gaps):
    """The oracle (single thread) on a bounded sample of the benchmarked workload: the
    environments sample_ids for `gaps` keyframe gaps.  Its time is the CPU baseline; its
    events and reference levels are compared bit for bit with those environments' share of
    a full launch of the library over every environment (the autotuned tile shapes)."""
    import oracle
    import scenes
    import torch
    sub = [w.envs[i] for i in sample_ids]
    o = oracle.Oracle(sub, eps=1e-4, flags=oracle.IN_LOG)
    kfs = [scenes.render(sub, k, want=("L", "mv", "Z")) for k in range(gaps + 1)]
    o.step(kfs[0].L, kfs[0].mv, kfs[0].Z, w.dt_ns)
    t0 = time.perf_counter()
    for kf in kfs[1:]:
        o.step(kf.L, kf.mv, kf.Z, w.dt_ns)
    sec = time.perf_counter() - t0
    want = oracle.sort_events(o.events())
    Lref_o = o.state()[0]

    cap = int(w.pixel_substeps * 0.15) + (1 << 20)
    ctx = ev.Context(w.envs, eps=1e-4, flags=ev.IN_LOG | ev.KEEP_INPUTS, capacity=cap)
    tw = [int(shapes[f"{e.W}x{e.H}"].split("x")[0]) for e in w.envs]
    th = [int(shapes[f"{e.W}x{e.H}"].split("x")[1]) for e in w.envs]
    ctx.set_env_tile_shapes(list(zip(tw, th)))
    ctx.step(*dev[0], w.dt_ns)
    got, total = [], 0
    for k in range(1, gaps + 1):
        ctx.step(*dev[k], w.dt_ns)
        sel, n = _events_of_envs_on_device(ev, ctx, sample_ids)
        got.append(sel)
        total += n
    Lref_g = ctx.state()[0]
    ctx.close()
    torch.cuda.synchronize()
    got = np.concatenate(got)
    remap = np.zeros(max(sample_ids) + 1, dtype=np.uint16)
    remap[sample_ids] = np.arange(len(sample_ids), dtype=np.uint16)
    got["env"] = remap[got["env"]]
    got = oracle.sort_events(got)
    same_events = len(got) == len(want) and np.array_equal(got.view(np.uint8), want.view(np.uint8))
    off_g = np.concatenate([[0], np.cumsum([(e.W * e.H + 3) // 4 * 4 for e in w.envs])])
    same_lref = True
    oo = 0
    for i, e in zip(sample_ids, sub):
        n = e.W * e.H
        same_lref &= np.array_equal(Lref_g[off_g[i]:off_g[i] + n], Lref_o[oo:oo + n])
        oo += (n + 3) // 4 * 4
    units = sum(e.W * e.H * e.K for e in sub) * gaps
    cpu = {"value": units / sec / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"environments {sample_ids} of the {len(w.envs)} (their own scenes, "
                     f"{sub[0].W}x{sub[0].H}, K={sub[0].K}) for {gaps} keyframe gaps, "
                     "single-threaded C++ oracle", "seconds": sec,
           "events_per_s": len(want) / sec}
    parity = {"envs": list(sample_ids), "gaps": gaps, "launch": f"all {len(w.envs)} environments",
              "events_compared": int(len(want)), "events_in_launch": int(total),
              "events_bit_exact": bool(same_events), "lref_bit_exact": bool(same_lref)}
    return cpu, parity


def oracle_parallel_rate(w, threads):
    """Env-parallel CPU baseline: one single-threaded oracle per host thread, each on its own
    environment of w for one keyframe gap, all at the same time (the oracle's C calls release
    the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    import scenes
    work = []
    for t in range(threads):
        e = w.envs[t % len(w.envs)]
        kfs = [scenes.render([e], k, want=("L", "mv", "Z")) for k in range(2)]
        o = oracle.Oracle([e], eps=1e-4, flags=oracle.IN_LOG)
        o.step(kfs[0].L, kfs[0].mv, kfs[0].Z, w.dt_ns)
        work.append((o, kfs[1], e))

    def run(item):
        o, kf, _ = item
        o.step(kf.L, kf.mv, kf.Z, w.dt_ns)

    with ThreadPoolExecutor(max_workers=threads) as pool:
        t0 = time.perf_counter()
        list(pool.map(run, work))
        sec = time.perf_counter() - t0
    units = sum(e.W * e.H * e.K for _, _, e in work)
    return {"value": units / sec / 1e6, "unit": UNIT, "cores": threads,
            "kind": "oracle, env-parallel", "seconds": sec,
            "sample": f"{threads} threads, each the single-threaded C++ oracle on one "
                      "environment for one keyframe gap"}


def reference_arm(args, world, rank):
    """The oracle as it stands, on the host cores, for the headline workload: each step is
    one keyframe gap of one environment (a bounded sample: environment 0, gap after gap)."""
    if rank != 0:
        return
    import oracle
    import scenes
    w = highspeed_workload(args.hs_envs)
    n_kf = args.warmup + args.steps + 1
    e = w.envs[0]
    kfs = [scenes.render([e], k, want=("L", "mv", "Z")) for k in range(n_kf)]
    o = oracle.Oracle([e], eps=1e-4, flags=oracle.IN_LOG)
    o.step(kfs[0].L, kfs[0].mv, kfs[0].Z, w.dt_ns)
    for kf in kfs[1:1 + args.warmup]:
        o.step(kf.L, kf.mv, kf.Z, w.dt_ns)
    o.events()
    t0 = time.perf_counter()
    for kf in kfs[1 + args.warmup:]:
        o.step(kf.L, kf.mv, kf.Z, w.dt_ns)
    sec = time.perf_counter() - t0
    nev = len(o.events())
    units = e.W * e.H * e.K * args.steps
    value = units / sec / 1e6
    sample = (f"each step: environment 0 of the {args.hs_envs} ({e.W}x{e.H}, K={e.K}) for its next "
              "keyframe gap, single-threaded C++ oracle")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": highspeed_config(w, args.hs_envs),
            "events_per_s": nev / sec,
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": sample, "value": value,
                             "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# the CUDA path
# ------------------------------------------------------------------------------------------

def headline_arm(args, world, rank, local):
    import torch
    import paper_2607_08098_b300 as ev

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = highspeed_workload(args.hs_envs, rank)
    n_kf = max(args.warmup + args.steps + 1, 4)
    dev = upload_keyframes(w, n_kf, "L", world)
    flags = ev.IN_LOG | ev.KEEP_INPUTS
    clocks = ClockSampler(local)            # sampled from the autotuner and warm-up on
    r = timed_gaps(ev, w, dev, flags, args.steps, args.warmup, dist=dist, tile=args.tile)
    clk = clocks.stop()
    total_ms = float(sum(r["step_ms"]))
    n_events = int(sum(r["events"]))
    units = w.pixel_substeps * args.steps
    if dist:
        total_ms, units, n_events = reduce_over_ranks(total_ms, units, n_events, "cuda")
    value = units / (total_ms / 1e3) / 1e6
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roof = roofline_block(w.envs, sum(r["events"]) / args.steps, r["syn_ms"], r["prep_ms"],
                          r["shapes"], r["tuned_ms"], "highspeed_1024x640x480_K32"
                          if args.hs_envs == 1024 else f"highspeed_{args.hs_envs}x640x480_K32",
                          clk, sms)
    holes = hole_fraction_leg(ev, w, dev) if rank == 0 else None
    keep = max(4, args.e2e_steps + 1)
    del dev[keep:]                          # the legs below need the first keyframes only
    torch.cuda.empty_cache()
    e2e = None
    if args.e2e_steps > 0:
        # the read-back empties the buffer every gap: room for the largest gap seen, and more
        cap_e2e = min(r["capacity"], int(1.3 * max(r["events"])) + 4096)
        e2e = e2e_leg(ev, w, dev, args.e2e_steps, cap_e2e, ev.IN_LOG, dist, world, r["shapes"],
                      args.e2e_slices)
    cpu = cpu_par = parity = None
    if world == 1 and not args.no_cpu_baseline:
        n = len(w.envs)
        ids = sorted({0, max(0, n // 2 - 1), n - 1})
        cpu, parity = parity_and_cpu_baseline(ev, w, dev, r["shapes"], ids, gaps=3)
        cpu_par = oracle_parallel_rate(w, os.cpu_count() or 1)
    del dev
    torch.cuda.empty_cache()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded layered scenes; the paper's scenes are not available)",
            "config": highspeed_config(w, args.hs_envs), "events_per_s": n_events / (total_ms / 1e3),
            "events_per_step": n_events / args.steps / max(world, 1), "step_ms": r["step_ms"],
            "wall_s": r["wall_s"], "roofline": roof, "cpu_baseline": cpu,
            "cpu_baseline_parallel": cpu_par, "parity": parity, "e2e": e2e,
            "gpu_launches": 2 * args.steps, "clocks": clk, "holes": holes,
            "parallelism": f"env shards x{world}, no collective on the data path"}
    if world == 1 and not args.no_extras:
        line["config2"] = config2_leg(ev, args)
        line["config3"] = config3_leg(ev, args)
        line["soft_surrogate"] = soft_leg()
    print(json.dumps(line), flush=True)


def config2_leg(ev, args, world=1, rank=0, dist=None):
    """The 64-environment 346x260 workload (K=16, refractory 100 us, linear luminance with
    the log on the path): device-timed gaps and the roofline of its synthesis kernel."""
    import torch
    w = config2_workload(args.envs, rank)
    steps = args.steps
    dev = upload_keyframes(w, args.warmup + steps + 1, "I", world)
    clocks = ClockSampler(torch.cuda.current_device())
    r = timed_gaps(ev, w, dev, ev.IN_LUM | ev.KEEP_INPUTS, steps, args.warmup, dist=dist,
                   reps_autotune=2, tile=args.tile)
    clk = clocks.stop()
    e2e = None
    if args.e2e_steps > 0:  # the same sliced host pipeline as the headline's
        cap_e2e = min(r["capacity"], int(1.3 * max(r["events"])) + 4096)
        e2e = e2e_leg(ev, w, dev, args.e2e_steps, cap_e2e, ev.IN_LUM, dist, world, r["shapes"],
                      args.e2e_slices)
    del dev
    torch.cuda.empty_cache()
    total_ms = float(sum(r["step_ms"]))
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out = {"config": config2_config(w, args.envs), "metric": METRIC, "unit": UNIT,
           "value": w.pixel_substeps * steps / (total_ms / 1e3) / 1e6,
           "ms_per_step": total_ms / steps, "events_per_step": sum(r["events"]) / steps,
           "events_per_s": sum(r["events"]) / (total_ms / 1e3), "steps": steps,
           "roofline": roofline_block(w.envs, sum(r["events"]) / steps, r["syn_ms"], r["prep_ms"],
                                      r["shapes"], r["tuned_ms"], f"config2_{args.envs}x346x260_K16",
                                      clk, sms),
           "clocks": clk, "e2e": e2e}
    return out


def config3_leg(ev, args):
    """The uneven 256-environment batch (128x128, 346x260, 640x480, 1280x720 in 4:2:1:1, K ~
    U{4..32}, per-pixel thresholds, linear inputs): the same keyframe gaps run (a) as one
    context per environment, (b) as one batched context with evis_step, (c) autotuned and
    replayed from a captured CUDA graph.  Device time of the timed steps."""
    import torch
    import scenes
    w = scenes.config3()
    steps = min(args.steps, 5)
    warmup = args.warmup
    n_kf = warmup + steps + 1
    off, total = scenes.pixel_offsets(w.envs)
    dev = upload_keyframes(w, n_kf, "I")
    units = w.pixel_substeps
    cap_env = [int(e.H * e.W * e.K * 1.7) + 4096 for e in w.envs]  # ~1.4 events per px-substep
    stream = torch.cuda.Stream()
    res = {}
    with torch.cuda.stream(stream):
        ctxs = [ev.Context([e], eps=1e-4, flags=ev.IN_LUM | ev.KEEP_INPUTS, capacity=c,
                           stream=stream) for e, c in zip(w.envs, cap_env)]

        def views(k, i):
            e, o = w.envs[i], int(off[i])
            n = e.H * e.W
            I, mv, Z = dev[k]
            return I[o:o + n], mv[2 * o:2 * (o + n)], Z[o:o + n]

        def run_per_env(k):
            for i, c in enumerate(ctxs):
                c.clear_events()
                c.step(*views(k, i), w.dt_ns)

        def timed(fn, first):
            t = 0.0
            for k in range(first, first + steps):
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                fn(k, prepare=True)
                a_.record(stream)
                fn(k, prepare=False)
                b_.record(stream)
                b_.synchronize()
                t += a_.elapsed_time(b_)
            return t

        run_per_env(0)
        for k in range(1, 1 + warmup):
            run_per_env(k)
        res["per_env_contexts"] = timed(lambda k, prepare: None if prepare else run_per_env(k),
                                        1 + warmup)
        for c in ctxs:
            c.close()
        big = ev.Context(w.envs, eps=1e-4, flags=ev.IN_LUM | ev.KEEP_INPUTS,
                         capacity=sum(cap_env), stream=stream)

        def run_big(k, prepare):
            if prepare:
                big.clear_events()
            else:
                big.step(*dev[k], w.dt_ns)

        big.step(*dev[0], w.dt_ns)
        for k in range(1, 1 + warmup):
            run_big(k, True)
            run_big(k, False)
        res["batched_step"] = timed(run_big, 1 + warmup)
        big.close()
        graph = ev.Context(w.envs, eps=1e-4, flags=ev.IN_LUM, capacity=sum(cap_env), stream=stream)
        graph.step(*dev[0], w.dt_ns)
        best = graph.autotune(*dev[1], w.dt_ns, reps=2)
        shapes = graph.tile_shapes()
        for k in range(1, 1 + warmup):
            graph.step(*dev[k], w.dt_ns)
        graph.capture(w.dt_ns)

        def run_graph(k, prepare):
            if prepare:
                graph.clear_events()
                graph.write_inputs(*dev[k])
            else:
                graph.replay()

        res["batched_graph_autotuned"] = timed(run_graph, 1 + warmup)
        n_events = graph.event_count()
        graph.close()
    del dev
    torch.cuda.empty_cache()
    classes = {}
    for e, sh in zip(w.envs, shapes):
        classes[f"{e.W}x{e.H}"] = f"{sh[0]}x{sh[1]}"
    vals = {k: units * steps / (v / 1e3) / 1e6 for k, v in res.items()}
    return {"workload": "batched uneven: 256 envs (128x128, 346x260, 640x480, 1280x720 in "
                        "4:2:1:1), K~U{4..32}, per-pixel C, linear inputs",
            "metric": METRIC, "unit": UNIT, "steps": steps, "warmup": warmup,
            "pixel_substeps_per_step": units, "value": vals,
            "ms_per_step": {k: v / steps for k, v in res.items()},
            "batched_over_per_env": vals["batched_step"] / vals["per_env_contexts"],
            "graph_over_per_env": vals["batched_graph_autotuned"] / vals["per_env_contexts"],
            "events_last_step": n_events, "event_buffer_overflow": n_events > sum(cap_env),
            "autotuned_tile_shapes": classes, "autotune_best_ms": best,
            "graph_on_config1": graph_small_leg(ev)}


def graph_small_leg(ev, reps=200):
    """The graph form on the smallest workload, config 1 (one 128x128 environment, K=8,
    131 k pixel-substeps per gap, a few microseconds of kernel work).  `reps` consecutive gaps
    of the same keyframe pair (identical device work on both paths): through evis_step
    (caller's buffers kept) and through evis_replay of a captured graph whose input buffers
    already hold the keyframe (where a renderer would write it).
    CUDA events around each whole run of gaps, so the time includes the device idling while
    the host launches, and the host's wall clock; per gap.  Then the host's own cost per call,
    issued while the stream is held by a spin kernel.  At this size a gap is bound by the step
    kernel's latency (its passes' dependent phases in 32 CTAs), not by launches."""
    import time
    import torch
    import scenes
    w = scenes.config1()
    dev = upload_keyframes(w, 11, "I")
    stream = torch.cuda.Stream()
    out = {}
    with torch.cuda.stream(stream):
        def run(name, one_gap):
            for k in range(1, 11):
                one_gap(k)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            a.record(stream)
            for j in range(reps):
                one_gap(1 + j % 10)
            b.record(stream)
            b.synchronize()
            wall = time.perf_counter() - t0
            # the host's own cost per call: the calls are issued while the stream is held by
            # a spin kernel, so none of them waits for the device
            torch.cuda._sleep(int(1e9))
            t1 = time.perf_counter()
            for j in range(reps):
                one_gap(1 + j % 10)
            host = time.perf_counter() - t1
            torch.cuda.synchronize()
            out[name] = {"device_us_per_gap": a.elapsed_time(b) * 1e3 / reps,
                         "wall_us_per_gap": wall * 1e6 / reps,
                         "host_us_per_call": host * 1e6 / reps}

        cap = (2 * reps + 12) * 131072
        step_ctx = ev.Context(w.envs, eps=1e-4, flags=ev.IN_LUM | ev.KEEP_INPUTS, capacity=cap,
                              stream=stream)
        step_ctx.step(*dev[0], w.dt_ns)
        run("evis_step", lambda k: step_ctx.step(*dev[1], w.dt_ns))
        step_ctx.close()
        graph = ev.Context(w.envs, eps=1e-4, flags=ev.IN_LUM, capacity=cap, stream=stream)
        graph.step(*dev[0], w.dt_ns)
        graph.step(*dev[1], w.dt_ns)
        graph.capture(w.dt_ns)
        graph.write_inputs(*dev[1])
        run("evis_replay", lambda k: graph.replay())
        graph.close()
    del dev
    out["workload"] = ("config 1: one env at 128x128, K=8, 131,072 pixel-substeps per gap, "
                       "linear inputs, the same keyframe pair every gap")
    out["gaps"] = reps
    out["replay_speedup_device"] = out["evis_step"]["device_us_per_gap"] / out["evis_replay"]["device_us_per_gap"]
    out["replay_host_saving"] = out["evis_step"]["host_us_per_call"] / out["evis_replay"]["host_us_per_call"]
    return out


def envs64_arm(args, world, rank, local):
    """The 346x260 workload as a line of its own (N ranks: disjoint environments)."""
    import torch
    import paper_2607_08098_b300 as ev
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    out = config2_leg(ev, args, world, rank, dist)
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def batched_arm(args):
    import torch
    import paper_2607_08098_b300 as ev
    torch.cuda.set_device(0)
    print(json.dumps(config3_leg(ev, args)), flush=True)


def soft_leg(reps=10):
    """Differentiable workload (16 envs at 346x260, K=8, tau=0.02): device time of the soft
    forward and of the backward under a random cotangent, their ratio, and the forward's
    HBM roofline (per pixel: L_A, L_B, both motion fields, both depths and the start
    reference level read, 36 B; the ON / OFF counts written, 8 B)."""
    import torch
    import paper_2607_08098_b300 as ev
    import scenes
    w = scenes.config5()
    kf = [scenes.render(w.envs, k) for k in range(2)]
    d = [torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()
         for a in (kf[0].L, kf[1].L, kf[0].mv, kf[1].mv, kf[0].Z, kf[1].Z, kf[0].L)]
    C = torch.full((len(w.envs),), 0.2, dtype=torch.float32, device="cuda")
    counts, ws = ev._soft_forward(w.envs, 0.02, 1e-3, *d, C)
    gc = torch.randn(counts.numel(), generator=torch.Generator().manual_seed(5)).cuda()
    ev._soft_backward(w.envs, 0.02, 1e-3, *d[:6], C, ws, gc)
    st = torch.cuda.current_stream()
    tf = tb = 0.0
    for _ in range(reps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(st)
        ev._soft_forward(w.envs, 0.02, 1e-3, *d, C, ws=ws)
        e1.record(st)
        ev._soft_backward(w.envs, 0.02, 1e-3, *d[:6], C, ws, gc)
        e2.record(st)
        e2.synchronize()
        tf += e0.elapsed_time(e1)
        tb += e1.elapsed_time(e2)
    fwd_ms, bwd_ms = tf / reps, tb / reps
    peak, peak_kind = measured_peak()
    alg = w.pixels * (36 + 8)
    ach = alg / (fwd_ms / 1e3) / 1e9
    return {"workload": "16 envs at 346x260, K=8, tau=0.02, delta=1e-3, random cotangent",
            "fwd_ms": fwd_ms, "bwd_ms": bwd_ms, "bwd_fwd_ratio": bwd_ms / fwd_ms,
            "pixel_substeps": w.pixel_substeps,
            "fwd_mpx_substeps_per_s": w.pixel_substeps / fwd_ms / 1e3,
            "roofline": {"kernel": "soft forward (winners, surface sums, per-target counts)",
                         "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "algorithmic_bytes_per_launch": alg,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}}


def _timed_gaps(ev, envs, dev, dt, steps, warmup, flags, setup=None):
    """ms per keyframe gap (CUDA events on the context's stream, L2 flushed between gaps),
    events per gap and the autotuned tile shape of a context over dev[k] = (frames, mv, depth)
    device tensors."""
    import torch
    probe = ev.Context(envs, eps=1e-4, flags=flags, capacity=1 << 27)
    if setup:
        setup(probe)
    probe.step(*dev[0], dt)
    probe.step(*dev[1], dt)
    per = probe.event_count()
    probe.close()
    ctx = ev.Context(envs, eps=1e-4, flags=flags, capacity=int(per * 1.5 * (steps + 1)) + (1 << 20))
    if setup:
        setup(ctx)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    ctx.step(*dev[0], dt)
    ctx.autotune(*dev[1], dt, reps=2)
    for k in range(1, 1 + warmup):
        ctx.step(*dev[k], dt)
    ctx.clear_events()
    st = torch.cuda.current_stream()
    ms = 0.0
    for s_ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        ctx.step(*dev[1 + warmup + s_], dt)
        b.record(st)
        b.synchronize()
        ms += a.elapsed_time(b)
    n = ctx.event_count()
    sh = ctx.tile_shapes()[0]
    ctx.close()
    return ms / steps, n / steps, f"{sh[0]}x{sh[1]}"


def stages_arm(args):
    """Device timings of the stages around the synthesis: sensor noise and colour events on
    the 64 x 346x260 workload (against the plain step), an 8-pixel over-render margin, the
    defocus kernel and the event voxel grid with their HBM rooflines."""
    import numpy as np
    import torch
    import paper_2607_08098_b300 as ev
    import scenes
    peak, peak_src = measured_peak()
    steps, warmup = args.steps, args.warmup
    w = scenes.config2(n_envs=args.envs)
    rng = np.random.default_rng(7)
    for e in w.envs:                                  # colour needs channels that differ
        for lay in e.layers:
            lay.tint_r, lay.tint_g, lay.tint_b = rng.uniform(0.4, 1.5, 3)
    out = {"bench": "stages", "steps": steps, "warmup": warmup,
           "workload": f"{args.envs} envs at 346x260, K=16, C=0.25, refractory 100us"}
    if args.stage in ("all", "synthesis"):
        out.update(_stage_synthesis(ev, scenes, w, args))
    if args.stage in ("all", "defocus"):
        out["defocus"] = _stage_defocus(ev, peak, peak_src)
    if args.stage in ("all", "voxel"):
        out["voxel_grid"] = _stage_voxel(ev, scenes, peak, peak_src, args.voxel_envs)
    print(json.dumps(out), flush=True)


def _stage_synthesis(ev, scenes, w, args):
    import torch
    steps, warmup = args.steps, args.warmup
    n_kf = warmup + steps + 1
    out = {}
    units = w.pixel_substeps
    kfs = [scenes.render(w.envs, k, want=("I", "rgb", "mv", "Z")) for k in range(n_kf)]
    mono = [tuple(torch.from_numpy(a.reshape(-1)).cuda() for a in (kf.I, kf.mv, kf.Z)) for kf in kfs]
    base_ms, base_ev, sh = _timed_gaps(ev, w.envs, mono, w.dt_ns, steps, warmup,
                                       ev.IN_LUM | ev.KEEP_INPUTS)
    out["plain"] = {"ms_per_gap": base_ms, "mpx_substeps_per_s": units / base_ms / 1e3,
                    "events_per_gap": base_ev, "tile_shape": sh}
    noise = [dict(leak_hz=0.1, shot_hz=5.0, hot_hz=100.0, hot_fraction=1e-3, lo=-3.0, hi=3.0,
                  seed=11)] * len(w.envs)
    nz_ms, nz_ev, sh = _timed_gaps(ev, w.envs, mono, w.dt_ns, steps, warmup,
                                   ev.IN_LUM | ev.KEEP_INPUTS, setup=lambda c: c.set_noise(noise))
    out["noise"] = {"rates": "leak 0.1 Hz, shot 5 Hz (dark), hot 100 Hz on 0.1 % of pixels",
                    "ms_per_gap": nz_ms, "mpx_substeps_per_s": units / nz_ms / 1e3,
                    "events_per_gap": nz_ev, "cost_vs_plain": nz_ms / base_ms, "tile_shape": sh}
    del mono
    colour = [tuple(torch.from_numpy(a.reshape(-1)).cuda() for a in (kf.rgb, kf.mv, kf.Z)) for kf in kfs]
    c_ms, c_ev, sh = _timed_gaps(ev, w.envs, colour, w.dt_ns, steps, warmup,
                                 ev.IN_RGB | ev.COLOR | ev.KEEP_INPUTS)
    out["colour"] = {"ms_per_gap": c_ms, "mpx_substeps_per_s": units / c_ms / 1e3,
                     "events_per_gap": c_ev, "cost_vs_plain": c_ms / base_ms, "tile_shape": sh,
                     "note": "three event models per pixel-substep over one splat"}
    del colour, kfs
    # margin: the same scenes rendered 8 pixels larger on each side, the sensor unchanged
    m = 8
    wm = scenes.config2(n_envs=args.envs)
    for e in wm.envs:
        e.W, e.H, e.margin = e.W + 2 * m, e.H + 2 * m, m
    kfm = [scenes.render(wm.envs, k, want=("I", "mv", "Z")) for k in range(n_kf)]
    devm = [tuple(torch.from_numpy(a.reshape(-1)).cuda() for a in (kf.I, kf.mv, kf.Z)) for kf in kfm]
    m_ms, m_ev, sh = _timed_gaps(ev, wm.envs, devm, wm.dt_ns, steps, warmup,
                                 ev.IN_LUM | ev.KEEP_INPUTS)
    out["margin"] = {"margin_px": m, "ms_per_gap": m_ms, "tile_shape": sh,
                     "sensor_mpx_substeps_per_s": units / m_ms / 1e3, "cost_vs_plain": m_ms / base_ms}
    del devm, kfm
    return out


def _stage_defocus(ev, peak, peak_src):
    """The defocus kernel on four 4096 x 4096 planes in a row (256 MB read for luminance:
    beyond L2), sigma 0.5 px (5 taps)."""
    import numpy as np
    import torch
    res = {}
    for mode, ch in (("luminance", 1), ("rgb", 3)):
        imgs = [torch.rand((4096, 4096, 3) if ch == 3 else (4096, 4096), device="cuda") + 0.01
                for _ in range(4)]
        st = torch.cuda.current_stream()
        for img in imgs:
            ev.defocus(img, 0.5)
        ts = []
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            outs = [ev.defocus(img, 0.5) for img in imgs]
            b.record(st)
            b.synchronize()
            ts.append(a.elapsed_time(b))
            del outs
        t = float(np.median(ts))
        alg = 4 * 4096 * 4096 * (4 * ch + 4)
        res[mode] = {"ms": t, "roofline": {"bound": "hbm", "achieved": alg / t / 1e6,
                     "peak": peak, "unit": "GB/s", "frac": alg / t / 1e6 / peak,
                     "algorithmic_bytes": alg, "peak_source": peak_src}}
        del imgs
    return res


def _stage_voxel(ev, scenes, peak, peak_src, n_envs=8):
    """The voxel grid of a 16-gap segment (128 ms) of the high-speed workload, n_envs envs
    at 640x480, 128 bins per polarity."""
    import numpy as np
    import torch
    w4 = scenes.config4(n_envs=n_envs)
    gaps = 16
    k4 = [scenes.render(w4.envs, k, want=("L", "mv", "Z")) for k in range(gaps + 1)]
    d4 = [tuple(torch.from_numpy(a.reshape(-1)).cuda() for a in (kf.L, kf.mv, kf.Z)) for kf in k4]
    ctx = ev.Context(w4.envs, flags=ev.IN_LOG | ev.KEEP_INPUTS, capacity=1 << 28)
    for d in d4:
        ctx.step(*d, w4.dt_ns)
    n_ev = ctx.event_count()
    segs = [(e.W, e.H, e.t0_ns, e.t0_ns + gaps * w4.dt_ns) for e in w4.envs]
    bins = 128
    wsb = ev.voxel_workspace_size(segs, bins, ctx.capacity)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    ctx.voxel_grid(segs, bins, ws)
    st = torch.cuda.current_stream()
    ts = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        g = ctx.voxel_grid(segs, bins, ws)
        b.record(st)
        b.synchronize()
        ts.append(a.elapsed_time(b))
        del g
    t = float(np.median(ts))
    vox = sum(2 * bins * W * H for W, H, _, _ in segs)
    alg = n_ev * 16 + vox * 4
    dense = n_ev * 16 + vox * 12
    res = {"workload": f"{n_envs} envs at 640x480, 16 keyframe gaps (128 ms) of the "
                       "high-speed scenes, 128 bins per polarity",
           "events": n_ev, "voxels": vox, "ms": t,
           "events_per_s": n_ev / t * 1e3,
           "roofline": {"bound": "hbm", "achieved": alg / t / 1e6, "peak": peak,
                        "unit": "GB/s", "frac": alg / t / 1e6 / peak,
                        "algorithmic_bytes": alg, "peak_source": peak_src,
                        "bytes_model": "16 B per event read + 4 B per voxel written (the "
                                       "records in, the grid out)"},
           "frac_dense_accumulator_model": dense / t / 1e6 / peak,
           "dense_accumulator_model": "16 B per event + 12 B per voxel (a dense uint32 "
                                      "accumulator cleared, read and the grid written)"}
    ctx.close()
    return res


def main():
    args = parse()
    world, rank, local = dist_info()
    if args.impl == "reference":
        reference_arm(args, world, rank)
    elif args.workload == "batched":
        batched_arm(args)
    elif args.workload == "stages":
        stages_arm(args)
    elif args.workload == "envs64":
        envs64_arm(args, world, rank, local)
    elif args.workload == "soft":
        import torch
        torch.cuda.set_device(local)
        print(json.dumps(soft_leg()), flush=True)
    else:
        headline_arm(args, world, rank, local)


if __name__ == "__main__":
    main()
