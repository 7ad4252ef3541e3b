"""Benchmark: batched SIFT extraction on GB300 (one JSON line on stdout).

Workload (timed as `value`): the mixed-resolution batch, 64 FP32 grayscale
images extracted in one sift_extract_batch call per step; long sides uniform
in 480-1600 px, aspect ratios 4:3 / 3:4 / 16:9, seeded synthetic content with
1/f texture, no upsampling, cap 8192 keypoints per image. value = input
megapixels per second over all ranks. The step's inputs (about 200 MB) and
its pyramid (about 1.6 GB) are far larger than L2; L2 is also flushed between
timed steps by writing a 256 MB buffer (outside the timed events).

Also reported: keypoints/s; the same images through the per-image entry
point and the batched/per-image ratio; per-class device times with the
roofline of each class; end-to-end throughput through the public API from
pinned host buffers; the homography-sequence batch (6 x 1000x750, 2x
upsampled) with matching accuracy and with DSP pooling + RootSIFT; the
single-image and image-pair latencies (with the matcher and MAGSAC++);
serving images/s with p50/p99 latency under Poisson arrivals; and the FP64
oracle timed on the host cores on a bounded sample.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-serving]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import matching, synth  # noqa: E402

METRIC = "SIFT Mpix/s and keypoints/s, batched vs per-image; serving p50/p99 latency"
N_IMAGES = 64
WORKLOAD = ("mixed-resolution batch: 64 FP32 grayscale images in one call, long side uniform "
            "480-1600 px, aspect 4:3/3:4/16:9, seeded synthetic content with 1/f texture, "
            "no upsampling, cap 8192 keypoints/image")
HOMOGRAPHY_WORKLOAD = ("homography-sequence batch: 6 x 1000x750 FP32 grayscale (seeded base + 5 "
                       "homography warps), 2x upsampled first octave, cap 8000 keypoints/image")
SERVING_RATES = (50, 100, 200, 500, 1000, 2000)
SERVING_REQUESTS = 1000
MAX_KPTS = 8192
L2_FLUSH_BYTES = 256 << 20


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------ inputs
# Multi-GPU runs are independent replicas: rank r extracts its own batch (the
# mixed-resolution batch drawn with shape index r and image seeds 100 r + i;
# rank 0's is the canonical batch); the only communication is a barrier and
# the max of the timed-region durations.

class Batch:
    def __init__(self, images):
        self.images = images
        self.shapes = [im.shape for im in images]


def _mixed_one(args):
    rank, i, n = args
    (h, w) = synth.mixed_batch_shapes(n, index=rank)[i]
    return synth.make_image(synth.rng_for(3, 100 * rank + i), h, w, fractal_std=0.05)


def replica_batch(rank, n_images=N_IMAGES, pool=None):
    """The images rank `rank` processes (distinct per rank)."""
    jobs = [(rank, i, n_images) for i in range(n_images)]
    imgs = pool.map(_mixed_one, jobs) if pool is not None else [_mixed_one(j) for j in jobs]
    return Batch(imgs)


def max_over_ranks(x, device):
    """Max of a per-rank float over the process group (then a barrier)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def whole_job_value(world, mpix_per_rank, steps, max_ms):
    """Whole-job throughput: the pixels all ranks processed / the slowest rank's time."""
    return world * mpix_per_rank * steps / (max_ms / 1e3)


# ------------------------------------------------------------ oracle (CPU)

def _oracle_one(args):
    img, upsample, max_kpts = args
    from oracle import sift_oracle as so
    t = time.perf_counter()
    r = so.extract(img, so.Params(upsample=bool(upsample), max_kpts=max_kpts))
    return time.perf_counter() - t, len(r)


def _oracle_pool(n):
    return mp.get_context("spawn").Pool(n)


def _oracle_workers():
    return max(1, min(16, os.cpu_count() or 1))


def _center_crop(im, h, w):
    y0 = (im.shape[0] - h) // 2
    x0 = (im.shape[1] - w) // 2
    return np.ascontiguousarray(im[y0:y0 + h, x0:x0 + w])


def _oracle_sample(pool, n_workers, images, budget_s):
    """A bounded sample of the workload for the oracle: the first n_workers
    images, centre-cropped (same aspect) so that one pass over them takes about
    budget_s on the pool. Returns (crops, description)."""
    imgs = images[:n_workers]
    small = [_center_crop(im, im.shape[0] // 4, im.shape[1] // 4) for im in imgs]
    t0 = time.perf_counter()
    pool.map(_oracle_one, [(im, False, MAX_KPTS) for im in small])  # also warms the workers
    t_small = max(1e-3, time.perf_counter() - t0)
    frac = min(1.0, budget_s / (16.0 * t_small))
    crops = []
    for im in imgs:
        h = max(64, min(im.shape[0], int(round(im.shape[0] * math.sqrt(frac)))))
        w = max(64, min(im.shape[1], int(round(im.shape[1] * math.sqrt(frac)))))
        crops.append(_center_crop(im, h, w))
    full = all(c.shape == im.shape for c, im in zip(crops, imgs))
    what = (f"the first {len(crops)} images of the timed batch "
            f"({'full size' if full else 'centre crops of ' + f'{100 * frac:.0f}% of the area'}, "
            f"{sum(c.size for c in crops) / 1e6:.2f} Mpx), no upsampling, cap {MAX_KPTS}, one image "
            f"per worker process")
    return crops, what


def cpu_baseline(pool, n_workers, images, budget_s=12.0):
    crops, what = _oracle_sample(pool, n_workers, images, budget_s)
    t0 = time.perf_counter()
    res = pool.map(_oracle_one, [(im, False, MAX_KPTS) for im in crops])
    wall = time.perf_counter() - t0
    mpix = sum(im.size for im in crops) / 1e6
    return {"value": round(mpix / wall, 4), "unit": "Mpix/s", "cores": n_workers,
            "kind": "oracle", "keypoints_per_s": round(sum(k for _, k in res) / wall, 1),
            "sample": f"{what}; {wall:.1f} s wall"}


# ------------------------------------------------------------ clocks

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index):
        self.proc = None
        self.dev = dev_index
        self.path = os.path.join(tempfile.gettempdir(), f"sift_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # Wait (at most 5 s) for the first sample so the sampler covers the
        # whole timed region rather than starting part-way through it.
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ algorithmic bytes

def _octaves(h, w, upsample, min_side=16):
    H, W = (2 * h, 2 * w) if upsample else (h, w)
    out = []
    while min(H, W) >= min_side:
        out.append((H, W))
        H, W = H // 2, W // 2
    return out


def _alg_blur_bytes(shapes, upsample, S=3, min_side=16):
    """Algorithmic bytes and pixels of all level-blur launches of one step.

    A level blur reads its source level once and writes the new level once
    (8 B per octave pixel); octave 0 has S + 2 of them. In octaves above 0 the
    first one also decimates: it reads one source value per output pixel and
    writes levels 0 and 1 (12 B per octave pixel), and S + 1 plain ones follow.
    Returns (bytes, pixels processed), the pixels summed over launches."""
    tot = px_tot = 0
    for (h, w) in shapes:
        for o, (H, W) in enumerate(_octaves(h, w, upsample, min_side)):
            px = H * W
            tot += 8 * px * (S + 2) + (4 * px if o > 0 else 0)
            px_tot += px * (S + 2)
    return tot, px_tot


def _level_radii(S=3, sigma0=1.6):
    """Blur radius ceil(4 kappa_i) of the incremental level blurs i = 1 .. S + 2,
    kappa_i = sigma0 sqrt(2^(2i/S) - 2^(2(i-1)/S)) (§3.2)."""
    return [math.ceil(4.0 * sigma0 * math.sqrt(2.0 ** (2.0 * i / S) - 2.0 ** (2.0 * (i - 1) / S))
                      - 1e-9) for i in range(1, S + 3)]


def _alg_blur_flops(shapes, upsample, S=3, min_side=16):
    """FP32 operations of all level-blur launches of one step: a separable blur
    of radius R is 2 (2R + 1) FMAs, 4 (2R + 1) FLOP, per octave pixel."""
    radii = _level_radii(S)
    tot = 0
    for (h, w) in shapes:
        for (H, W) in _octaves(h, w, upsample, min_side):
            tot += H * W * sum(4 * (2 * r + 1) for r in radii)
    return tot


def _fp32_peak_tflops(sm_mhz):
    """FP32 FMA peak from unit counts and the SM clock: 128 FP32 lanes per SM,
    2 FLOP per FMA."""
    import torch
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12


def _pyramid_bytes(shapes, upsample, fp16, S=3, min_side=16):
    """Device bytes of one step's Gaussian pyramids: S + 3 levels per octave,
    rows padded to 32 elements; 4-byte elements, or 2-byte ones above octave 0
    in the fp16 storage mode."""
    tot = 0
    for (h, w) in shapes:
        for o, (H, W) in enumerate(_octaves(h, w, upsample, min_side)):
            tot += (S + 3) * H * ((W + 31) // 32 * 32) * (2 if fp16 and o > 0 else 4)
    return tot


def _alg_class_bytes(shapes, upsample, S=3, min_side=16):
    """Algorithmic bytes of one step for the base blur and the extrema scan.
    Base: the input read once (4 B per input pixel) and level 0 of octave 0
    written once (4 B per octave pixel). Extrema: the S + 3 levels of every
    octave read once (the DoG is formed on the fly) plus the candidate bitmap
    (S bits per octave pixel)."""
    base = ext = 0
    for (h, w) in shapes:
        octs = _octaves(h, w, upsample, min_side)
        base += 4 * h * w + 4 * octs[0][0] * octs[0][1]
        for (H, W) in octs:
            ext += 4 * (S + 3) * H * W + S * H * W // 8
    return {"base": base, "extrema": ext}


# ------------------------------------------------------------ GPU arm

def _device_images(imgs, torch):
    return [torch.from_numpy(np.ascontiguousarray(im)).cuda() for im in imgs]


def timed_steps(torch, fn, steps, warmup, flush, stream):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    times = []
    t_wall = time.perf_counter()
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    torch.cuda.synchronize()
    return times, time.perf_counter() - t_wall


def queued_steps(torch, fn, steps, warmup, stream):
    """Device time of `steps` steps queued back to back between one pair of
    CUDA events on `stream`, after `warmup` untimed ones: the throughput of a
    steady stream of batches, the host's launch work for step k + 1 overlapping
    the device's work on step k. No flush between steps: every step reads its
    inputs and writes a pyramid far larger than L2. Returns (ms, wall s)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    t_wall = time.perf_counter()
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    b.synchronize()
    torch.cuda.synchronize()
    return a.elapsed_time(b), time.perf_counter() - t_wall


def best_queued_ms(torch, fn, steps, warmup, stream, reps=3):
    """ms per step of the best of `reps` runs of queued_steps (steps / reps
    steps each): the side records are timed after other work on the same
    device, and one slow stretch there should not stand for the path."""
    n = max(1, steps // reps)
    return min(queued_steps(torch, fn, n, warmup, stream)[0] / n for _ in range(reps))


def profiled_classes(torch, ex, step, flush, reps):
    """Per-class device time of one step (ms) and launches: a profiled graph
    with a CUDA event pair around every launch, all launches on one stream."""
    ex.set_profiling(True)
    step()
    torch.cuda.synchronize()
    acc = {}
    for _ in range(reps):
        flush.zero_()
        step()
        for k, (ms, n) in ex.kernel_times().items():
            a = acc.setdefault(k, [0.0, 0])
            a[0] += ms / reps
            a[1] = n
    ex.set_profiling(False)
    return acc


def _traffic_per_launch(px_step, blur_n):
    """DRAM bytes of an average level-blur launch of this workload: the per-pixel
    DRAM traffic of a captured level-blur launch (profiles/blur_level_traffic.json)
    times the pixels an average launch processes; only while pyramid.cu is the
    source the counters were read from."""
    tpath = os.path.join(ROOT, "profiles", "blur_level_traffic.json")
    if not os.path.exists(tpath) or not blur_n:
        return None
    with open(tpath) as f:
        tj = json.load(f)
    src = open(os.path.join(ROOT, "paper_2605_17869_gb300", "csrc", "pyramid.cu"), "rb").read()
    if tj.get("pyramid_cu_sha256") != hashlib.sha256(src).hexdigest():
        return None
    return int(tj["dram_bytes_per_px"] * px_step / blur_n)


def _is_default_tuning(js):
    """Whether a tuning JSON is the defaults (32-row tiles, occupancy-maximum
    grids, a batch split over two lanes): a tuned time then differs from the
    untuned one by noise only."""
    t = json.loads(js)
    rows = t.get("blur_tile_rows", [])
    rows = rows if rows and isinstance(rows[0], list) else [rows]
    return (all(r == 32 for oc in rows for r in oc)
            and all(c == 0 for c in t.get("blur_ctas_per_sm", []))
            and all(v == 0 for k, v in t.items() if k.endswith("_ctas_per_sm") and not isinstance(v, list))
            and t.get("batch_lanes", 2) == 2)


def rooflines(acc, shapes, upsample, kpts, sm_mhz=None):
    peak, peak_kind = _peaks()
    src = "hbm_gbs, " + ("of measured (MEASURED_PEAKS.json)" if peak_kind == "measured"
                         else "of fallback")
    alg_step, px_step = _alg_blur_bytes(shapes, upsample)
    blur_ms, blur_n = acc["blur"]
    achieved = alg_step / (blur_ms / 1e3) / 1e9 if blur_ms > 0 else 0.0
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": _traffic_per_launch(px_step, blur_n),
                "kernel": "k_blur (pyramid level blur; all launches of a step)",
                "alg_bytes_per_launch": int(alg_step / max(1, blur_n)),
                "launch_ms_avg": round(blur_ms / max(1, blur_n), 5),
                "peak_source": src}
    if blur_ms > 0 and sm_mhz:
        # The level blur sits at the ridge of the dual roofline (HBM bytes vs
        # FP32 FMAs): its attainable time is the larger of the two.
        flops = _alg_blur_flops(shapes, upsample)
        fp32_peak = _fp32_peak_tflops(sm_mhz)
        t_hbm = alg_step / (peak * 1e9)
        t_fp32 = flops / (fp32_peak * 1e12)
        roofline["dual"] = {
            "fp32_tflops_achieved": round(flops / (blur_ms / 1e3) / 1e12, 2),
            "fp32_peak_tflops": round(fp32_peak, 1),
            "fp32_peak_source": "SMs x 128 FP32 lanes x 2 FLOP x median SM clock under load",
            "hbm_time_ms": round(t_hbm * 1e3, 4), "fp32_time_ms": round(t_fp32 * 1e3, 4),
            "frac_of_attainable": round(max(t_hbm, t_fp32) / (blur_ms / 1e3), 4)}
    cls_bytes = _alg_class_bytes(shapes, upsample)
    cls_bytes["blur"] = alg_step
    per_class = {}
    for k in ("blur", "base", "extrema"):
        ms = acc.get(k, (0.0, 0))[0]
        if ms > 0:
            gbs = cls_bytes[k] / (ms / 1e3) / 1e9
            per_class[k] = {"alg_bytes_per_step": int(cls_bytes[k]), "ms_per_step": round(ms, 4),
                            "achieved_gbs": round(gbs, 1), "frac_of_measured": round(gbs / peak, 4),
                            "frac_of_nominal_8tbs": round(gbs / 8000.0, 4)}
    for k in ("refine", "orientation", "keypoint", "descriptor"):
        ms = acc.get(k, (0.0, 0))[0]
        if ms > 0:
            per_class[k] = {"ms_per_step": round(ms, 4),
                            "keypoints_per_s": round(kpts / (ms / 1e3), 1)}
    return roofline, per_class


E2E_LANES = 4


def e2e_throughput(torch, pkg, ex, imgs_np, tuning, steps, warmup, world, ext_kw,
                   n_lanes=E2E_LANES):
    """End to end: pinned host images -> device -> extract -> results back in one
    packed copy. n_lanes handles on their own streams take the steps in turn:
    steps k + 1 .. k + n_lanes - 1 are uploaded and queued before step k is read
    back, so the GPU does not wait for the host and one batch's latency-bound
    stretches (the small octaves, the keypoint chain) overlap another's work,
    as in a serving pipeline. Every step uploads its own inputs and reads back
    its own results. The handles run their batches whole (batch_lanes 1): the
    pipeline already overlaps batches, and a second lane per handle measured
    slower with three handles and no faster with four."""
    host = [torch.from_numpy(np.ascontiguousarray(im)).pin_memory() for im in imgs_np]
    h2d = sum(h.numel() * 4 for h in host)
    extra = [pkg.Extractor(**ext_kw) for _ in range(n_lanes - 1)]
    for e in [ex] + extra:
        e.set_tuning(tuning)
        e.set_tuning('{"batch_lanes": 1}')
    warmup = max(warmup, n_lanes)  # every handle captures its graph before the timed steps
    lanes = [(e, torch.cuda.Stream(), [torch.empty_like(h, device="cuda") for h in host])
             for e in [ex] + extra]

    def submit(lane):
        e, st, din = lane
        with torch.cuda.stream(st):
            for d, h in zip(din, host):
                d.copy_(h, non_blocking=True)
        e.extract_batch_async(din, st)

    def collect(lane):
        e, st, _ = lane
        counts_h, _ = e.download(st)
        return 4 * len(counts_h) + 540 * sum(counts_h)

    for it in range(warmup):
        submit(lanes[it % n_lanes])
        collect(lanes[it % n_lanes])
    torch.cuda.synchronize()
    d2h_bytes = []
    mpix = sum(im.size for im in imgs_np) / 1e6
    t0 = time.perf_counter()
    for k in range(min(n_lanes - 1, steps)):
        submit(lanes[k])
    for it in range(steps):
        if it + n_lanes - 1 < steps:
            submit(lanes[(it + n_lanes - 1) % n_lanes])
        d2h_bytes.append(collect(lanes[it % n_lanes]))
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    for e in extra:
        e.close()
    ex.set_tuning(tuning)
    return {"value": round(world * mpix * steps / t_e2e, 3), "unit": "Mpix/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(np.mean(d2h_bytes)),
            "steps": steps, "lanes": n_lanes, "batch_lanes": 1,
            "api": f"Extractor.extract_batch_async (sift_extract_batch) from pinned host buffers, "
                   f"results by Extractor.download (sift_pack_outputs + one copy); {n_lanes} "
                   f"handles on {n_lanes} streams take the steps in turn (steps k+1 .. "
                   f"k+{n_lanes - 1} queued before step k is read back)"}


def gpu_arm(args, rank, world, pool, batch):
    import torch
    import paper_2605_17869_gb300 as pkg

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    imgs_np = batch.images
    shapes = batch.shapes
    imgs = _device_images(imgs_np, torch)
    mpix = sum(h * w for h, w in shapes) / 1e6
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    ext_kw = dict(upsample=0, max_kpts=MAX_KPTS)
    ex = pkg.Extractor(**ext_kw)

    def step():
        ex.extract_batch_async(imgs, stream)

    autotune = None
    if args.tuning:
        ex.set_tuning(args.tuning)
    else:
        # The defaults first (32-row tiles, occupancy-maximum grids), then the
        # batch autotuner on this very batch; the timed steps use its choice.
        n_def = max(10, args.steps // 4)
        t_def, _ = queued_steps(torch, step, n_def, args.warmup, stream)
        t0 = time.perf_counter()
        _, hit = ex.autotune_batch(imgs, stream, cache=args.tuning_cache or None)
        torch.cuda.synchronize()
        autotune = {"untuned_ms_per_step": round(t_def / n_def, 4),
                    "search_s": round(time.perf_counter() - t0, 3), "from_cache": hit}
    tuning = ex.get_tuning()
    if autotune is not None:
        autotune["chose_defaults"] = _is_default_tuning(tuning)

    if args.minimal:
        total, _ = queued_steps(torch, step, args.steps, args.warmup, stream)
        return {"metric": METRIC, "value": round(mpix * args.steps / (total / 1e3), 2),
                "unit": "Mpix/s", "mode": "minimal (timed loop only)", "images": len(imgs),
                "ms_per_step": round(total / args.steps, 4),
                "gpu_launches_per_step": ex.launch_count(), "tuning": tuning}

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = Clocks(dev)
    clocks.start()
    total_ms, wall = queued_steps(torch, step, args.steps, args.warmup, stream)
    clock_info = clocks.stop()
    counts = ex._counts[:len(imgs)].tolist()
    kpts = sum(counts)
    launches_per_step = ex.launch_count()
    if world > 1:
        total_ms = max_over_ranks(total_ms, "cuda")
    value = whole_job_value(world, mpix, args.steps, total_ms)
    # One step at a time (L2 flushed, the host's launch work not overlapped).
    t_iso, _ = timed_steps(torch, step, max(5, args.steps // 4), 2, flush, stream)

    # Per-image path on the same images, timed the same way as the batch.
    def step_single():
        for im in imgs:
            ex.extract_async(im, stream)
    n_single = max(3, args.steps // 4)
    t_single, _ = queued_steps(torch, step_single, n_single, 2, stream)
    per_image = mpix * n_single / (t_single / 1e3)

    reps = max(3, args.steps // 4)
    acc = profiled_classes(torch, ex, step, flush, reps)
    roofline, per_class = rooflines(acc, shapes, False, kpts, clock_info.get("sm_mhz"))
    e2e = e2e_throughput(torch, pkg, ex, imgs_np, tuning, max(3, args.steps // 2), args.warmup,
                         world, ext_kw)

    extra = {}
    if rank == 0 and not args.no_configs:
        extra["fp16_pyramid"] = fp16_side(torch, pkg, imgs, shapes, mpix, flush, stream, tuning,
                                          max(10, args.steps // 2))
        extra["keypoint_heavy"] = keypoint_heavy_side(torch, pkg, flush, stream, tuning,
                                                      max(10, args.steps // 2))
        extra["homography_sequence"] = homography_side(torch, pkg, flush, stream, tuning,
                                                       max(10, args.steps // 2))
        extra["single_and_pair"] = other_configs(torch, pkg, flush, stream, tuning)
    if rank == 0 and not args.no_serving:
        extra["serving"] = serving_bench(torch, pkg, SERVING_RATES, args.serving_requests)

    res = {
        "metric": METRIC, "value": round(value, 2), "unit": "Mpix/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "isolated_ms_per_step": round(statistics.mean(t_iso), 4),
        "isolated_note": "one step at a time: L2 flushed before it and the host's launch work "
                         "(about 0.1 ms for 64 images) not overlapped",
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "images_per_step_per_gpu": len(imgs),
                   "input_mpix_per_step_per_gpu": round(mpix, 3),
                   "l2": "inputs and pyramid larger than L2 (198 MB of images in, about 1.6 GB "
                         "of pyramid written per step); steps queued back to back, no flush",
                   "parallelism": f"replicas x{world} (independent images per rank)",
                   "tuning": tuning},
        "keypoints_per_s": round(world * kpts * args.steps / (total_ms / 1e3), 1),
        "keypoints_per_step_per_gpu": kpts,
        "per_image_mpix_s": round(per_image, 2),
        "batched_vs_per_image": round(value / world / per_image, 3),
        "wall_s_timed_region": round(wall, 3),
        "gpu_launches": launches_per_step * args.steps,
        "gpu_launches_per_step": launches_per_step,
        "kernel_ms_per_step": {k: round(v[0], 4) for k, v in acc.items()},
        # Per-class times come from the profiled graph (an event pair around every
        # launch, all on one stream); their sum against the live step shows how
        # much the side branches and programmatic dependent launch overlap.
        "kernel_ms_per_step_note": "profiled graph: each launch timed alone on one stream",
        "kernel_ms_sum": round(sum(v[0] for v in acc.values()), 4),
        "live_over_kernel_sum": round((total_ms / args.steps) / max(1e-9, sum(v[0] for v in acc.values())), 4),
        "autotune": autotune and {**autotune, "tuned_ms_per_step": round(total_ms / args.steps, 4),
                                  "untuned_over_tuned": round(autotune["untuned_ms_per_step"] /
                                                              (total_ms / args.steps), 4)},
        "roofline": roofline,
        "per_class_roofline": per_class,
        "e2e": e2e,
        "clocks": clock_info,
        **extra,
    }
    return res


def fp16_side(torch, pkg, imgs, shapes, mpix, flush, stream, tuning, steps):
    """The timed batch in the fp16 storage mode (§3.2: octaves above 0 stored
    as binary16, octave 0 FP32): throughput, per-class time and the pyramid's
    device bytes against the FP32 mode."""
    ex = pkg.Extractor(upsample=0, max_kpts=MAX_KPTS, fp16_pyramid=1)
    ex.set_tuning(tuning)
    step = lambda: ex.extract_batch_async(imgs, stream)  # noqa: E731
    ms = best_queued_ms(torch, step, steps, 3, stream)
    counts = ex._counts[:len(imgs)].tolist()
    cls = profiled_classes(torch, ex, step, flush, 3)
    ex.close()
    return {"workload": "the timed batch with fp16_pyramid=1",
            "timing": "best of 3 runs of queued steps",
            "ms_per_step": round(ms, 4),
            "mpix_s": round(mpix / (ms / 1e3), 1),
            "keypoints_per_step": sum(counts),
            "kernel_ms_per_step": {k: round(v[0], 4) for k, v in cls.items()},
            "pyramid_bytes_per_step": _pyramid_bytes(shapes, False, True),
            "pyramid_bytes_per_step_fp32": _pyramid_bytes(shapes, False, False)}


def keypoint_heavy_side(torch, pkg, flush, stream, tuning, steps):
    """The per-keypoint stages under keypoint-heavy load: 4 images of 1600x1200
    (the wide-baseline generator with 200 blobs and strong 1/f texture, std
    0.12), 2x upsampled, cap 8192, one batched call. Reports keypoints per
    image and, for refinement, orientation and descriptor, their device time
    and inputs/s: candidates for refinement, refined keypoints for
    orientation, kept (capped) keypoints for the descriptor."""
    imgs_np = [synth.make_image(synth.rng_for(2, 700 + i), 1200, 1600, n_blobs=200,
                                fractal_std=0.12) for i in range(4)]
    imgs = _device_images(imgs_np, torch)
    ex = pkg.Extractor(upsample=1, max_kpts=MAX_KPTS)
    ex.set_tuning(tuning)
    step = lambda: ex.extract_batch_async(imgs, stream)  # noqa: E731
    ms_step = best_queued_ms(torch, step, steps, 3, stream)
    counts = ex._counts[:len(imgs)].tolist()
    _, stats = ex.stats(len(imgs))
    cls = profiled_classes(torch, ex, step, flush, 3)
    ex.close()
    n_in = {"refine": sum(s[0] for s in stats),        # candidates after the contrast gate
            "orientation": sum(s[1] for s in stats),   # refined keypoints
            "descriptor": sum(counts)}                 # oriented keypoints kept by the cap
    out = {"workload": "4 x 1600x1200, 200 blobs + 1/f texture (std 0.12), 2x upsampled, cap 8192",
           "timing": "best of 3 runs of queued steps",
           "keypoints_per_image": counts,
           "candidates_per_image": [s[0] for s in stats],
           "refined_per_image": [s[1] for s in stats],
           "oriented_per_image": [s[2] for s in stats],
           "ms_per_step": round(ms_step, 4),
           "kernel_ms_per_step": {k: round(v[0], 4) for k, v in cls.items()}}
    for k, n in n_in.items():
        ms = cls.get(k, (0.0, 0))[0]
        if ms > 0 and n:
            out[k] = {"ms": round(ms, 4), "inputs": n, "inputs_per_s": round(n / (ms / 1e3), 1)}
    return out


def homography_side(torch, pkg, flush, stream, tuning, steps):
    """The homography-sequence batch (6 x 1000x750, 2x upsampled, cap 8000):
    throughput, per-class time, matching accuracy against the known
    homographies, and the same batch with DSP pooling + RootSIFT (§3.2)."""
    seq = synth.homography_sequence(index=0)
    imgs = _device_images(seq.images, torch)
    mpix = sum(im.size for im in seq.images) / 1e6
    out = {"workload": HOMOGRAPHY_WORKLOAD}
    for label, kw in (("plain", {}), ("dsp_rootsift", {"dsp": 1, "rootsift": 1})):
        ex = pkg.Extractor(upsample=1, max_kpts=8000, **kw)  # default tuning
        step = lambda: ex.extract_batch_async(imgs, stream)  # noqa: E731
        ms_step = best_queued_ms(torch, step, steps, 3, stream)
        counts = ex._counts[:len(imgs)].tolist()
        feats = [ex._bufs[i].view(counts[i]) for i in range(len(imgs))]
        acc = matching.sequence_mma(feats, seq.homographies)
        cls = profiled_classes(torch, ex, step, flush, 3)
        r = {"ms_per_step": round(ms_step, 4), "timing": "best of 3 runs of queued steps",
             "mpix_s": round(mpix / (ms_step / 1e3), 1),
             "keypoints_per_s": round(sum(counts) / (ms_step / 1e3), 1),
             "kernel_ms_per_step": {k: round(v[0], 4) for k, v in cls.items()},
             "matches": acc["matches"], **{k: v for k, v in acc.items() if k.startswith("mma@")}}
        if label == "plain":
            def single():
                for im in imgs:
                    ex.extract_async(im, stream)
            n_s = max(3, steps // 2)
            ts = queued_steps(torch, single, n_s, 2, stream)[0]
            r["per_image_mpix_s"] = round(mpix * n_s / (ts / 1e3), 1)
            r["accuracy"] = {"what": "image 0 matched to each warped image; MMA against the known "
                                     "homographies (harness: torch mutual NN + ratio 0.8)", **acc}
            # The batch autotuner on this batch: the steps above used the defaults.
            t0 = time.perf_counter()
            js, _ = ex.autotune_batch(imgs, stream)
            torch.cuda.synchronize()
            search = time.perf_counter() - t0
            tt = queued_steps(torch, step, steps, 3, stream)[0] / steps
            r["autotune"] = {"untuned_ms_per_step": r["ms_per_step"],
                             "tuned_ms_per_step": round(tt, 4),
                             "untuned_over_tuned": round(r["ms_per_step"] / tt, 4),
                             "search_s": round(search, 3), "tuning": js,
                             "chose_defaults": _is_default_tuning(js)}
        out[label] = r
        ex.close()
    return out


def homography_loop(torch, pkg, stream, tuning, steps, warmup):
    """A timed loop of the homography-sequence batch alone: `warmup` steps,
    then `steps` steps queued back to back (one graph per lane and step)."""
    seq = synth.homography_sequence(index=0)
    imgs = _device_images(seq.images, torch)
    ex = pkg.Extractor(upsample=1, max_kpts=8000)
    ex.set_tuning(tuning)
    ms, _ = queued_steps(torch, lambda: ex.extract_batch_async(imgs, stream), steps, warmup, stream)
    r = {"workload": HOMOGRAPHY_WORKLOAD, "mode": "timed loop only", "steps": steps,
         "warmup": warmup, "ms_per_step": round(ms / steps, 4),
         "gpu_launches_per_step": ex.launch_count(), "tuning": ex.get_tuning()}
    ex.close()
    return r


def serving_bench(torch, pkg, rates, n_req, budget=8 << 30):
    """Poisson arrivals at each rate: submit on arrival, collect every result,
    report images/s and p50 / p99 latency (from submission to completion)."""
    pool = {}
    for (h, w) in ((480, 640), (1080, 1920), (2160, 3840)):
        pool[(h, w)] = [torch.from_numpy(synth.serving_image(h, w, i)).cuda() for i in range(2)]
    ex = pkg.Extractor(max_kpts=MAX_KPTS)
    srv = pkg.Server(ex, budget_bytes=budget, max_slots=256)
    # warm-up: one of each size
    for k in pool:
        t = srv.submit(pool[k][0])
        srv.result(t)
        srv.release(t)
    out = []
    for lam in rates:
        prev = srv.steps()
        t_before = prev[-1][3] if prev else float("-inf")
        trace = synth.serving_trace(lam, n_req, index=int(lam))
        tickets = []
        t0 = time.perf_counter()
        for (ta, h, w, i) in trace:
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            tickets.append(srv.submit(pool[(h, w)][i % 2]))
        lat = []
        px = 0
        for tk, (_, h, w, _) in zip(tickets, trace):
            f, ms, st = srv.result(tk)
            lat.append(ms)
            px += h * w
            srv.release(tk)
        span = time.perf_counter() - t0
        lat.sort()
        steps = [s for s in srv.steps() if s[2] > t_before]
        # Device time during which steps of two or more lanes ran at once.
        ev = sorted([(a, 1) for _, _, a, _ in steps] + [(b, -1) for _, _, _, b in steps])
        busy = conc = 0.0
        depth, last = 0, None
        for t, dlt in ev:
            if last is not None and depth > 0:
                busy += t - last
                if depth > 1:
                    conc += t - last
            depth += dlt
            last = t
        out.append({"rate_per_s": lam, "requests": n_req, "images_per_s": round(n_req / span, 1),
                    "mpix_per_s": round(px / 1e6 / span, 1),
                    "p50_ms": round(lat[len(lat) // 2], 3),
                    "p99_ms": round(lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)], 3),
                    "steps": len(steps),
                    "images_per_step": round(n_req / max(1, len(steps)), 2),
                    "device_busy_ms": round(busy, 2),
                    "lanes_concurrent_frac_of_busy": round(conc / busy, 4) if busy > 0 else 0.0})
    srv.close()
    ex.close()
    return {"workload": "Poisson arrivals, 640x480 (50%) / 1920x1080 (35%) / 3840x2160 (15%), "
                        "8 GB device-memory budget, no upsampling, cap 8192",
            "points": out}


def other_configs(torch, pkg, flush, stream, tuning):
    """Latency of the single-image and wide-baseline-pair workloads (device
    time per call, warm, L2 flushed before each), with MMA for the pair."""
    out = {}
    vga = _device_images([synth.single_vga(0)], torch)
    ex0 = pkg.Extractor(upsample=0)
    t0, _ = timed_steps(torch, lambda: ex0.extract_async(vga[0], stream), 20, 3, flush, stream)
    n0 = int(ex0._counts[0].item())
    out["single_vga"] = {"workload": "one 640x480 image, plain SIFT, no upsampling",
                         "ms_per_image": round(statistics.median(t0), 4), "keypoints": n0}
    js, _ = ex0.autotune_batch(vga, stream)
    torch.cuda.synchronize()
    t0t, _ = timed_steps(torch, lambda: ex0.extract_async(vga[0], stream), 20, 3, flush, stream)
    out["single_vga"]["autotune"] = {
        "untuned_ms_per_image": round(statistics.median(t0), 4),
        "tuned_ms_per_image": round(statistics.median(t0t), 4),
        "untuned_over_tuned": round(statistics.median(t0) / statistics.median(t0t), 4),
        "tuning": js, "chose_defaults": _is_default_tuning(js)}
    ex0.close()
    seq = synth.wide_baseline_pair(0)
    pair = _device_images(seq.images, torch)
    ex2 = pkg.Extractor(upsample=1, max_kpts=8192)
    ex2.set_tuning(tuning)
    t2, _ = timed_steps(torch, lambda: ex2.extract_batch_async(pair, stream), 10, 3, flush, stream)
    c2 = ex2._counts[:2].tolist()
    feats = [ex2._bufs[i].view(c2[i]) for i in range(2)]
    acc = matching.sequence_mma(feats, seq.homographies)
    # The library's tensor-core matcher on the pair's descriptors.
    da, db = feats[0].desc.contiguous(), feats[1].desc.contiguous()
    tm, _ = timed_steps(torch, lambda: ex2.match(da, db), 20, 3, flush, stream)
    m = ex2.match(da, db).cpu().numpy()
    ia = np.nonzero(m >= 0)[0]
    xy0 = np.stack([feats[0].x.cpu().numpy(), feats[0].y.cpu().numpy()], 1).astype(np.float64)
    xy1 = np.stack([feats[1].x.cpu().numpy(), feats[1].y.cpu().numpy()], 1).astype(np.float64)
    mm, nm = matching.mma(xy0, xy1, ia, m[ia], seq.homographies[1])
    # GPU MAGSAC++ on the matched keypoints (1,500 minimal samples, drawn once).
    mi = torch.from_numpy(ia).cuda()
    mj = torch.from_numpy(m[ia].astype(np.int64)).cuda()
    xa = torch.stack([feats[0].x[mi], feats[0].y[mi]], 1).contiguous()
    xb = torch.stack([feats[1].x[mj], feats[1].y[mj]], 1).contiguous()
    samples = torch.from_numpy(pkg.draw_samples(len(ia), 1500, seed=0)).cuda()
    tv, _ = timed_steps(torch, lambda: ex2.magsac(xa, xb, samples, sigma_max=1.0), 20, 3, flush, stream)
    rv = ex2.magsac(xa, xb, samples, sigma_max=1.0)
    Hg = rv["H"].cpu().numpy()
    h_, w_ = seq.images[0].shape
    corners = np.array([[0.0, 0.0], [w_, 0.0], [w_, h_], [0.0, h_]])
    corner_err = float(np.abs(matching.project(Hg, corners)
                              - matching.project(seq.homographies[1], corners)).max())
    gpu_magsac = {"what": "sift_magsac: 1500 minimal samples, FP64 normalised DLT, MAGSAC++ "
                          "loss (chi 4 dof, sigma_max 1 px), best by score",
                  "ms": round(statistics.median(tv), 4), "correspondences": int(len(ia)),
                  "inliers": int(rv["inliers"].sum().item()),
                  "corner_err_px": round(corner_err, 3)}
    out["pair"] = {"workload": "two 1600x1200 images (textured base + homography warp with "
                               "N(0, 0.02) noise), 2x upsampled, cap 8192, one batched call",
                   "ms_per_pair": round(statistics.median(t2), 4),
                   "pairs_per_s": round(1e3 / statistics.median(t2), 1), "keypoints": c2,
                   "matches": acc["matches"],
                   **{k: v for k, v in acc.items() if k.startswith("mma@")},
                   "gpu_matcher": {"what": "sift_match: fp16 tcgen05 similarity, mutual NN, "
                                           "ratio 0.8 both ways",
                                   "ms": round(statistics.median(tm), 4), "matches": nm,
                                   **{k: round(v, 4) for k, v in mm.items()}},
                   "gpu_magsac": gpu_magsac,
                   "ms_extract_match_verify": round(statistics.median(t2) + statistics.median(tm)
                                                    + statistics.median(tv), 4)}
    ex2.close()
    return out


# ------------------------------------------------------------ reference arm

def reference_arm(args, pool, n_workers, batch, budget_s=110.0):
    """The FP64 oracle timed on the host cores, on the timed workload's images:
    each step runs the first n_workers images of the batch (one per worker
    process), centre-cropped so that the warm-up and the K timed steps take
    about budget_s in total; the sample is stated in the output."""
    per_step = budget_s / (args.steps + args.warmup)
    crops, what = _oracle_sample(pool, n_workers, batch.images, per_step)
    mpix = sum(im.size for im in crops) / 1e6
    jobs = [(im, False, MAX_KPTS) for im in crops]
    for _ in range(args.warmup):
        pool.map(_oracle_one, jobs)
    times, kp = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = pool.map(_oracle_one, jobs)
        times.append(time.perf_counter() - t0)
        kp += sum(k for _, k in r)
    total = sum(times)
    value = mpix * args.steps / total
    return {"metric": METRIC, "value": round(value, 4), "unit": "Mpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * total / args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": {"workload": WORKLOAD},
            "keypoints_per_s": round(kp / total, 1),
            "cpu_baseline": {"value": round(value, 4), "unit": "Mpix/s", "cores": n_workers,
                             "kind": "oracle", "sample": "each step: " + what},
            "e2e": {"value": round(value, 4), "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------ main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the homography-sequence, single-image and image-pair runs")
    ap.add_argument("--minimal", action="store_true",
                    help="only the timed batch loop (for profiler launch lists)")
    ap.add_argument("--homography-loop", action="store_true",
                    help="only a timed loop of the homography-sequence batch (6 x 1000x750, "
                         "2x upsampled, cap 8000) at the given tuning (for profiler captures)")
    ap.add_argument("--pair-only", action="store_true",
                    help="only the single-image and wide-baseline pair runs (extraction, "
                         "matcher, MAGSAC++), e.g. for profiling those kernels")
    ap.add_argument("--keypoint-heavy", action="store_true",
                    help="only the keypoint-heavy run (4 x 1600x1200 textured, 2x upsampled), "
                         "e.g. for profiling the orientation and descriptor kernels")
    ap.add_argument("--images", type=int, default=N_IMAGES,
                    help=f"images per batch (default {N_IMAGES}; the first n of the batch)")
    ap.add_argument("--serving-requests", type=int, default=SERVING_REQUESTS)
    ap.add_argument("--tuning", default="", help='fixed tiles, e.g. {"blur_tile_rows": [32,...]}')
    ap.add_argument("--tuning-cache", default="",
                    help="tuning cache file for the batch autotuner (default: none, always search)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))

    if args.impl == "reference":
        if rank != 0:
            return
        n_workers = _oracle_workers()
        with _oracle_pool(n_workers) as pool:
            batch = replica_batch(0, args.images, pool)
            print(json.dumps(reference_arm(args, pool, n_workers, batch)))
        return

    if args.pair_only or args.keypoint_heavy or args.homography_loop:
        import torch
        import paper_2605_17869_gb300 as pkg
        stream = torch.cuda.current_stream()
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        tuning = args.tuning or '{"blur_tile_rows": [32, 32, 32, 32, 32]}'
        if args.homography_loop:
            print(json.dumps(homography_loop(torch, pkg, stream, tuning, max(1, args.steps),
                                             args.warmup)))
        elif args.keypoint_heavy:
            print(json.dumps({"keypoint_heavy": keypoint_heavy_side(
                torch, pkg, flush, stream, tuning, max(1, args.steps))}))
        else:
            print(json.dumps({"single_and_pair": other_configs(torch, pkg, flush, stream, tuning)}))
        return

    # The worker pool is started (spawn) before any GPU call; it generates the
    # inputs and later runs the oracle for the CPU baseline.
    n_workers = _oracle_workers()
    pool = _oracle_pool(n_workers)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    try:
        batch = replica_batch(rank, args.images, pool)
        res = gpu_arm(args, rank, world, pool, batch)
        if rank == 0:
            if not args.no_cpu_baseline and not args.minimal:
                res["cpu_baseline"] = cpu_baseline(pool, n_workers, batch.images)
            print(json.dumps(res))
    finally:
        pool.close()
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
