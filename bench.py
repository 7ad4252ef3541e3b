"""Benchmark: batched SIFT extraction on GB300 (one JSON line on stdout).

Workload (timed as `value`): a homography-sequence batch, 6 FP32 grayscale
images of 1000x750 (one seeded base image plus 5 warps by random
homographies with gain), 2x bilinear upsampled first octave, 8000 keypoints
cap, extracted in one sift_extract_batch call per step. value = input
megapixels per second over all ranks. Between timed steps L2 is flushed by
writing a 256 MB buffer (outside the timed events).

Also reported: keypoints/s; the same images through the per-image entry
point and the batched/per-image ratio; the same for a 64-image mixed-size
batch; serving images/s with p50/p99 latency under Poisson arrivals;
end-to-end throughput through the public API from pinned host buffers;
the blur kernel's achieved HBM bandwidth against the measured peak; and the
FP64 oracle timed on the host cores on a bounded sample.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-serving]
"""
from __future__ import annotations

import argparse
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
WORKLOAD = ("homography-sequence batch: 6 x 1000x750 FP32 grayscale (seeded base + 5 "
            "homography warps), 2x upsampled first octave, cap 8000 keypoints/image")
L2_FLUSH_BYTES = 256 << 20


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------ oracle (CPU)

def _oracle_one(args):
    img, upsample, max_kpts = args
    from oracle import sift_oracle as so
    t = time.perf_counter()
    r = so.extract(img, so.Params(upsample=bool(upsample), max_kpts=max_kpts))
    return time.perf_counter() - t, len(r)


def _oracle_pool(n):
    return mp.get_context("spawn").Pool(n)


def cpu_baseline(pool, n_workers, imgs, upsample=True, max_kpts=8000):
    t0 = time.perf_counter()
    res = pool.map(_oracle_one, [(im, upsample, max_kpts) for im in imgs])
    wall = time.perf_counter() - t0
    mpix = sum(im.size for im in imgs) / 1e6
    return {"value": round(mpix / wall, 4), "unit": "Mpix/s", "cores": n_workers,
            "kind": "oracle", "keypoints_per_s": round(sum(k for _, k in res) / wall, 1),
            "sample": f"{len(imgs)} images of the timed batch (1000x750, 2x upsampled), "
                      f"one image per worker process, {wall:.1f} s wall"}


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


# ------------------------------------------------------------ GPU arm

def _device_images(imgs, torch):
    return [torch.from_numpy(np.ascontiguousarray(im)).cuda() for im in imgs]


def _alg_blur_bytes(shapes, upsample, S=3, min_side=16):
    """Algorithmic bytes and pixels of all level-blur launches of one step.

    A level blur reads its source level once and writes the new level once
    (8 B per octave pixel); octave 0 has S + 2 of them. In octaves above 0 the
    first one also decimates: it reads one source value per output pixel and
    writes levels 0 and 1 (12 B per octave pixel), and S + 1 plain ones follow.
    Returns (bytes, pixels processed), the pixels summed over launches."""
    tot = px_tot = 0
    for (h, w) in shapes:
        if upsample:
            h, w = 2 * h, 2 * w
        o = 0
        while min(h, w) >= min_side:
            px = h * w
            tot += 8 * px * (S + 2) + (4 * px if o > 0 else 0)
            px_tot += px * (S + 2)
            h, w = h // 2, w // 2
            o += 1
    return tot, px_tot


# ------------------------------------------------------------ replicas
# Multi-GPU runs are independent replicas: rank r extracts its own batch (the
# homography sequence with seed index r); the only communication is a barrier
# and the max of the timed-region durations.

def replica_batch(rank, n_images):
    """The images rank `rank` processes (distinct per rank)."""
    return synth.homography_sequence(index=rank, n_warped=n_images - 1)


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


def _alg_class_bytes(shapes, upsample, S=3, min_side=16):
    """Algorithmic bytes of one step for the base blur and the extrema scan.
    Base: the input read once (4 B per input pixel) and level 0 of octave 0
    written once (4 B per octave pixel). Extrema: the S + 3 levels of every
    octave read once (the DoG is formed on the fly) plus the candidate bitmap
    (S bits per octave pixel)."""
    base = ext = 0
    for (h, w) in shapes:
        H, W = (2 * h, 2 * w) if upsample else (h, w)
        base += 4 * h * w + 4 * H * W
        while min(H, W) >= min_side:
            ext += 4 * (S + 3) * H * W + S * H * W // 8
            H, W = H // 2, W // 2
    return {"base": base, "extrema": ext}


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


def serving_bench(torch, pkg, rates, n_req, budget=8 << 30):
    pool = {}
    for (h, w) in ((480, 640), (1080, 1920), (2160, 3840)):
        pool[(h, w)] = [torch.from_numpy(synth.serving_image(h, w, i)).cuda() for i in range(2)]
    ex = pkg.Extractor(max_kpts=8192)
    srv = pkg.Server(ex, budget_bytes=budget, max_slots=256)
    # warm-up: one of each size
    for k in pool:
        t = srv.submit(pool[k][0])
        srv.result(t)
        srv.release(t)
    out = []
    for lam in rates:
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
        out.append({"rate_per_s": lam, "requests": n_req, "images_per_s": round(n_req / span, 1),
                    "mpix_per_s": round(px / 1e6 / span, 1),
                    "p50_ms": round(lat[len(lat) // 2], 3),
                    "p99_ms": round(lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)], 3)})
    srv.close()
    ex.close()
    return {"workload": "Poisson arrivals, 640x480 (50%) / 1920x1080 (35%) / 3840x2160 (15%), "
                        "8 GB device-memory budget, no upsampling, cap 8192",
            "points": out}


def gpu_arm(args, rank, world, pool, n_workers):
    import torch
    import paper_2605_17869_gb300 as pkg

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    seq = replica_batch(rank, args.images)
    imgs_np = seq.images
    shapes = [im.shape for im in imgs_np]
    imgs = _device_images(imgs_np, torch)
    mpix = sum(h * w for h, w in shapes) / 1e6
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    ex = pkg.Extractor(upsample=1, max_kpts=8000)
    if args.tuning:
        ex.set_tuning(args.tuning)
        tuning = ex.get_tuning()
    else:
        tuning = ex.autotune(1500, 2000)

    if args.minimal:
        def step_min():
            ex.extract_batch_async(imgs, stream)
        times, _ = timed_steps(torch, step_min, args.steps, args.warmup, flush, stream)
        return {"metric": METRIC, "value": round(mpix * args.steps / (sum(times) / 1e3), 2),
                "unit": "Mpix/s", "mode": "minimal (timed loop only)", "images": len(imgs),
                "ms_per_step": round(sum(times) / args.steps, 4),
                "gpu_launches_per_step": ex.launch_count(), "tuning": tuning}, imgs_np

    def step():
        ex.extract_batch_async(imgs, stream)

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = Clocks(dev)
    clocks.start()
    times, wall = timed_steps(torch, step, args.steps, args.warmup, flush, stream)
    clock_info = clocks.stop()
    counts = ex._counts[:len(imgs)].tolist()
    kpts = sum(counts)
    accuracy = None
    if rank == 0:
        feats = [ex._bufs[i].view(counts[i]) for i in range(len(imgs))]
        accuracy = {"what": "image 0 matched to each warped image of the timed batch; MMA against "
                            "the known homographies (harness: torch mutual NN + ratio 0.8)",
                    **matching.sequence_mma(feats, seq.homographies)}
    launches_per_step = ex.launch_count()
    total_ms = sum(times)
    if world > 1:
        total_ms = max_over_ranks(total_ms, "cuda")
    value = whole_job_value(world, mpix, args.steps, total_ms)

    # Per-image path on the same images.
    def step_single():
        for im in imgs:
            ex.extract_async(im, stream)
    t_single, _ = timed_steps(torch, step_single, max(3, args.steps // 2), 2, flush, stream)
    per_image = mpix * len(t_single) / (sum(t_single) / 1e3)

    # Per-kernel device times (profiled graph: an event pair around every launch).
    ex.set_profiling(True)
    step()
    torch.cuda.synchronize()
    acc = {}
    reps = max(3, args.steps // 2)
    for _ in range(reps):
        flush.zero_()
        step()
        for k, (ms, n) in ex.kernel_times().items():
            a = acc.setdefault(k, [0.0, 0])
            a[0] += ms
            a[1] += n
    ex.set_profiling(False)
    blur_ms, blur_n = acc["blur"]
    alg_step, px_step = _alg_blur_bytes(shapes, True)
    alg_total = alg_step * reps
    peak, peak_kind = _peaks()
    achieved = alg_total / (blur_ms / 1e3) / 1e9 if blur_ms > 0 else 0.0
    kernel_share = {k: round(v[0] / reps, 4) for k, v in acc.items()}
    # DRAM bytes per launch: the per-pixel DRAM traffic of a captured level-blur
    # launch (a 12-image batch whose levels exceed L2) times the pixels an
    # average launch of this workload processes; taken only while the kernel
    # source is the one the counters were read from.
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "blur_level_traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tj = json.load(f)
        import hashlib
        src = open(os.path.join(ROOT, "paper_2605_17869_gb300", "csrc", "pyramid.cu"), "rb").read()
        if tj.get("pyramid_cu_sha256") == hashlib.sha256(src).hexdigest() and blur_n:
            traffic = int(tj["dram_bytes_per_px"] * px_step * reps / blur_n)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": "k_blur (pyramid level blur)",
                "alg_bytes_per_launch": int(alg_total / max(1, blur_n)),
                "launch_ms_avg": round(blur_ms / max(1, blur_n), 5),
                "peak_source": "hbm_gbs, " + ("of measured (MEASURED_PEAKS.json)"
                                              if peak_kind == "measured" else "of fallback")}

    # Per-class rooflines (CUDA-event time of each class inside the graph).
    cls_bytes = _alg_class_bytes(shapes, True)
    cls_bytes["blur"] = alg_step
    nominal = 8000.0
    per_class = {}
    for k in ("blur", "base", "extrema"):
        ms = acc.get(k, (0.0, 0))[0] / reps
        if ms > 0:
            gbs = cls_bytes[k] / (ms / 1e3) / 1e9
            per_class[k] = {"alg_bytes_per_step": int(cls_bytes[k]), "ms_per_step": round(ms, 4),
                            "achieved_gbs": round(gbs, 1), "frac_of_measured": round(gbs / peak, 4),
                            "frac_of_nominal_8tbs": round(gbs / nominal, 4)}
    for k in ("keypoint", "descriptor"):
        ms = acc.get(k, (0.0, 0))[0] / reps
        if ms > 0:
            per_class[k] = {"ms_per_step": round(ms, 4),
                            "keypoints_per_s": round(kpts / (ms / 1e3), 1)}

    # End to end: pinned host images -> device -> extract -> results back in one packed copy.
    # Two handles on two streams take alternate steps: step k + 1's upload and launches are
    # queued before step k's results are read back, so the GPU does not wait for the host.
    # Every step still uploads its own inputs and reads back its own results. No L2 flush:
    # a step's working set (its pyramid, ~0.6 GB) is far larger than L2.
    host = [torch.from_numpy(np.ascontiguousarray(im)).pin_memory() for im in imgs_np]
    h2d = sum(h.numel() * 4 for h in host)
    ex_b = pkg.Extractor(upsample=1, max_kpts=8000)
    ex_b.set_tuning(json.dumps(tuning) if isinstance(tuning, dict) else tuning)
    lanes = [(e, torch.cuda.Stream(), [torch.empty_like(h, device="cuda") for h in host])
             for e in (ex, ex_b)]

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

    for it in range(args.warmup):
        submit(lanes[it % 2])
        collect(lanes[it % 2])
    torch.cuda.synchronize()
    n_e2e = max(3, args.steps // 2)
    d2h_bytes = []
    t0 = time.perf_counter()
    submit(lanes[0])
    for it in range(n_e2e):
        if it + 1 < n_e2e:
            submit(lanes[(it + 1) % 2])
        d2h_bytes.append(collect(lanes[it % 2]))
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    ex_b.close()
    e2e = {"value": round(world * mpix * n_e2e / t_e2e, 3), "unit": "Mpix/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(np.mean(d2h_bytes)),
           "steps": n_e2e,
           "api": "Extractor.extract_batch_async (sift_extract_batch) from pinned host buffers, "
                  "results by Extractor.download (sift_pack_outputs + one copy); two handles on "
                  "two streams take alternate steps (step k+1 queued before step k is read back)"}

    # Mixed-size 64-image batch (batching workload): batched vs per-image.
    mixed = None
    if rank == 0 and not args.no_mixed:
        mimgs_np = pool.map(_mixed_one, list(range(64))) if pool else [
            _mixed_one(i) for i in range(64)]
        mimgs = _device_images(mimgs_np, torch)
        mmpix = sum(im.size for im in mimgs_np) / 1e6
        exm = pkg.Extractor(max_kpts=8192)
        exm.set_tuning(tuning)
        tb, _ = timed_steps(torch, lambda: exm.extract_batch_async(mimgs, stream), 5, 2, flush,
                            stream)
        mcounts = exm._counts[:64].tolist()

        def single_all():
            for im in mimgs:
                exm.extract_async(im, stream)
        ts, _ = timed_steps(torch, single_all, 3, 1, flush, stream)
        mixed = {"workload": "64 mixed-size images, long side 480-1600, aspect 4:3/3:4/16:9, "
                             "1/f texture, no upsampling, cap 8192",
                 "batched_mpix_s": round(mmpix * len(tb) / (sum(tb) / 1e3), 1),
                 "per_image_mpix_s": round(mmpix * len(ts) / (sum(ts) / 1e3), 1),
                 "keypoints_per_s": round(sum(mcounts) * len(tb) / (sum(tb) / 1e3), 1),
                 "ms_per_batch": round(statistics.mean(tb), 3)}
        mixed["batched_vs_per_image"] = round(mixed["batched_mpix_s"] / mixed["per_image_mpix_s"], 2)
        exm.close()

    configs = None
    if rank == 0 and not args.no_configs:
        configs = other_configs(torch, pkg, flush, stream, tuning)
        configs["dsp_rootsift"] = dsp_variant(torch, pkg, imgs, mpix, flush, stream, tuning,
                                              seq, max(10, args.steps // 4))

    serving = None
    if rank == 0 and not args.no_serving:
        serving = serving_bench(torch, pkg, (50, 200, 1000, 2000), 200)

    res = {
        "metric": METRIC, "value": round(value, 2), "unit": "Mpix/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "images_per_step_per_gpu": len(imgs),
                   "input_mpix_per_step_per_gpu": round(mpix, 3),
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{world} (independent images per rank)",
                   "tuning": tuning},
        "keypoints_per_s": round(world * kpts * args.steps / (total_ms / 1e3), 1),
        "keypoints_per_step_per_gpu": kpts,
        "per_image_mpix_s": round(per_image, 2),
        "batched_vs_per_image": round(value / world / per_image, 3),
        "wall_s_timed_region": round(wall, 3),
        "gpu_launches": launches_per_step * args.steps,
        "gpu_launches_per_step": launches_per_step,
        "kernel_ms_per_step": kernel_share,
        "roofline": roofline,
        "per_class_roofline": per_class,
        "e2e": e2e,
        "clocks": clock_info,
        "accuracy": accuracy,
        "mixed_batch": mixed,
        "single_and_pair": configs,
        "serving": serving,
    }
    return res, imgs_np


def dsp_variant(torch, pkg, imgs, mpix, flush, stream, tuning, seq, steps):
    """The timed batch again with DSP pooling and RootSIFT (§3.2): throughput,
    per-class device time and matching accuracy."""
    ex = pkg.Extractor(upsample=1, max_kpts=8000, dsp=1, rootsift=1)
    ex.set_tuning(tuning)
    t, _ = timed_steps(torch, lambda: ex.extract_batch_async(imgs, stream), steps, 3, flush, stream)
    counts = ex._counts[:len(imgs)].tolist()
    feats = [ex._bufs[i].view(counts[i]) for i in range(len(imgs))]
    acc = matching.sequence_mma(feats, seq.homographies)
    ex.set_profiling(True)
    ex.extract_batch_async(imgs, stream)
    torch.cuda.synchronize()
    acc_t = {}
    for _ in range(3):
        flush.zero_()
        ex.extract_batch_async(imgs, stream)
        for k, (ms, n) in ex.kernel_times().items():
            acc_t[k] = acc_t.get(k, 0.0) + ms / 3
    ex.close()
    return {"workload": "the timed batch with dsp=1, rootsift=1",
            "ms_per_step": round(statistics.mean(t), 4),
            "mpix_s": round(mpix * len(t) / (sum(t) / 1e3), 1),
            "keypoints_per_s": round(sum(counts) * len(t) / (sum(t) / 1e3), 1),
            "kernel_ms_per_step": {k: round(v, 4) for k, v in acc_t.items()},
            "matches": acc["matches"], **{k: v for k, v in acc.items() if k.startswith("mma@")}}


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


def _mixed_one(i):
    (h, w) = synth.mixed_batch_shapes(64)[i]
    return synth.make_image(synth.rng_for(3, i), h, w, fractal_std=0.05)


# ------------------------------------------------------------ reference arm

def _center_crop(im, h, w):
    y0 = (im.shape[0] - h) // 2
    x0 = (im.shape[1] - w) // 2
    return np.ascontiguousarray(im[y0:y0 + h, x0:x0 + w])


def reference_arm(args, pool, n_workers, budget_s=110.0):
    """The FP64 oracle timed on the host cores. Each step runs the 6 images of
    the batch (one per worker process), centre-cropped so that the warm-up and
    the K timed steps take about budget_s in total (full images when K is
    small); the crop is stated in the output."""
    seq = synth.homography_sequence(index=0)
    full = seq.images
    H, W = full[0].shape
    # Calibrate on a 1/9-area crop (also warms up the workers).
    ch, cw = H // 3, W // 3
    t0 = time.perf_counter()
    pool.map(_oracle_one, [(_center_crop(im, ch, cw), True, 8000) for im in full[:n_workers]])
    t_cal = time.perf_counter() - t0
    per_step = budget_s / (args.steps + args.warmup)
    frac = min(1.0, per_step / max(1e-6, 9.0 * t_cal))
    h = max(64, min(H, int(round(H * math.sqrt(frac)))))
    w = max(64, min(W, int(round(W * math.sqrt(frac)))))
    imgs = [_center_crop(im, h, w) for im in full]
    mpix = sum(im.size for im in imgs) / 1e6
    for _ in range(args.warmup):
        pool.map(_oracle_one, [(im, True, 8000) for im in imgs[:n_workers]])
    times, kp = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = pool.map(_oracle_one, [(im, True, 8000) for im in imgs])
        times.append(time.perf_counter() - t0)
        kp += sum(k for _, k in r)
    total = sum(times)
    value = mpix * args.steps / total
    crop = "full 1000x750 images" if (h, w) == (H, W) else f"centre {w}x{h} crops"
    sample = (f"each step: the {len(imgs)} images of the timed batch ({crop}, 2x upsampled) "
              f"through the FP64 oracle, one image per worker process ({n_workers} workers)")
    return {"metric": METRIC, "value": round(value, 4), "unit": "Mpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * total / args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": {"workload": WORKLOAD},
            "keypoints_per_s": round(kp / total, 1),
            "cpu_baseline": {"value": round(value, 4), "unit": "Mpix/s", "cores": n_workers,
                             "kind": "oracle", "sample": sample},
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
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the single-image and image-pair latency runs")
    ap.add_argument("--minimal", action="store_true",
                    help="only the timed batch loop (for profiler launch lists)")
    ap.add_argument("--pair-only", action="store_true",
                    help="only the single-image and wide-baseline pair runs (extraction, "
                         "matcher, MAGSAC++), e.g. for profiling those kernels")
    ap.add_argument("--images", type=int, default=6, help="images per batch (default 6)")
    ap.add_argument("--tuning", default="", help='fixed tiles, e.g. {"blur_tile_rows": [32,...]}')
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))

    if args.impl == "reference":
        if rank != 0:
            return
        n_workers = min(6, os.cpu_count() or 1)
        with _oracle_pool(n_workers) as pool:
            print(json.dumps(reference_arm(args, pool, n_workers)))
        return

    if args.pair_only:
        import torch
        import paper_2605_17869_gb300 as pkg
        stream = torch.cuda.current_stream()
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        tuning = args.tuning or '{"blur_tile_rows": [32, 32, 32, 32, 32]}'
        print(json.dumps({"single_and_pair": other_configs(torch, pkg, flush, stream, tuning)}))
        return

    # The oracle's worker pool is started (spawn) before any GPU call.
    n_workers = min(6, os.cpu_count() or 1)
    pool = _oracle_pool(n_workers) if rank == 0 and not args.minimal else None
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    try:
        res, imgs_np = gpu_arm(args, rank, world, pool, n_workers)
        if rank == 0:
            if not args.no_cpu_baseline and not args.minimal:
                res["cpu_baseline"] = cpu_baseline(pool, n_workers, imgs_np)
            print(json.dumps(res))
    finally:
        if pool is not None:
            pool.close()
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
