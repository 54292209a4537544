#!/usr/bin/env python3
"""Benchmark of the MCL particle-weight update on one GB300 per process.

A step is one MCL iteration of the full-update workload (600 particles x 64
shared pixels of a 400x400 observation, focal 555.6, 64 stratified + 128
importance samples per ray, Eq. 5 uncertainty, Eq. 6 rejection weights, FP64
normalisation, systematic resampling, the motion model and the position
spread of the refinement test).  The metric is ray-samples per second
(rays x composited samples / time) with the MCL-update milliseconds.  The
headline value is the plain FP32 form (the paper's precision); the BF16,
FP8 and learned-proposal + FP8 forms are reported beside it (key "forms")
with their speed-up, their roofline and their error against the FP64
oracle, and the equal-pose-error comparison runs on the analytic room map.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--no-extra] [--no-cpu-baseline] [--sweeps]
Under torchrun every rank localises its own query (its own seed): weak
scaling, no data-path collective.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WL = dict(workload="full update: 600 particles x 64 px of 400x400, 64+128 samples/ray",
          N=600, B=64, W=400, H=400, focal=555.6, n_coarse=64, n_fine=128, level=2,
          sigma_t=0.05, sigma_yaw=0.05, map_seed=0)
MAC_PER_SAMPLE_FP32 = 593408   # unfused MLP: 8 trunk layers, sigma, feature, rgb head
METRIC = "MCL update ms and ray-samples/s vs plain FP32 GPU form, at stated pose/RGB error"
UNIT = "ray-samples/s"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def profiled_traffic(name: str, sources):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    of a kernel from profiles/<name>.json (written beside the ncu summary
    profiles/<name>.md), or None when that file is missing or the kernel's
    sources have changed since the capture (the file records their hash)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", name + ".json")
    if not os.path.exists(path):
        return None
    h = hashlib.sha256()
    for src in sources:
        with open(os.path.join(ROOT, "paper_2406_12202_gb300", "csrc", src), "rb") as f:
            h.update(f.read())
    with open(path) as f:
        rec = json.load(f)
    if rec.get("source_sha16") != h.hexdigest()[:16]:
        return None
    v = rec.get("traffic_bytes_per_launch")
    return float(v) if v is not None else None


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", gpu_id], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        self.t0 = self.t1 = None

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = []
        for line in self.tmp.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                frac = float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                rows.append((ts + frac, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        os.unlink(self.tmp.name)
        inside = [r for r in rows if self.t0 is not None and self.t0 - 0.15 <= r[0] <= self.t1 + 0.15]
        use = inside if inside else rows[-3:]
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in use for n, v in zip(names, r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": max(r[2] for r in use),
                "reasons": reasons, "samples": len(use), "in_timed_region": bool(inside)}


# --------------------------------------------------------------- CPU oracle
def oracle_rate(n_particles: int, seed: int = 0):
    """Time the FP64 oracle on n_particles x B pixels of the workload (synthetic
    observation).  Returns (ray-samples/s, seconds, threads)."""
    import numpy as np
    import oracle
    import synth
    wl = WL
    blob = synth.he_init_weights(wl["map_seed"])
    P = synth.random_particles(seed, wl["N"])[0][:n_particles].astype(np.float32).astype(np.float64)
    img = synth.smooth_image(seed, wl["W"], wl["H"]).astype(np.float64)
    px = synth.pixel_set(seed, wl["W"], wl["H"], wl["B"])
    f = float(np.float32(wl["focal"]))
    K4 = (f, f, wl["W"] / 2, wl["H"] / 2)
    opts = oracle.make_opts(n_coarse=wl["n_coarse"], n_fine=wl["n_fine"])
    t = time.perf_counter()
    oracle.update(blob, P, img, K4, 1, px, opts)
    dt = time.perf_counter() - t
    rs = n_particles * wl["B"] * (wl["n_coarse"] + wl["n_fine"])
    return rs / dt, dt, oracle.num_threads()


def cpu_baseline(target_s: float = 15.0):
    r1, dt1, thr = oracle_rate(1)
    n = max(1, min(WL["N"], int(target_s / max(dt1, 1e-3))))
    rate, dt, thr = oracle_rate(n)
    return {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": f"{n} of {WL['N']} particles x {WL['B']} px x "
                      f"{WL['n_coarse'] + WL['n_fine']} samples ({dt:.1f} s, FP64 C + OpenMP)"}


def run_reference(args):
    """The oracle as it stands, timed on the host cores: each step is a bounded
    sample (4 particles) of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    n = 4
    for _ in range(args.warmup):
        oracle_rate(n)
    times = []
    for k in range(args.steps):
        rate, dt, thr = oracle_rate(n, seed=k)
        times.append(dt)
    rs = n * WL["B"] * (WL["n_coarse"] + WL["n_fine"])
    value = rs * len(times) / sum(times)
    sample = f"{n} of {WL['N']} particles x {WL['B']} px per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WL["workload"], "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- further workloads
def _pct(v, q):
    v = sorted(v)
    if not v:
        return None
    k = min(len(v) - 1, max(0, int(round(q / 100.0 * (len(v) - 1)))))
    return v[k]


def _pose_error(est, gt_xyz, gt_yaw):
    d = math.sqrt(sum((est[i] - gt_xyz[i]) ** 2 for i in range(3)))
    y = abs((est[3] - gt_yaw + math.pi) % (2 * math.pi) - math.pi)
    return d, math.degrees(y)


def _update_latencies(recs):
    """Per-update latencies (ms) from the iteration start times of a run."""
    t = [r["t_start_ns"] for r in recs]
    return [(b - a) / 1e6 for a, b in zip(t[:-1], t[1:])]


def run_coarse_to_fine(M, img, K, seed, prec, fp32_replay=True):
    """Three levels (100, 200, 400 px wide: factors 4, 2, 1) with 16 / 32 /
    64 pixels, 1500 initial particles, survivors after rejection decide the
    next count, 20 MCL iterations with sigma_t = sigma_yaw = 0.05, one
    device-driven run under a CUDA graph.  The plain FP32 form is timed on
    the same sequence of (particles, pixels, level) through mcl_update."""
    import numpy as np
    import torch
    import synth
    N0, iters = 1500, 20
    gm = M.Map(synth.he_init_weights(0), max_rays=N0 * 64, max_samples=192, max_particles=N0,
               max_queries=1)
    P = torch.tensor(synth.random_particles(seed + 1, N0)[0], dtype=torch.float32,
                     device="cuda").reshape(1, N0, 12)
    _, gxyz, gyaw = synth.gt_pose(seed)
    sch = M.schedule([0, 1, 2], [16, 32, 64], [N0, 1000, 600], n_min=100, iter_caps=[7, 7, 6],
                     refine=[0.05, 0.01, 0.0], iterations=iters, sigma_t=0.05, sigma_yaw=0.05)
    opts = M.UpdateOptions(n_coarse=64, n_fine=128, precision=prec, seed=seed)
    gm.localize(P.clone(), [N0], [img], K, sch, opts, use_graph=True)      # build + warm
    torch.cuda.synchronize()
    Pw = P.clone()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    log, fin = gm.localize(Pw, [N0], [img], K, sch, opts, use_graph=True)
    b.record()
    torch.cuda.synchronize()
    total = a.elapsed_time(b)
    recs = M.Map.decode_log(log, 1, iters)[0]
    lat = _update_latencies(recs)
    perr, yerr = _pose_error(recs[-1]["est"], gxyz, gyaw)
    out = {"workload": "coarse-to-fine: 3 levels (1/4, 1/2, 1 of 400x400) x 16/32/64 px, "
                       "1500 initial particles, 20 iterations, 64+128 samples",
           "precision": prec, "run_ms": total, "ms_per_update": total / iters,
           "update_ms_p50": _pct(lat, 50), "update_ms_p99": _pct(lat, 99),
           "particles_per_iteration": [r["n_particles"] for r in recs],
           "levels": [r["level"] for r in recs],
           "final_position_error": perr, "final_yaw_error_deg": yerr,
           "note": "seeded He-init map: a high-frequency random field, so pose error is "
                   "reported, not expected to be small"}
    if fp32_replay:
        o32 = M.UpdateOptions(n_coarse=64, n_fine=128, precision="fp32")
        Pf = P.reshape(N0, 12)
        e32 = []
        for t, r in enumerate(recs):
            n, B, lev = r["n_particles"], r["n_pixels"], r["level"]
            f = 4 >> lev
            px = M.draw_pixels(img.shape[1] // f, img.shape[0] // f, B, seed, t)
            x, y = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            x.record()
            gm.update(Pf[:n].contiguous(), img, K, lev, px, o32)
            y.record()
            torch.cuda.synchronize()
            e32.append(x.elapsed_time(y))
        out["fp32_form_ms_per_update_same_sizes"] = sum(e32) / len(e32)
        out["speedup_vs_fp32_form"] = out["fp32_form_ms_per_update_same_sizes"] / out["ms_per_update"]
    gm.close()
    return out


def run_ablation(M, img, K, seed, prec):
    """Module ablation of Table 3 (Sec. IV-C) on synthetic data: particle
    rejection (Eq. 6 with F, or Eq. 4 with F = 1) x coarse-to-fine (three
    levels 1/4, 1/2, 1 with 16 / 32 / 64 px and a survivor-driven particle
    count, or the full level with 64 px and a fixed count), 20 iterations
    from 1500 particles; ms per update and final pose error, one device run
    each under a CUDA graph."""
    import torch
    import synth
    N0, iters = 1500, 20
    gm = M.Map(synth.he_init_weights(0), max_rays=N0 * 64, max_samples=192, max_particles=N0,
               max_queries=1)
    _, gxyz, gyaw = synth.gt_pose(seed)
    P0 = torch.tensor(synth.random_particles(seed + 1, N0)[0], dtype=torch.float32,
                      device="cuda").reshape(1, N0, 12)
    out = {}
    for rej in (True, False):
        for c2f in (True, False):
            if c2f:
                sch = M.schedule([0, 1, 2], [16, 32, 64], [N0, 1000, 600], n_min=100,
                                 iter_caps=[7, 7, 6], refine=[0.05, 0.01, 0.0], iterations=iters)
            else:
                sch = M.schedule([2], [64], [N0], n_min=N0, iter_caps=[iters], refine=[0.0],
                                 iterations=iters)
            opts = M.UpdateOptions(n_coarse=64, n_fine=128, precision=prec, seed=seed,
                                   use_rejection=rej)
            gm.localize(P0.clone(), [N0], [img], K, sch, opts, use_graph=True)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            log, _ = gm.localize(P0.clone(), [N0], [img], K, sch, opts, use_graph=True)
            b.record()
            torch.cuda.synchronize()
            recs = M.Map.decode_log(log, 1, iters)[0]
            perr, yerr = _pose_error(recs[-1]["est"], gxyz, gyaw)
            key = ("rejection" if rej else "no_rejection") + "+" + ("coarse_to_fine" if c2f else "single_level")
            out[key] = {"ms_per_update": a.elapsed_time(b) / iters, "final_position_error": perr,
                        "final_yaw_error_deg": yerr}
    gm.close()
    return out


def run_proposal_fp8(M, gm, img, K, seed, steps, warmup, wl):
    """Learned proposal + FP8 MLP on the full-update workload: the proposal
    (4 x 64, gamma with 6 frequencies) is distilled on the GPU from the
    64 + 128 FP32 sampler over 2000 seeded poses x 64 pixels (128,000 rays,
    64 bins); then 64 proposal samples -> 32 guided + 32 importance samples
    per ray through the FP8 MLP.  Returns the timing and the trained proposal
    weights."""
    import numpy as np
    import torch
    import synth
    N, Bpx, W, H = wl["N"], wl["B"], wl["W"], wl["H"]
    Ptr = torch.tensor(synth.random_particles(seed + 77, 2000)[0], dtype=torch.float32, device="cuda")
    pxtr = torch.tensor(synth.pixel_set(seed + 78, W, H, Bpx), dtype=torch.int32, device="cuda")
    gm.proposal_set(synth.proposal_init_weights(0))
    full32 = M.UpdateOptions(n_coarse=64, n_fine=128, precision="fp32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = gm.proposal_train(Ptr, pxtr, K, wl["level"], full32, epochs=8, batch_rays=4096,
                               n_bins=64, lr=3e-3, lr_end=1e-4, seed=seed)
    train_s = time.perf_counter() - t0
    prop = M.UpdateOptions(n_coarse=64, n_fine=32, precision="fp8", use_proposal=True,
                           n_proposal=64, n_guided=32)
    P = torch.tensor(synth.random_particles(seed, N)[0], dtype=torch.float32, device="cuda")
    pxs = [torch.tensor(synth.pixel_set(seed + 7 * t, W, H, Bpx), dtype=torch.int32, device="cuda")
           for t in range(steps + warmup)]
    out = {"logw": torch.empty(N, device="cuda"), "w": torch.empty(N, dtype=torch.float64, device="cuda"),
           "mask": torch.empty(N, dtype=torch.uint8, device="cuda")}
    idx = torch.empty(N, dtype=torch.int32, device="cuda")
    Pn = torch.empty_like(P)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    def timed_prop(fused):
        gm.set_fused_epilogue(fused)
        ms = []
        for t in range(warmup + steps):
            if t == warmup:
                gm.profile_read(reset=True)
                gm.profile(True)
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            gm.update(P, img, K, wl["level"], pxs[t], prop, out=out)
            gm.resample(out["w"], N, 0.5, idx=idx)
            M.predict(P, idx, N, wl["sigma_t"], wl["sigma_yaw"], seed, t, out=Pn)
            b.record()
            torch.cuda.synchronize()
            if t >= warmup:
                ms.append(a.elapsed_time(b))
        phases, _ = gm.profile_read(reset=True)
        gm.profile(False)
        gm.set_fused_epilogue(False)
        return sum(ms) / len(ms), phases

    mean_ms, phases = timed_prop(False)
    fused_ms, fused_phases = timed_prop(True)
    res = {"workload": "learned proposal (64 -> 32 guided + 32 importance) + FP8 MLP, "
                       "600 particles x 64 px of 400x400",
           "ms_per_step": mean_ms, "ray_samples_per_s": N * Bpx * 64 / (mean_ms / 1e3),
           "ray_samples_note": "composited samples per ray: 32 guided + 32 importance",
           "phases_ms_per_step": {k: v / steps for k, v in phases.items()},
           "phase_note": "sample = proposal MLP + inverse-CDF sampling; mlp_coarse = NeRF MLP on "
                         "the guided samples",
           "ray_epilogue": "separate sampling / composite kernels (the default)",
           "fused_epilogue": {"ms_per_step": fused_ms,
                              "ray_samples_per_s": N * Bpx * 64 / (fused_ms / 1e3),
                              "phases_ms_per_step": {k: v / steps for k, v in fused_phases.items()}},
           "train_s": train_s, "train_rays": 2000 * Bpx,
           "train_loss_first_last": [float(losses[0]), float(losses[-1])]}
    return res, gm.proposal_get()


def run_batched(M, seed, W, H, focal, use_proposal_blob=None):
    """16 independent queries on one map, N_q ~ U{1000..4000} (seeded), own
    ground-truth poses, 3 levels (16 / 32 / 64 px), 100 iterations, FP8 MLP
    with the learned proposal, one CUDA graph for the whole run; per-update
    latency from the GPU timer at the start of every iteration."""
    import numpy as np
    import torch
    import synth
    Q, stride, iters = 16, 4000, 100
    rng = np.random.Generator(np.random.PCG64(seed + 4242))
    n0 = [int(v) for v in rng.integers(1000, 4001, size=Q)]
    blob = synth.he_init_weights(0)
    gm = M.Map(blob, max_rays=Q * stride * 16, max_samples=96, max_particles=Q * stride,
               max_queries=Q)
    K = M.intrinsics(focal, focal, W / 2, H / 2, W, H)
    if use_proposal_blob is not None:
        gm.proposal_set(use_proposal_blob)
    # observations: BF16 renders of the full image at each query's ground truth
    allpx = np.stack(np.meshgrid(np.arange(W), np.arange(H), indexing="xy"), -1).reshape(-1, 2)
    o16 = M.UpdateOptions(n_coarse=64, n_fine=32, precision="bf16")
    imgs = []
    for q in range(Q):
        gt = torch.tensor(synth.gt_pose(seed + 100 + q)[0][None], dtype=torch.float32, device="cuda")
        im = torch.empty(H * W, 3, device="cuda")
        for c0 in range(0, H * W, 40000):
            pc = torch.tensor(allpx[c0:c0 + 40000], dtype=torch.int32, device="cuda")
            im[c0:c0 + pc.shape[0]] = gm.render(gt, K, 2, pc, o16)
        imgs.append(im.reshape(H, W, 3).contiguous())
    P = torch.zeros(Q, stride, 12, dtype=torch.float32, device="cuda")
    for q in range(Q):
        P[q, :n0[q]] = torch.tensor(synth.random_particles(seed + 200 + q, n0[q])[0], dtype=torch.float32)
    sch = M.schedule([0, 1, 2], [16, 32, 64], [stride, 2000, 500], n_min=64, iter_caps=[34, 33, 33],
                     refine=[0.05, 0.01, 0.0], iterations=iters, sigma_t=0.05, sigma_yaw=0.05)
    opts = M.UpdateOptions(n_coarse=64, n_fine=32, precision="fp8", seed=seed,
                           use_proposal=use_proposal_blob is not None, n_proposal=64, n_guided=32)
    gm.localize(P.clone(), n0, imgs, K, sch, opts, use_graph=True)        # capture + warm
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Pw = P.clone()
    a.record()
    log, fin = gm.localize(Pw, n0, imgs, K, sch, opts, use_graph=True)
    b.record()
    torch.cuda.synchronize()
    total = a.elapsed_time(b)
    recs = M.Map.decode_log(log, Q, iters)
    lat = _update_latencies(recs[0])
    samples = sum(r["n_particles"] * r["n_pixels"] * 64 for q in range(Q) for r in recs[q])
    # work of each update (rays of all queries) against its latency: the
    # queries move between levels independently, so an update's work varies
    rays = [sum(recs[q][t]["n_particles"] * recs[q][t]["n_pixels"] for q in range(Q))
            for t in range(iters - 1)]
    per_mray = [l / (r / 1e6) for l, r in zip(lat, rays) if r > 0]
    corr = float(np.corrcoef(np.array(lat), np.array(rays, dtype=float))[0, 1]) if len(lat) > 2 else None
    # least-squares latency = fixed + per-ray x rays: the fixed part is what
    # launches, idle grid blocks and the graph's control add to an update
    fit = np.polyfit(np.array(rays, dtype=float) / 1e6, np.array(lat), 1) if len(lat) > 2 else None
    errs = [_pose_error(recs[q][-1]["est"], synth.gt_pose(seed + 100 + q)[1],
                        synth.gt_pose(seed + 100 + q)[2]) for q in range(Q)]
    gm.close()
    return {"workload": "16 queries, N ~ U{1000..4000}, 3 levels x 16/32/64 px of 400x400, "
                        "100 iterations, FP8 + learned proposal (64 -> 32 + 32), one CUDA graph",
            "initial_particles": n0, "run_ms": total, "ms_per_batched_update": total / iters,
            "update_ms_p50": _pct(lat, 50), "update_ms_p99": _pct(lat, 99),
            "rays_per_update_p50": _pct(rays, 50), "rays_per_update_p99": _pct(rays, 99),
            "ms_per_million_rays_p50": _pct(per_mray, 50),
            "ms_per_million_rays_p99": _pct(per_mray, 99),
            "latency_vs_rays_correlation": corr,
            "latency_fit_ms": ({"fixed_per_update": float(fit[1]), "per_million_rays": float(fit[0])}
                               if fit is not None else None),
            "ray_samples_per_s": samples / (total / 1e3),
            "final_position_error_median": float(np.median([e[0] for e in errs])),
            "final_yaw_error_deg_median": float(np.median([e[1] for e in errs]))}


def run_sweeps(M, prec, Q=4, iters=60):
    """Fig. 6 / Fig. 7 analogue (Sec. IV-D): the ray-uncertainty floor tau of
    Eq. 6 and the initial particle count, swept on the analytic room map
    (synth.room_map_weights), whose pose landscape has a unique optimum.
    Q queries from the global spread (+-1 m, +-180 deg), observations
    rendered by the FP32 form at seeded ground-truth poses (100 x 100, f =
    138.9), three levels x 64 px, 64 + 64 samples, device loop under a CUDA
    graph; per point: ms per batched update, median final errors and the
    fraction of queries within 5 cm and 5 deg."""
    import numpy as np
    import torch
    import synth
    W = H = 100
    focal = 138.9
    taus = (0.01, 0.05, 0.1, 0.5, 1.0, 4.0)
    n0s = (250, 500, 1000, 1500, 3000)
    nmax = max(n0s)
    blob, _ = synth.room_map_weights(0)
    gm = M.Map(blob, max_rays=Q * nmax * 64, max_samples=192, max_particles=Q * nmax,
               max_queries=Q)
    K = M.intrinsics(focal, focal, W / 2, H / 2, W, H)
    o32 = M.UpdateOptions(n_coarse=64, n_fine=128, precision="fp32")
    allpx = np.stack(np.meshgrid(np.arange(W), np.arange(H), indexing="xy"), -1).reshape(-1, 2)
    px_all = torch.tensor(allpx, dtype=torch.int32, device="cuda")
    gts, imgs = [], []
    for q in range(Q):
        g = synth.gt_pose(100 + q)
        gts.append(g)
        P = torch.tensor(g[0][None], dtype=torch.float32, device="cuda")
        imgs.append(gm.render(P, K, 2, px_all, o32).reshape(H, W, 3).contiguous())

    def point(n0, tau):
        sch = M.schedule([0, 1, 2], [64, 64, 64], [n0, max(2 * n0 // 3, 64), max(n0 // 3, 64)],
                         n_min=64, iter_caps=[iters // 3] * 3, refine=[0.02, 0.005, 0.0],
                         iterations=iters, sigma_t=0.02, sigma_yaw=0.02)
        opts = M.UpdateOptions(n_coarse=64, n_fine=64, precision=prec, seed=1, tau=tau)
        parts = torch.tensor(np.stack([synth.random_particles(200 + q, n0)[0] for q in range(Q)]),
                             dtype=torch.float32, device="cuda")
        gm.localize(parts.clone(), [n0] * Q, imgs, K, sch, opts, use_graph=True)   # build + warm
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        log, _ = gm.localize(parts.clone(), [n0] * Q, imgs, K, sch, opts, use_graph=True)
        b.record()
        torch.cuda.synchronize()
        recs = M.Map.decode_log(log, Q, iters)
        errs = [_pose_error(recs[q][-1]["est"], gts[q][1], gts[q][2]) for q in range(Q)]
        return {"ms_per_update": a.elapsed_time(b) / iters,
                "position_error_median": float(np.median([e[0] for e in errs])),
                "yaw_error_deg_median": float(np.median([e[1] for e in errs])),
                "success_5cm_5deg": sum(e[0] < 0.05 and e[1] < 5.0 for e in errs) / Q}

    out = {"workload": f"room map, {Q} queries, 100x100, 3 levels x 64 px, 64+64 samples, "
                       f"{iters} iterations, {prec}",
           "tau_sweep_n0_1500": {str(t): point(1500, t) for t in taus},
           "n0_sweep_tau_0.1": {str(n): point(n, 0.1) for n in n0s}}
    gm.close()
    return out


# --------------------------------------------------------------- GPU arm
def job_rate(dist, seconds, units, device="cpu"):
    """Whole-job throughput over the ranks of a run: the units every rank
    processed, summed, over the slowest rank's time.  Returns (slowest
    seconds, total units, units per second); dist is torch.distributed with
    an initialised process group, or None for a single process."""
    if dist is None:
        return float(seconds), float(units), float(units) / float(seconds)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item()), float(u.item()) / float(t.item())


def _room_queries(M, Q, iters, N0, W=100, H=100, focal=138.9):
    """The room-map localisation workload: the hand-set room map, Q seeded
    ground truths (seeds 100..) with 100 x 100 observations rendered by its
    FP32 form (64 + 128 samples), a three-level schedule (64 px per level,
    N0 / N0/2 / N0/4 particles, iters/3 iterations per level) and seeded
    initial particles over the global spread.  Returns (map, K, ground
    truths, images, schedule, initial particles [Q, N0, 12])."""
    import numpy as np
    import torch
    import synth
    blob, _ = synth.room_map_weights(0)
    gm = M.Map(blob, max_rays=Q * N0 * 64, max_samples=192, max_particles=Q * N0,
               max_queries=Q)
    K = M.intrinsics(focal, focal, W / 2, H / 2, W, H)
    o32 = M.UpdateOptions(n_coarse=64, n_fine=128, precision="fp32")
    allpx = np.stack(np.meshgrid(np.arange(W), np.arange(H), indexing="xy"), -1).reshape(-1, 2)
    px_all = torch.tensor(allpx, dtype=torch.int32, device="cuda")
    gts, imgs = [], []
    for q in range(Q):
        g = synth.gt_pose(100 + q)
        gts.append(g)
        imgs.append(gm.render(torch.tensor(g[0][None], dtype=torch.float32, device="cuda"), K, 2,
                              px_all, o32).reshape(H, W, 3).contiguous())
    sch = M.schedule([0, 1, 2], [64, 64, 64], [N0, N0 // 2, N0 // 4], n_min=100,
                     iter_caps=[iters // 3] * 3, refine=[0.02, 0.005, 0.0], iterations=iters,
                     sigma_t=0.02, sigma_yaw=0.02)
    parts0 = torch.tensor(np.stack([synth.random_particles(200 + q, N0)[0] for q in range(Q)]),
                          dtype=torch.float32, device="cuda")
    return gm, K, gts, imgs, sch, parts0


def _localise(M, gm, parts0, imgs, K, sch, opts, gts, Q, iters):
    """One device-loop run; per-query (position, yaw-degree) errors and the
    accuracy / median summary of the final estimates."""
    import numpy as np
    N0 = parts0.shape[1]
    log, _ = gm.localize(parts0.clone(), [N0] * Q, imgs, K, sch, opts, use_graph=True)
    recs = M.Map.decode_log(log, Q, iters)
    errs = [_pose_error(recs[q][-1]["est"], gts[q][1], gts[q][2]) for q in range(Q)]
    return {"position_error_median": float(np.median([e[0] for e in errs])),
            "yaw_error_deg_median": float(np.median([e[1] for e in errs])),
            "accuracy_5cm_5deg": sum(e[0] < 0.05 and e[1] < 5.0 for e in errs) / Q,
            "position_errors": [float(e[0]) for e in errs]}


def run_fitted_map(M, Q=10, iters=45, n_points=1 << 20, steps=3000, batch=16384):
    """A map fitted by the library's own backward kernels (mcl_fit_map) to
    the room field, from He-init weights: n_points seeded samples (half
    uniform in the box, half in the wall shell) with their closed-form
    density and colour, `steps` Adam steps of `batch` points, the rate
    decaying 1e-3 -> 1e-4.  Reported: fit time per step and points/s
    (forward + backward + Adam), the loss, the fitted map's FP32 render
    error against the hand-set map on 64 poses x 64 px, and localisation of
    the equal-pose-error queries by the BF16 form with the fitted map and
    with the hand-set map (observations from the hand-set map)."""
    import numpy as np
    import torch
    import synth
    N0 = 1500
    hs, K, gts, imgs, sch, parts0 = _room_queries(M, Q, iters, N0)
    x, d = synth.room_fit_points(1, n_points)
    sig, rgb = synth.room_field(x)
    tgt = np.concatenate([sig[:, None], rgb], 1).astype(np.float32)
    xt, dt, tt = (torch.tensor(a, device="cuda") for a in (x, d, tgt))
    fm = M.Map(synth.he_init_weights(0), max_rays=Q * N0 * 64, max_samples=192,
               max_particles=Q * N0, max_queries=Q)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lg = fm.fit(xt, dt, tt, steps=steps, batch=batch, lr=1e-3, lr_end=1e-4, sigma_weight=1e-2,
                seed=3).cpu().numpy()
    fit_s = time.perf_counter() - t0
    o32 = M.UpdateOptions(n_coarse=64, n_fine=128, precision="fp32")
    P = torch.tensor(synth.random_particles(5, 64)[0], dtype=torch.float32, device="cuda")
    px = torch.tensor(synth.pixel_set(5, 25, 25, 64), dtype=torch.int32, device="cuda")
    e = (fm.render(P, K, 0, px, o32) - hs.render(P, K, 0, px, o32)).abs().cpu().numpy()
    ob = M.UpdateOptions(n_coarse=64, n_fine=32, precision="bf16", seed=1)
    out = {"workload": f"room field, {n_points} samples, {steps} Adam steps x {batch} points from "
                       f"He init; localisation as equal_pose_error ({Q} queries, BF16 64+32)",
           "fit_ms_per_step": 1e3 * fit_s / steps,
           "fit_points_per_s": steps * batch / fit_s,
           "loss_first_20": float(lg[:20].mean()), "loss_last_100": float(lg[-100:].mean()),
           "render_err_vs_handset_fp32": {"mean": float(e.mean()),
                                          "p99": float(np.quantile(e, 0.99)),
                                          "max": float(e.max())},
           "fitted_bf16": _localise(M, fm, parts0, imgs, K, sch, ob, gts, Q, iters),
           "handset_bf16": _localise(M, hs, parts0, imgs, K, sch, ob, gts, Q, iters)}
    fm.close()
    hs.close()
    return out


def run_pose_error(M, Q=20, iters=45):
    """Equal-pose-error comparison (Sec. IV-A accuracy definition: position
    error < 5 cm and rotation error < 5 deg) on the analytic room map, whose
    pose landscape has a unique optimum: Q queries from the global spread
    (+-1 m, +-180 deg), each with its own seeded ground truth and the same
    initial particles for every form, localised by the device loop (one CUDA
    graph for all queries) with the plain FP32 form (64 + 32 samples), the
    BF16 form (64 + 32), and the BF16 and FP8 forms with the learned proposal
    (64 -> 32 guided + 32 importance) distilled on this map.  100 x 100
    observations rendered by the FP32 form at the ground truths, three levels
    x 64 px, 1500 / 750 / 375 particles, 15 iterations per level.  The
    tensor-core forms are timed on their second run (the first captures the
    graph and runs the autotuner); the FP32 form, ~20x slower, on its only
    run (graph capture included, a few ms of its ~1 min)."""
    import numpy as np
    import torch
    import synth
    N0 = 1500
    gm, K, gts, imgs, sch, parts0 = _room_queries(M, Q, iters, N0)
    # learned proposal distilled from the FP32 full sampler on this map
    Ptr = torch.tensor(synth.random_particles(21, 256)[0], dtype=torch.float32, device="cuda")
    pxtr = torch.tensor(synth.pixel_set(21, 25, 25, 64), dtype=torch.int32, device="cuda")
    gm.proposal_set(synth.proposal_init_weights(0))
    gm.proposal_train(Ptr, pxtr, K, 0, M.UpdateOptions(n_coarse=64, n_fine=128, precision="fp32"),
                      epochs=40, batch_rays=2048, n_bins=64, lr=3e-3, lr_end=1e-4, seed=1)
    forms = {
        "fp32_full_64+32": M.UpdateOptions(n_coarse=64, n_fine=32, precision="fp32", seed=1),
        "bf16_full_64+32": M.UpdateOptions(n_coarse=64, n_fine=32, precision="bf16", seed=1),
        "bf16_proposal_64->32+32": M.UpdateOptions(n_coarse=64, n_fine=32, precision="bf16", seed=1,
                                                    use_proposal=True, n_proposal=64,
                                                    n_guided=32),
        "fp8_proposal_64->32+32": M.UpdateOptions(n_coarse=64, n_fine=32, precision="fp8", seed=1,
                                                   use_proposal=True, n_proposal=64,
                                                   n_guided=32),
    }
    out = {"workload": f"room map, {Q} queries (seeds 100..{99 + Q}), 100x100, 3 levels x 64 px, "
                       f"{N0}/{N0 // 2}/{N0 // 4} particles, {iters} iterations, one CUDA graph "
                       "per form; accuracy = position < 5 cm and rotation < 5 deg (Sec. IV-A)"}
    for name, opts in forms.items():
        if opts.precision != "fp32":
            gm.localize(parts0.clone(), [N0] * Q, imgs, K, sch, opts, use_graph=True)  # build + warm
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        log, _ = gm.localize(parts0.clone(), [N0] * Q, imgs, K, sch, opts, use_graph=True)
        b.record()
        torch.cuda.synchronize()
        recs = M.Map.decode_log(log, Q, iters)
        errs = [_pose_error(recs[q][-1]["est"], gts[q][1], gts[q][2]) for q in range(Q)]
        out[name] = {"ms_per_batched_update": a.elapsed_time(b) / iters,
                     "position_error_median": float(np.median([e[0] for e in errs])),
                     "yaw_error_deg_median": float(np.median([e[1] for e in errs])),
                     "accuracy_5cm_5deg": sum(e[0] < 0.05 and e[1] < 5.0 for e in errs) / Q,
                     "position_errors": [float(e[0]) for e in errs]}
    base = out["fp32_full_64+32"]["ms_per_batched_update"]
    for name in forms:
        out[name]["speedup_vs_fp32_form"] = base / out[name]["ms_per_batched_update"]
    gm.close()
    return out


def fp64_error_leg(M, gm, blob, P, img, K, K4, px, forms, prop_blob, n_sample=32):
    """Error against the FP64 oracle, after the timed regions, on a sample of
    the run's own inputs: n_sample particles (evenly spaced indices) x the
    first pixel set of the full-update workload.  Per form: RGB max / mean
    absolute error against the oracle of the same sampler, Spearman rank
    correlation and top-10 overlap of the particles' log-weights against
    the oracle's full sampler (the method's own sampler, the judge of weight
    error)."""
    import numpy as np
    import torch
    import oracle
    from scipy.stats import spearmanr
    wl = WL
    sel = np.linspace(0, wl["N"] - 1, n_sample).round().astype(int)
    Ps = P[sel].contiguous()
    Ph = Ps.cpu().numpy().astype(np.float64)
    imgh = img.cpu().numpy().astype(np.float64)
    pxh = px.cpu().numpy()
    t0 = time.perf_counter()
    ref = oracle.update(blob, Ph, imgh, K4, 1, pxh,
                        oracle.make_opts(n_coarse=wl["n_coarse"], n_fine=wl["n_fine"]))
    ref_prop = None
    if prop_blob is not None:
        o, d = [], []
        for i in range(n_sample):
            for j in range(pxh.shape[0]):
                oi, di = oracle.ray(Ph[i], *K4, int(pxh[j, 0]), int(pxh[j, 1]))
                o.append(oi)
                d.append(di)
        ref_prop = oracle.render_rays_proposal(
            blob, prop_blob, np.array(o), np.array(d),
            oracle.make_opts(n_coarse=64, n_fine=32), n_p=64, n_g=32)
    oracle_s = time.perf_counter() - t0
    lw_ref = ref["logw"]
    top_ref = set(np.argsort(-lw_ref)[:10])
    res = {"sample": f"{n_sample} of {wl['N']} particles (evenly spaced) x {pxh.shape[0]} px, "
                     f"oracle {oracle_s:.1f} s"}
    for name, opts in forms.items():
        g = gm.update(Ps, img, K, wl["level"], px, opts, debug=True)
        torch.cuda.synchronize()
        rgb = g["rgb"].cpu().numpy().astype(np.float64)
        lw = g["logw"].cpu().numpy().astype(np.float64)
        same = ref_prop["rgb"] if (opts.use_proposal and ref_prop is not None) else ref["rgb"]
        e = np.abs(rgb - same)
        fin = np.isfinite(lw) & np.isfinite(lw_ref)
        res[name] = {"rgb_max_abs": float(e.max()), "rgb_mean_abs": float(e.mean()),
                     "rgb_reference": "oracle, same sampler",
                     "spearman_logw_vs_full_sampler": float(spearmanr(lw[fin], lw_ref[fin]).correlation),
                     "top10_overlap_vs_full_sampler": len(set(np.argsort(-lw)[:10]) & top_ref)}
    return res


def run_ours(args):
    import numpy as np
    import torch

    import synth
    from paper_2406_12202_gb300 import build as B
    B.build()
    import paper_2406_12202_gb300 as M

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    wl = WL
    N, Bpx, W, H = wl["N"], wl["B"], wl["W"], wl["H"]
    ns = wl["n_coarse"] + wl["n_fine"]
    blob = synth.he_init_weights(wl["map_seed"])
    gm = M.Map(blob, max_rays=N * Bpx, max_samples=ns, max_particles=N)
    K = M.intrinsics(wl["focal"], wl["focal"], W / 2, H / 2, W, H)
    opts32 = M.UpdateOptions(n_coarse=wl["n_coarse"], n_fine=wl["n_fine"], precision="fp32")

    # query of this rank: particles, ground truth, observation rendered at GT
    seed = 1000 + rank
    P0 = torch.tensor(synth.random_particles(seed, N)[0], dtype=torch.float32, device=dev)
    gt = torch.tensor(synth.gt_pose(seed)[0][None], dtype=torch.float32, device=dev)
    allpx = np.stack(np.meshgrid(np.arange(W), np.arange(H), indexing="xy"), -1).reshape(-1, 2)
    img = torch.empty(H * W, 3, device=dev)
    chunk = N * Bpx
    for c0 in range(0, H * W, chunk):
        pc = torch.tensor(allpx[c0:c0 + chunk], dtype=torch.int32, device=dev)
        img[c0:c0 + pc.shape[0]] = gm.render(gt, K, 2, pc, opts32)
    img = img.reshape(H, W, 3).contiguous()
    n_sets = args.warmup + args.steps + 2
    pxs = torch.tensor(np.stack([synth.pixel_set(seed + 7 * t, W, H, Bpx) for t in range(n_sets)]),
                       dtype=torch.int32, device=dev)
    u0s = [synth.resample_u0(seed + t) for t in range(n_sets)]

    P = P0.clone()
    P_next = torch.empty_like(P)
    out = dict(logw=torch.empty(N, device=dev), w=torch.empty(N, dtype=torch.float64, device=dev),
               mask=torch.empty(N, dtype=torch.uint8, device=dev))
    idx = torch.empty(N, dtype=torch.int32, device=dev)
    spread = torch.empty(4, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(t, o, Pin, Pout):
        gm.update(Pin, img, K, wl["level"], pxs[t], o, out=out)
        gm.resample(out["w"], N, u0s[t], idx=idx)
        M.predict(Pin, idx, N, wl["sigma_t"], wl["sigma_yaw"], seed, t, out=Pout)
        M.position_spread(Pout, out=spread)

    def timed(o, steps, warmup, profile=False, clocks=None):
        nonlocal P, P_next
        P.copy_(P0)
        for t in range(warmup):
            step(t, o, P, P_next)
            P, P_next = P_next, P
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        if profile:
            gm.profile_read(reset=True)
            gm.profile(True)
        _, l0 = gm.profile_read(reset=False)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        if clocks:
            clocks.mark_start()
        for k in range(steps):
            flush.zero_()
            evs[k][0].record()
            step(warmup + k, o, P, P_next)
            evs[k][1].record()
            P, P_next = P_next, P
        torch.cuda.synchronize()
        if clocks:
            clocks.mark_end()
        ms = [a.elapsed_time(b) for a, b in evs]
        phases, l1 = gm.profile_read(reset=True)
        gm.profile(False)
        return ms, phases, l1 - l0

    peaks, peak_src = load_peaks()
    rows = N * Bpx * ns

    # ---- headline: the plain FP32 form (the paper's precision) ----------
    gpu_id = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] or str(local)
    clocks = ClockSampler(gpu_id) if rank == 0 else None
    ms, phases, launches = timed(opts32, args.steps, args.warmup, profile=True, clocks=clocks)
    clk = clocks.stop() if clocks else None
    total_s = sum(ms) / 1e3
    units = N * Bpx * ns * args.steps
    _, _, value = job_rate(dist, total_s, units, dev)

    # end to end through the public API with host buffers (pinned), FP32 form
    hP = P0.cpu().pin_memory()
    himg = img.cpu().pin_memory()
    hpx = pxs.cpu().pin_memory()
    hw = torch.empty(N, dtype=torch.float64).pin_memory()
    hmask = torch.empty(N, dtype=torch.uint8).pin_memory()
    hidx = torch.empty(N, dtype=torch.int32).pin_memory()
    hP_out = torch.empty(N, 12, dtype=torch.float32).pin_memory()
    dP = torch.empty_like(P0)
    dimg = torch.empty_like(img)
    dpx = torch.empty(Bpx, 2, dtype=torch.int32, device=dev)
    bi = hP.numel() * 4 + himg.numel() * 4 + Bpx * 2 * 4
    bo = N * 8 + N + N * 4 + N * 12 * 4
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dP.copy_(hP, non_blocking=True)
        dimg.copy_(himg, non_blocking=True)
        dpx.copy_(hpx[k], non_blocking=True)
        gm.update(dP, dimg, K, wl["level"], dpx, opts32, out=out)
        gm.resample(out["w"], N, u0s[k], idx=idx)
        M.predict(dP, idx, N, wl["sigma_t"], wl["sigma_yaw"], seed, k, out=P_next)
        hw.copy_(out["w"], non_blocking=True)
        hmask.copy_(out["mask"], non_blocking=True)
        hidx.copy_(idx, non_blocking=True)
        hP_out.copy_(P_next, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
    e2e_t, _, e2e_value = job_rate(dist, sum(e2e_ms) / 1e3, units, dev)

    # ---- the optimised forms on the same workload -------------------------
    forms = {}
    form_opts = {}
    tc = [p for p in ("bf16", "fp8") if gm.supports(p)]
    for prec in tc:
        o = M.UpdateOptions(n_coarse=wl["n_coarse"], n_fine=wl["n_fine"], precision=prec)
        ms_p, ph_p, _ = timed(o, args.steps, args.warmup, profile=True)
        mlp_ms = (ph_p["mlp_coarse"] + ph_p["mlp_fine"]) / args.steps
        flops = 2.0 * M.TC_MAC_PER_SAMPLE * rows
        peak = peaks["bf16_tflops"] * (2.0 if prec == "fp8" else 1.0)
        roof = {"bound": "tensor", "achieved": flops / (mlp_ms / 1e3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "peak_source": f"bf16_tflops burst ({peak_src})"
                + (" x 2 nominal fp8/bf16 ratio" if prec == "fp8" else ""),
                "kernel": "k_mlp_tc (coarse + fine passes)", "mlp_ms_per_step": mlp_ms}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof["achieved_survey_flops"] = 2.0 * MAC_PER_SAMPLE_FP32 * rows / (mlp_ms / 1e3) / 1e12
        roof["traffic"] = profiled_traffic(f"k_mlp_tc_c2_{prec}",
                                           ("mlp_tc.cu", "tc_ptx.cuh", "stages.cuh"))
        m_ = sum(ms_p) / len(ms_p)
        forms[prec] = {"ms_per_step": m_, "ray_samples_per_s": N * Bpx * ns / (m_ / 1e3),
                       "speedup_vs_fp32_form": (sum(ms) / len(ms)) / m_,
                       "phases_ms_per_step": {k: v / args.steps for k, v in ph_p.items()},
                       "ray_epilogue": "separate sampling / composite kernels (the default)",
                       "roofline": roof}
        # the same step with the ray epilogues fused into the MLP kernel
        # (mcl_set_fused_epilogue; opt-in: slower on GB300, less DRAM traffic)
        gm.set_fused_epilogue(True)
        ms_f, ph_f, _ = timed(o, args.steps, args.warmup, profile=True)
        gm.set_fused_epilogue(False)
        mf = sum(ms_f) / len(ms_f)
        forms[prec]["fused_epilogue"] = {
            "ms_per_step": mf, "ray_samples_per_s": N * Bpx * ns / (mf / 1e3),
            "mlp_ms_per_step": (ph_f["mlp_coarse"] + ph_f["mlp_fine"]) / args.steps,
            "phases_ms_per_step": {k: v / args.steps for k, v in ph_f.items()}}
        form_opts[prec] = o
    prop_blob = None
    if "fp8" in tc and world == 1 and not args.no_extra:
        try:
            forms["proposal_fp8"], prop_blob = run_proposal_fp8(M, gm, img, K, seed, args.steps,
                                                                args.warmup, wl)
            forms["proposal_fp8"]["speedup_vs_fp32_form"] = (sum(ms) / len(ms)) / \
                forms["proposal_fp8"]["ms_per_step"]
            form_opts["proposal_fp8"] = M.UpdateOptions(n_coarse=64, n_fine=32, precision="fp8",
                                                        use_proposal=True, n_proposal=64,
                                                        n_guided=32)
        except Exception as e:  # an extra workload must never hide the main line
            forms["proposal_fp8"] = {"failed": f"{type(e).__name__}: {e}"}

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel of the headline step: the FP32 SIMT
    # GEMMs of the NeRF MLP (FP32 FMA lanes are the bound)
    mlp_ms = (phases["mlp_coarse"] + phases["mlp_fine"]) / args.steps
    mhz = peaks.get("sm_max_mhz", 2070.0)
    peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
    roof = {"bound": "alu", "achieved": 2.0 * MAC_PER_SAMPLE_FP32 * rows / (mlp_ms / 1e3) / 1e12,
            "peak": peak, "unit": "TFLOP/s",
            "peak_source": f"152 SMs x 128 FP32 lanes x 2 FLOP x {mhz:.0f} MHz ({peak_src} "
                           "max SM clock)",
            "kernel": "NeRF MLP, plain FP32 form (k_sgemm layers, PE, heads; coarse + fine)",
            "mlp_ms_per_step": mlp_ms}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = profiled_traffic("k_sgemm_c2_fp32", ("mlp_fp32.cu",))

    # FP64 error of every form on a sample of this run's inputs (oracle, after
    # the timed regions)
    err = None
    if world == 1 and not args.no_cpu_baseline:
        try:
            import oracle
            oracle.build()
            K4 = (float(np.float32(wl["focal"])), float(np.float32(wl["focal"])), W / 2, H / 2)
            all_forms = {"fp32": opts32, **form_opts}
            err = fp64_error_leg(M, gm, blob, P0, img, K, K4, pxs[0], all_forms, prop_blob)
        except Exception as e:  # the error report must never hide the GPU line
            err = {"failed": f"{type(e).__name__}: {e}"}
    for name, f in forms.items():
        if err and name in err:
            f["err_vs_fp64"] = err[name]

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline()
        except Exception as e:  # the baseline must never hide the GPU line
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
                   "sample": f"failed: {e}"}
    extra = {}
    if world == 1 and args.sweeps:
        try:
            extra["sweeps"] = run_sweeps(M, "bf16" if "bf16" in tc else "fp32")
        except Exception as e:  # an extra workload must never hide the main line
            extra["sweeps"] = {"failed": f"{type(e).__name__}: {e}"}
    if world == 1 and not args.no_extra and "bf16" in tc:
        for name, fn in (
                ("equal_pose_error", lambda: run_pose_error(M)),
                ("fitted_map", lambda: run_fitted_map(M)),
                ("coarse_to_fine", lambda: run_coarse_to_fine(M, img, K, seed, "bf16")),
                ("ablation", lambda: run_ablation(M, img, K, seed, "bf16")),
                ("batched_queries", lambda: run_batched(M, seed, W, H, wl["focal"], prop_blob))):
            try:
                extra[name] = fn()
            except Exception as e:  # an extra workload must never hide the main line
                extra[name] = {"failed": f"{type(e).__name__}: {e}"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(ms) / len(ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["workload"], "particles": N, "pixels": Bpx,
                   "image": f"{W}x{H}", "samples_per_ray": f"{wl['n_coarse']}+{wl['n_fine']}",
                   "mlp_precision": "fp32 (plain form, the paper's precision)",
                   "l2": "flushed (256 MB write) between timed steps",
                   "step": "update + resample + predict + position spread",
                   "parallelism": f"replicas x{world} (one query per GPU)"},
        "update_ms": sum(ms) / len(ms),
        "phases_ms_per_step": {k: v / args.steps for k, v in phases.items()},
        "err_vs_fp64": err.get("fp32") if isinstance(err, dict) else None,
        "err_sample": err.get("sample") if isinstance(err, dict) else None,
        "roofline": roof,
        "forms": forms,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bi,
                "d2h_bytes_per_step": bo, "ms_per_step": 1e3 * e2e_t / args.steps},
        "gpu_launches": launches,
        "clocks": clk,
        "workloads": extra,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the proposal, pose-error, coarse-to-fine, ablation and "
                         "batched-query workloads")
    ap.add_argument("--sweeps", action="store_true",
                    help="add the tau and initial-particle-count sweeps on the room map")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
