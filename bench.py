#!/usr/bin/env python
"""TT-ICE* increment-update throughput on one GB300 (and N independent replicas under torchrun).

Headline workload (the large video stream): frames of 1080x1920x3 moving Gaussian blobs (40 blobs,
sigma 8-40 px, per-channel amplitude U(0,1), linear trajectories reflected at the borders, a new
scene every 500 frames, N(0, 0.01^2) pixel noise) viewed as the 5-way tensor 27x40x48x40x3, FP32
input, eps = 0.05, increments of 32 frames (796 MB each).  A step is one TT-ICE* update of one
increment through the whole path (first pass with per-observation errors, skip test, subselection,
per-core residual / Gram / truncated eigen-solve / CGS2 / append / padding, final projection and
last-core append).  The stream is consumed in order: W warm-up increments, then K timed increments,
each a fresh slice of a stream pre-generated in device memory (inputs larger than L2).

Side legs, reported in the same line: the end-to-end rate from pinned host memory (`e2e`), the
128^3 x 4 simulation-shaped stream at eps 0.05 and 0.01 timed in its skip regime (`flow`), the
480x640x3 video stream with the plain FP64 GPU path beside the mixed one (`video_480p`), projection
of unseen frames (`project`), the paper's heuristics against the exact defaults (`paper_variants`),
the many-stream serving loop (`serving`), and the FP64 CPU oracle on a bounded sample
(`cpu_baseline`).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (27, 40, 48, 40, 3)
EPS = 0.05
BATCH = 32
WORKLOAD = ("video 1080x1920x3 as 27x40x48x40x3, fp32 input, eps=0.05, 40 blobs (sigma 8-40 px), "
            "noise 0.01, new scene every 500 frames, increments of 32 frames")
METRIC = "increment elements/s"
V480 = (20, 24, 20, 32, 3)

# Unit each phase of an update runs on (mixed path), for the roofline of a phase: its algorithmic
# flops are held against the peak of that unit, its algorithmic bytes against HBM.  The projections,
# residuals, Grams and the large re-orthogonalisations run on the tensor cores (TF32 head/tail
# split); the block-Jacobi eigen-solve is FP32 SIMT (its flops: 8 s^3 per sweep).
PHASE_UNIT = {"k1_stage1": "tf32", "chain": "tf32", "final": "tf32", "d_project": "tf32",
              "residual": "tf32", "gram": "tf32", "eig": "fp32", "orth_append": "tf32"}


def frames_1080(t0: int, n: int, seed: int = 1004, device="cuda"):
    import torch

    from tt_streams import blob_video

    return blob_video(t0, n, height=1080, width=1920, n_blobs=40, view=DIMS, scene_len=500, noise_std=0.01,
                      seed=seed, device=device, compute_dtype=torch.float32 if device != "cpu" else torch.float64)


def _peaks_file():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm_gbs": float(p["hbm_gbs"]), "bf16_tflops": float(p["bf16_tflops"])}, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def measure_matmul_peaks():
    """Dense matmul throughput of the GPU's FP64, FP32 and TF32 units (cuBLAS through torch, square
    operands, a few repetitions after warm-up): the compute peaks the rooflines of the FP64 and
    FP32 SIMT phases and of the TF32 tensor-core phases are held against."""
    import torch

    out = {}
    for name, dt, tf32, n, reps in (("fp64", torch.float64, False, 4096, 3), ("fp32", torch.float32, False, 8192, 4),
                                    ("tf32", torch.float32, True, 8192, 10)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device="cuda", dtype=dt)
        b = torch.randn(n, n, device="cuda", dtype=dt)
        a @ b
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            a @ b
        e1.record()
        torch.cuda.synchronize()
        out[name + "_tflops"] = 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12
        del a, b
    torch.backends.cuda.matmul.allow_tf32 = False
    torch.cuda.empty_cache()
    return out


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def replica_seed(rank: int) -> int:
    """Seed of the stream replica `rank` runs (independent streams: weak scaling, no collective on
    the data path)."""
    return 1004 + 7919 * rank


def max_over_ranks(x: float, ws: int, device) -> float:
    """The slowest rank's value of a timed region (identity for one rank)."""
    if ws <= 1:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws: int, units_per_rank: float, seconds: float) -> float:
    """Units processed by all ranks over the slowest rank's time."""
    return ws * units_per_rank / seconds


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def percentile(vals, q):
    v = sorted(vals)
    return v[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))] if v else None


# ---------------------------------------------------------------- handles and streams
def headline_handle(T, precision: str, n_inc: int):
    """A handle for the 1080p stream with rank capacities for n_inc increments of 32 frames: the
    stream's pixel noise is ~9% of its energy against the 5% target, so TT-ICE keeps most of it and
    core 3 gains ~3300 directions per increment up to r_2 n_3 (<= 51840), core 4 ~90 per increment.
    Capacities are raised before the stream starts, so no timed step pays for a growth."""
    import torch

    h = T.TTICE(DIMS, EPS, precision=precision, input_dtype=torch.float32, max_batch=BATCH, max_rank=1024,
                obs_reserve=BATCH * n_inc)
    # rank 4 first, while rank 3's capacity (which sizes U_4's rows) is still small: each growth
    # holds the old and the new buffers at once
    h.reserve_rank(2, 1080)
    h.reserve_rank(4, 256 * math.ceil(max(1024, 100 * n_inc) / 256))
    h.reserve_rank(3, min(51840, 4096 * math.ceil(n_inc * 3840 / 4096)))
    return h


def update_growing(T, h, Y, stream=None):
    """ttice_update; an update that needs a rank above its capacity grows it (doubling) and is
    repeated (a failed update leaves the decomposition as it was).  Returns (stats, growths)."""
    grows = 0
    while True:
        try:
            return h.update(Y, stream=stream), grows
        except T.TTICEError as e:
            if e.code != T.TTICE_ECAPACITY:
                raise
            k, need = h.capacity_miss()
            if k == 0:
                raise
            h.reserve_rank(k, max(need, 2 * h.capacities()[k]))
            grows += 1


def phase_roofline(prof, name, peaks, peak_kind, live):
    """Roofline of one phase over the timed updates: its algorithmic bytes against HBM and its
    algorithmic flops against the peak of the unit it runs on; the bound is whichever gives the
    longer lower bound on its time."""
    ph = prof[name]
    if not ph["count"] or ph["ms"] <= 0:
        return None
    t = ph["ms"] / 1e3
    unit = PHASE_UNIT[name]
    p_flops = live[unit + "_tflops"] * 1e12
    p_bytes = peaks["hbm_gbs"] * 1e9
    if ph["bytes"] / p_bytes >= ph["flops"] / p_flops:
        ach = ph["bytes"] / t / 1e9
        return {"bound": "hbm", "phase": name, "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "peak_kind": peak_kind,
                "bytes_per_launch": ph["bytes"] / ph["count"], "avg_launch_ms": ph["ms"] / ph["count"]}
    ach = ph["flops"] / t / 1e12
    return {"bound": "tensor" if unit == "tf32" else "alu", "phase": name, "unit_kind": unit, "achieved": ach,
            "peak": live[unit + "_tflops"], "unit": "TFLOP/s", "frac": ach / live[unit + "_tflops"],
            "peak_kind": "measured live (cuBLAS " + unit + " matmul)",
            "flops_per_launch": ph["flops"] / ph["count"], "avg_launch_ms": ph["ms"] / ph["count"]}


def run_headline(T, args, dev, seed, precision):
    """W warm-up and K timed updates of the 1080p stream from device-resident input; afterwards the
    relative error of the last timed increment, measured in FP64 from its reconstruction (Theorem 2:
    later updates would leave it as it was right after its own).  One increment only: the FP64
    reconstruction of 32 frames through the grown cores takes ~15 s."""
    import torch

    b, W, K = BATCH, args.warmup, args.steps
    Y = torch.empty(((W + K) * b,) + DIMS, dtype=torch.float32, device=dev)
    for k in range(0, (W + K) * b, b):
        Y[k:k + b] = frames_1080(k, b, seed=seed)
    torch.cuda.synchronize()
    h = headline_handle(T, precision, W + K)
    try:
        grows = 0
        for k in range(W):
            _, g = update_growing(T, h, Y[k * b:(k + 1) * b])
            grows += g
        h.profile(True)
        st = torch.cuda.current_stream()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
        l0 = T.ttice_kernel_launches()
        torch.cuda.synchronize()
        evs[0].record(st)
        steps = []
        for k in range(K):
            i = W + k
            s, g = update_growing(T, h, Y[i * b:(i + 1) * b])
            grows += g
            evs[k + 1].record(st)
            steps.append({"skipped": int(s.skipped), "n_selected": s.n_selected, "ranks": list(s.ranks[:len(DIMS) + 2]),
                          "new_dirs": list(s.new_dirs[:len(DIMS)]), "krylov": s.krylov_solves,
                          "krylov_fallbacks": s.krylov_fallbacks, "rel_err_before": s.rel_err_before})
        torch.cuda.synchronize()
        launches = T.ttice_kernel_launches() - l0
        lat = [evs[k].elapsed_time(evs[k + 1]) for k in range(K)]
        total = evs[0].elapsed_time(evs[-1])
        prof = h.profile_read()
        errs = []
        for i in (W + K - 1,):
            Yi = Y[i * b:(i + 1) * b].double()
            rec = h.reconstruct(i * b, b)
            errs.append(math.sqrt(float(((Yi - rec) ** 2).sum()) / float((Yi ** 2).sum())))
            del Yi, rec
        out = {"total_ms": total, "lat": lat, "steps": steps, "prof": prof, "launches": launches, "grows": grows,
               "core_elems": int(h.stats().core_elems), "n_obs": int(h.stats().n_obs),
               "device_gb": h.device_bytes() / 1e9, "errs": errs}
        return out
    finally:  # also when an update fails (e.g. a capacity growth out of memory)
        h.close()
        del Y
        torch.cuda.empty_cache()


def sweep_row(hl, K: int) -> dict:
    """One precision's row of the 1080p precision sweep."""
    N = math.prod(DIMS)
    steps = hl["steps"]
    return {"value": K * BATCH * N / (hl["total_ms"] / 1e3), "unit": "elements/s", "ms_per_step": hl["total_ms"] / K,
            "latency_ms": {"p50": statistics.median(hl["lat"]), "p99": percentile(hl["lat"], 0.99)},
            "final_ranks": steps[-1]["ranks"], "core_elements": hl["core_elems"],
            "compression_ratio": hl["n_obs"] * N / max(hl["core_elems"], 1),
            "skipped": sum(s["skipped"] for s in steps),
            "eps_check": {"eps": EPS, "rel_err_last": hl["errs"][-1], "over_eps": hl["errs"][-1] > EPS * (1 + 1e-9),
                          "measured": "FP64, from the last timed increment's reconstruction"}}


def run_e2e(T, args, dev, seed, precision):
    """The same stream through the public API from pinned host memory: each step copies its increment
    host -> device, updates, and reads its rows of the last core back, all inside the timed region."""
    import torch

    b, W, K = BATCH, args.warmup, args.steps
    Yh = torch.empty(((W + K) * b,) + DIMS, dtype=torch.float32, pin_memory=True)
    for k in range(0, (W + K) * b, b):
        Yh[k:k + b] = frames_1080(k, b, seed=seed).cpu()
    h = headline_handle(T, precision, W + K)
    buf = torch.empty((b,) + DIMS, dtype=torch.float32, device=dev)
    for k in range(W):
        buf.copy_(Yh[k * b:(k + 1) * b], non_blocking=True)
        update_growing(T, h, buf)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0
    for k in range(K):
        i = W + k
        buf.copy_(Yh[i * b:(i + 1) * b], non_blocking=True)
        update_growing(T, h, buf)
        rows = h.last_core()[-b:]  # the step's result: its coefficient rows of the last core
        d2h += rows.nbytes
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h.close()
    torch.cuda.empty_cache()
    return dt, b * math.prod(DIMS) * 4, int(d2h / K)


def run_flow(T, eps: float, warmup: int, steps: int, b: int = 16, seed: int = 1002):
    """The simulation-shaped stream (128^3 grid x 4 fields, 64 Fourier modes per field, |k|^(-5/3)
    amplitudes, advected at (0.3, 0.1, 0.2) cells/snapshot), FP32, batches of b: `warmup` increments
    generated on the fly (the stream reaches its skip regime after ~80), then `steps` timed ones from
    a pre-generated device buffer.  Skip-path steps (one read of the 537 MB batch and the chain of
    projections) are reported apart from updating ones, each against the roofline of its
    algorithmic bytes (HBM) and flops (TF32 tensor peak)."""
    import torch

    from tt_streams import fourier_flow

    dims = (128, 128, 128, 4)
    h = T.TTICE(dims, eps, precision="fp32", input_dtype=torch.float32, max_batch=b, max_rank=1024)
    t0 = time.perf_counter()
    for k in range(warmup):
        update_growing(T, h, fourier_flow(k * b, b, seed=seed, device="cuda"))
    warm_s = time.perf_counter() - t0
    Y = torch.empty((steps * b,) + dims, dtype=torch.float32, device="cuda")
    for k in range(steps):
        Y[k * b:(k + 1) * b] = fourier_flow((warmup + k) * b, b, seed=seed, device="cuda")
    h.profile(True)
    st = torch.cuda.current_stream()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.synchronize()
    evs[0].record(st)
    flags = []
    for k in range(steps):
        s, _ = update_growing(T, h, Y[k * b:(k + 1) * b])
        flags.append(bool(s.skipped))
        evs[k + 1].record(st)
    torch.cuda.synchronize()
    lat = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
    total = evs[0].elapsed_time(evs[-1])
    ranks = h.ranks()
    prof = h.profile_read()
    h.close()
    del Y
    torch.cuda.empty_cache()
    n_el = b * math.prod(dims)
    skip = [x for x, f in zip(lat, flags) if f]
    upd = [x for x, f in zip(lat, flags) if not f]
    # algorithmic amounts of a skip step: the first pass and the chain (Sec. 8(d) with u = 0)
    k1, ch = prof["k1_stage1"], prof["chain"]
    cnt = max(k1["count"], 1)
    skip_bytes = (k1["bytes"] + ch["bytes"]) / cnt
    skip_flops = (k1["flops"] + ch["flops"]) / cnt
    out = {"workload": f"flow 128^3 x 4 (4-way 128x128x128x4), fp32 input, eps={eps}, 64 modes/field, batches of {b}",
           "warmup_increments": warmup, "warmup_s": warm_s, "steps": steps, "value": steps * n_el / (total / 1e3),
           "unit": "elements/s", "ms_per_step": total / steps,
           "latency_ms": {"p50": statistics.median(lat), "p99": percentile(lat, 0.99)},
           "skipped": len(skip), "final_ranks": ranks,
           "skip_path_ms": {"p50": statistics.median(skip), "min": min(skip)} if skip else None,
           "update_path_ms": {"p50": statistics.median(upd), "max": max(upd)} if upd else None,
           "skip_step_bytes": skip_bytes, "skip_step_flops": skip_flops, "prof": prof}
    return out


def run_video480(T, args, precision: str, steps: int, warmup: int = 5, b: int = 8, seed: int = 1001):
    """The 480x640x3 video stream (12 blobs, eps = 0.1, increments of 8 frames), timed after warm-up."""
    import torch

    from tt_streams import blob_video

    n = warmup + steps
    Y = torch.empty((n * b,) + V480, dtype=torch.float32, device="cuda")
    for k in range(0, n * b, 64):
        c = min(64, n * b - k)
        Y[k:k + c] = blob_video(k, c, seed=seed, device="cuda")
    h = T.TTICE(V480, 0.1, precision=precision, input_dtype=torch.float32, max_batch=b, max_rank=512)
    for k in range(warmup):
        update_growing(T, h, Y[k * b:(k + 1) * b])
    h.profile(True)
    st = torch.cuda.current_stream()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.synchronize()
    evs[0].record(st)
    for k in range(steps):
        i = warmup + k
        update_growing(T, h, Y[i * b:(i + 1) * b])
        evs[k + 1].record(st)
    torch.cuda.synchronize()
    lat = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
    total = evs[0].elapsed_time(evs[-1])
    rk = h.ranks()
    built = {"ranks": rk[:len(V480) + 1], "cores": [h.core(i) for i in range(1, len(V480) + 1)],
             "last": h.last_core()}
    prof = h.profile_read()
    h.close()
    return {"precision": precision, "steps": steps, "value": steps * b * math.prod(V480) / (total / 1e3),
            "unit": "elements/s", "ms_per_step": total / steps,
            "latency_ms": {"p50": statistics.median(lat), "p99": percentile(lat, 0.99)},
            "final_ranks": rk, "prof": prof}, built, Y


def run_project(T, built: dict, batches: int, b: int = 32, seed: int = 1001):
    """Projection of unseen frames onto the cores the 480p stream built (Algorithm 2 'project'; the
    relative prediction error workload of Sec. 5.1): `batches` calls of ttice_project on b frames
    each, frames 100000 onwards of the same generator, after 3 untimed calls."""
    import torch

    from tt_streams import blob_video

    N = math.prod(V480)
    hp = T.TTICE(V480, 0.1, precision="fp32", input_dtype=torch.float32, max_batch=b)
    hp.load(built["ranks"], built["cores"], built["last"])
    Z = torch.empty((batches * b,) + V480, dtype=torch.float32, device="cuda")
    for k in range(0, batches * b, 64):
        c = min(64, batches * b - k)
        Z[k:k + c] = blob_video(100000 + k, c, seed=seed, device="cuda")
    rd = built["ranks"][len(V480)]
    coeffs = torch.empty((b, max(rd, 1)), dtype=torch.float64, device="cuda")
    rel = torch.empty((batches, b), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    for k in range(3):
        T.ttice_project(hp.h, Z[k * b:(k + 1) * b], coeffs, rel[k], st)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(batches + 1)]
    torch.cuda.synchronize()
    evs[0].record(st)
    for k in range(batches):
        T.ttice_project(hp.h, Z[k * b:(k + 1) * b], coeffs, rel[k], st)
        evs[k + 1].record(st)
    torch.cuda.synchronize()
    lat = [evs[k].elapsed_time(evs[k + 1]) for k in range(batches)]
    total = evs[0].elapsed_time(evs[-1])
    hp.close()
    r = rel.cpu()
    return {"workload": f"ttice_project of unseen 480p frames, {b} per call, onto ranks {built['ranks']}",
            "calls": batches, "value": batches * b * N / (total / 1e3), "unit": "elements/s",
            "ms_per_call": total / batches, "p50_ms": statistics.median(lat),
            "rel_err_mean": float(r.mean()), "rel_err_max": float(r.max())}


def run_variants(T, Y, steps: int, b: int = 8):
    """The 480p stream run twice from empty cores: with the exact defaults (skip on the batch error
    of Eq. 20, eps_upd of Eq. 18, tau = 1) and with the paper's heuristics (skip on mean(eps_Y), eps_upd
    of Eq. 19, occupancy tau = 0.8), reconstructing every increment: the rate at which each exceeds
    eps, with the time and core sizes the heuristics save."""
    import torch

    out = {}
    for name, kw in (("exact", {}), ("paper", {"skip_mode": "mean", "eps_upd": "approx", "tau": 0.8})):
        h = T.TTICE(V480, 0.1, precision="fp32", input_dtype=torch.float32, max_batch=b, **kw)
        errs, skipped, ms = [], 0, 0.0
        for k in range(steps):
            Yk = Y[k * b:(k + 1) * b]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st, _ = update_growing(T, h, Yk)
            e1.record()
            rec = h.reconstruct(k * b, b, dtype=torch.float64)
            errs.append(float((Yk.double() - rec).reshape(-1).norm() / Yk.double().reshape(-1).norm()))
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            skipped += int(st.skipped)
        viol = [e for e in errs if e > 0.1 * (1 + 1e-9)]
        out[name] = {"increments": steps, "skipped": skipped, "update_ms_total": ms, "eps_violations": len(viol),
                     "violation_rate": len(viol) / steps, "max_rel_err": max(errs),
                     "final_ranks": h.ranks(), "core_elems": int(h.stats().core_elems)}
        h.close()
    return out


def run_serving(seconds: float, n_streams: int = 64, rates=(50.0, 400.0, 2000.0), slots: int = 16, seed: int = 1003,
                drain_s: float = 60.0):
    """Continuous batching over many streams: shapes drawn from {16^4 cosine stream, the 480p video
    view, 64^3 x 4 flow, 32^4 cosine stream}, batch sizes from {1, 4, 16, 32}, eps from {0.05, 0.1,
    0.3}; Poisson arrivals over all streams for `seconds` at each rate in `rates`.  Each stream cycles
    through a pool of pre-generated device-resident increments, so later requests of a stream are
    mostly represented already and take the skip path.  Latency = arrival -> completion."""
    import collections
    import random

    import torch

    from paper_2211_12487_gb300 import serving as S
    from tt_streams import blob_video, cp_cosine, fourier_flow

    rng = random.Random(seed)
    kinds = [("cosine16", (16, 16, 16, 16)), ("video", V480), ("flow64", (64, 64, 64, 4)), ("cosine32", (32, 32, 32, 32))]
    specs, pools = [], {}
    for i in range(n_streams):
        kind, dims = kinds[rng.randrange(len(kinds))]
        b = rng.choice([1, 4, 16, 32])
        eps = rng.choice([0.05, 0.1, 0.3])
        name = f"{kind}_{i}"
        specs.append(S.StreamSpec(name, dims, eps, b))
        n_el = b * math.prod(dims)
        npool = max(2, min(16, (192 << 20) // (4 * n_el)))
        frames = npool * b
        if kind.startswith("cosine"):
            y = cp_cosine(0, frames, dims=dims, seed=seed + i).to(torch.float32).cuda()
        elif kind == "video":
            y = blob_video(0, frames, seed=seed + i, device="cuda")
        else:
            y = fourier_flow(0, frames, grid=64, seed=seed + i, device="cuda")
        pools[name] = [y[k * b:(k + 1) * b] for k in range(npool)]
    torch.cuda.synchronize()
    eng = S.ServingEngine(specs, slots=slots)
    phases = []
    try:
        for sp in specs:
            eng.submit(S.Request(sp.name, pools[sp.name][0]))
        eng.drain(timeout=600)
        count = {sp.name: 1 for sp in specs}
        for rate in rates:
            with eng.lock:
                eng.completed.clear()
            t0 = time.perf_counter()
            t_next = t0
            n_sub, elements = 0, 0
            while True:
                t_next += rng.expovariate(rate)
                if t_next - t0 > seconds:
                    break
                now = time.perf_counter()
                if t_next > now:
                    time.sleep(t_next - now)
                sp = specs[rng.randrange(n_streams)]
                k = count[sp.name]
                count[sp.name] = k + 1
                y = pools[sp.name][k % len(pools[sp.name])]
                eng.submit(S.Request(sp.name, y, arrival=t_next))
                n_sub += 1
                elements += y.numel()
            ok = eng.drain(timeout=drain_s)
            wall = time.perf_counter() - t0
            with eng.lock:
                done = list(eng.completed)
            if not ok:
                with eng.lock:
                    for dq in eng.pending.values():
                        dq.clear()
                eng.drain(timeout=drain_s)
            lat = sorted((r.done - r.arrival) * 1e3 for r in done if r.error is None)
            skipped = sum(1 for r in done if r.stats is not None and r.stats.skipped)
            errors = collections.Counter(str(r.error)[:80] for r in done if r.error is not None)
            phases.append({"arrival_rate_per_s": rate, "seconds": seconds, "requests": n_sub, "completed": len(lat),
                           "errors": dict(errors), "drained": ok, "skipped_fraction": skipped / max(len(done), 1),
                           "p50_ms": S.percentile(lat, 0.50), "p99_ms": S.percentile(lat, 0.99),
                           "throughput_elements_per_s": elements / wall, "throughput_updates_per_s": len(lat) / wall})
        return {"streams": n_streams, "slots": slots, "phases": phases, "capacity_grows": eng.grow_events,
                "device_gb": eng.mem_used / 1e9}
    finally:
        eng.close(cancel_pending=True)


def oracle_sample(frames: int = 1, seed: int = 1004):
    """The FP64 CPU oracle on a bounded sample of the headline workload: the stream's first increment
    of `frames` frames, from empty cores (one frame of the 1080p stream is ~10-20 s of CPU work)."""
    from oracle.ttice_oracle import TTICEOracle

    Y = frames_1080(0, frames, seed=seed, device="cpu").double().numpy()
    o = TTICEOracle(DIMS, EPS)
    t = time.perf_counter()
    o.update(Y)
    busy = time.perf_counter() - t
    threads = os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS") or str(os.cpu_count())
    return Y.size / busy, busy, int(threads)


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample()
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, busy, threads = oracle_sample()
        vals.append(v)
    wall = time.perf_counter() - t0
    val = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "elements/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch": BATCH, "sample": "first increment of 1 frame, from empty cores"},
        "cpu_baseline": {"value": val, "unit": "elements/s", "cores": threads, "kind": "oracle",
                         "sample": "first increment of the stream, 1 frame (6.2e6 elements), from empty cores, per step"},
        "e2e": {"value": val, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def profile_case(case: str, warm: int, precision: str = "fp32") -> None:
    """Small, self-contained cases for ncu (each inside one cudaProfilerStart/Stop window, for
    `ncu --profile-from-start off`); prints one line and exits.

    c4_update: `warm` increments of the 1080p stream, then one steady-state update profiled (the whole
      handle, ~180 GB at warm = 24: only one-pass metrics such as the launch list on this case).
    flow_project: ttice_project of 16 snapshots of the 128^3 x 4 flow (537 MB) onto seeded random
      orthonormal cores at ranks [1, 33, 1177, 431, 207], twice (a few GB on the device): the first
      pass (tc_proj_kernel<64, 0>), stage 1 (tc_proj_kernel<128, 0>), stage 2 (K split), stage 3.
    c4_stage2: ttice_project of 32 frames of the 1080p view onto seeded random orthonormal cores at
      ranks [1, 27, 1005, 4096, 256, 64] (2.8 GB of cores): stage 2 is the large-K contraction of
      the 1080p stream's core 3 (K = 48240, 120 columns per frame) at a twelfth of its rank.
    noise_update: the first update of a 32^4 stream of N(0, 1) noise, 32 tensors, eps = 0.3 (a
      1024-sided Gram with a flat spectrum: the full block-Jacobi eigen-solve), profiled alone."""
    import numpy as np
    import torch

    from paper_2211_12487_gb300 import ttice as T

    if case == "c4_update":
        h = headline_handle(T, "fp32", warm + 1)
        for k in range(warm):
            update_growing(T, h, frames_1080(k * BATCH, BATCH))
        Y = frames_1080(warm * BATCH, BATCH)
        torch.cuda.synchronize()
        l0 = T.ttice_kernel_launches()
        torch.cuda.profiler.start()
        s, _ = update_growing(T, h, Y)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"case": case, "warm": warm, "ranks": list(s.ranks[:len(DIMS) + 2]),
                          "new_dirs": list(s.new_dirs[:len(DIMS)]), "krylov": s.krylov_solves,
                          "krylov_fallbacks": s.krylov_fallbacks, "eig_sweeps": s.eig_sweeps,
                          "launches": T.ttice_kernel_launches() - l0}))
        h.close()
        return
    from tt_streams import fourier_flow

    if case == "noise_update":
        g = torch.Generator(device="cuda").manual_seed(5)
        Y = torch.randn((32, 32, 32, 32, 32), generator=g, device="cuda", dtype=torch.float32)
        h = T.TTICE((32, 32, 32, 32), 0.3, precision="fp32", input_dtype=torch.float32, max_batch=32,
                    max_rank=1024)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        s = h.update(Y)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"case": case, "ranks": list(s.ranks[:6]), "krylov": s.krylov_solves,
                          "krylov_fallbacks": s.krylov_fallbacks, "eig_sweeps": s.eig_sweeps,
                          "device_gb": h.device_bytes() / 1e9}))
        h.close()
        return
    if case == "flow_project":
        dims, ranks, b = (128, 128, 128, 4), [1, 33, 1177, 431, 207], 16
        Y = fourier_flow(0, b, seed=1002, device="cuda")
    elif case == "c4_stage2":
        dims, ranks, b = DIMS, [1, 27, 1005, 4096, 256, 64], BATCH
        Y = frames_1080(0, b)
    else:
        raise SystemExit(f"unknown profile case {case}")
    rng = np.random.default_rng(3)
    cores = [np.linalg.qr(rng.normal(size=(ranks[i] * n, ranks[i + 1])))[0] for i, n in enumerate(dims)]
    eps = 0.1 if precision == "tf32" else 0.01
    h = T.TTICE(dims, eps, precision=precision, input_dtype=torch.float32, max_batch=b, max_rank=max(ranks))
    h.load(ranks, cores, np.zeros((1, ranks[-1])))
    coeffs = torch.empty((b, ranks[-1]), dtype=torch.float64, device="cuda")
    rel = torch.empty((b,), dtype=torch.float64, device="cuda")
    T.ttice_project(h.h, Y, coeffs, rel)  # warm-up (module load, tensor maps)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.profiler.start()
    ev[0].record()
    for k in range(2):
        T.ttice_project(h.h, Y, coeffs, rel)
        ev[k + 1].record()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"case": case, "precision": precision, "ranks": ranks, "rel_mean": float(rel.mean()),
                      "ms_per_call": [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])],
                      "device_gb": h.device_bytes() / 1e9}))
    h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "tf32"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-frames", type=int, default=1, help="frames of the oracle's sample (0 leaves it out)")
    ap.add_argument("--flow-steps", type=int, default=16, help="timed steps per flow leg (0 leaves them out)")
    ap.add_argument("--flow-warmup", type=int, default=84, help="untimed flow increments before the timed ones")
    ap.add_argument("--v480-steps", type=int, default=20, help="timed steps of the 480p video leg (0: out)")
    ap.add_argument("--fp64-steps", type=int, default=8, help="timed steps of the FP64 path on the 480p leg")
    ap.add_argument("--project-batches", type=int, default=16)
    ap.add_argument("--variant-steps", type=int, default=24)
    ap.add_argument("--serving-seconds", type=float, default=2.0)
    ap.add_argument("--no-sweep", action="store_true",
                    help="leave out the other precision of the 1080p stream (same warm-up and timed steps)")
    ap.add_argument("--profile-case", choices=["c4_update", "flow_project", "c4_stage2", "noise_update"],
                    help="run one small case for ncu instead of the benchmark")
    ap.add_argument("--profile-warm", type=int, default=24, help="warm-up increments of the c4_update case")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case(args.profile_case, args.profile_warm, args.precision)
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2211_12487_gb300 import ttice as T

    seed = replica_seed(rank)
    live = measure_matmul_peaks()
    peaks, peak_kind = _peaks_file()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    barrier()
    with ClockSampler(local) as clk:
        hl = run_headline(T, args, dev, seed, args.precision)
    barrier()
    total_ms = max_over_ranks(hl["total_ms"], ws, dev)
    N = math.prod(DIMS)
    value = whole_job_rate(ws, args.steps * BATCH * N, total_ms / 1e3)

    e2e = None
    if not args.no_e2e:
        dt, h2d, d2h = run_e2e(T, args, dev, seed, args.precision)
        e2e = {"value": whole_job_rate(ws, args.steps * BATCH * N, max_over_ranks(dt, ws, dev)), "unit": "elements/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    side = {}
    if rank == 0 and not args.no_sweep:
        try:
            rows = {args.precision: sweep_row(hl, args.steps)}
            for p in ("tf32", "fp32"):
                if p not in rows:
                    rows[p] = sweep_row(run_headline(T, args, dev, seed, p), args.steps)
            side["precision_sweep"] = {
                "workload": WORKLOAD, "rows": rows,
                "fp64": "not run at this size: the FP64 GPU path takes ~36x the mixed path's time per update "
                        "(measured on the 480p stream, video_480p.fp64_path)",
                "not_built": "bf16 and split-bf16 (TTICE_BF16, TTICE_SPLIT_BF16 are rejected by ttice_create)"}
        except Exception as e:
            side["precision_sweep"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        for key, fn in (("flow", lambda: {f"eps_{e}": run_flow(T, e, args.flow_warmup, args.flow_steps)
                                          for e in (0.05, 0.01)} if args.flow_steps > 0 else None),):
            try:
                side[key] = fn()
            except Exception as e:
                side[key] = {"error": f"{type(e).__name__}: {e}"}
        if args.v480_steps > 0:
            try:
                mixed, built, Y480 = run_video480(T, args, "fp32", args.v480_steps)
                fp64 = run_video480(T, args, "fp64", min(args.fp64_steps, args.v480_steps))[0] if args.fp64_steps > 0 else None
                side["video_480p"] = {"workload": "video 480x640x3 as 20x24x20x32x3, fp32 input, eps=0.1, 12 blobs, "
                                                  "noise 0.01, increments of 8 frames",
                                      "mixed": {k: v for k, v in mixed.items() if k != "prof"},
                                      "fp64_path": {k: v for k, v in fp64.items() if k != "prof"} if fp64 else None,
                                      "roofline_k1": phase_roofline(mixed["prof"], "k1_stage1", peaks, peak_kind, live)}
                if args.project_batches > 0:
                    side["project"] = run_project(T, built, args.project_batches)
                if args.variant_steps > 0:
                    side["paper_variants"] = run_variants(T, Y480, min(args.variant_steps, Y480.shape[0] // 8))
                del Y480
                torch.cuda.empty_cache()
            except Exception as e:
                side["video_480p"] = {"error": f"{type(e).__name__}: {e}"}
        if args.serving_seconds > 0:
            try:
                side["serving"] = run_serving(args.serving_seconds)
            except Exception as e:
                side["serving"] = {"error": f"{type(e).__name__}: {e}"}

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    prof = hl["prof"]
    names = [k for k in prof if k != "updates"]
    share = {n: round(prof[n]["ms"] / max(hl["total_ms"], 1e-9), 4) for n in names}
    dom = max(names, key=lambda n: prof[n]["ms"])
    roof = phase_roofline(prof, dom, peaks, peak_kind, live)
    if roof is not None:
        roof["traffic"] = None  # DRAM counters are taken from ncu captures (profiles/), not in this run
    flow = side.get("flow")
    if isinstance(flow, dict):
        for key, leg in flow.items():
            if not isinstance(leg, dict) or "prof" not in leg:
                continue
            p = leg.pop("prof")
            leg["roofline_k1"] = phase_roofline(p, "k1_stage1", peaks, peak_kind, live)
            if leg["skip_path_ms"]:
                t = leg["skip_path_ms"]["p50"] / 1e3
                t_roof = max(leg["skip_step_bytes"] / (peaks["hbm_gbs"] * 1e9), leg["skip_step_flops"] / (live["tf32_tflops"] * 1e12))
                leg["roofline_skip_step"] = {"t_roof_ms": t_roof * 1e3, "t_ms": t * 1e3, "frac": t_roof / t,
                                             "bytes": leg["skip_step_bytes"], "flops": leg["skip_step_flops"],
                                             "rule": "max(algorithmic bytes / HBM, algorithmic flops / TF32 peak) / measured"}
    cpu = None
    if args.cpu_frames > 0:
        v, busy, threads = oracle_sample(args.cpu_frames, seed=seed)
        cpu = {"value": v, "unit": "elements/s", "cores": threads, "kind": "oracle",
               "sample": f"first increment of {args.cpu_frames} frame(s) of the same stream from empty cores ({busy:.1f} s CPU)"}
    steps = hl["steps"]
    line = {
        "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "tf32": "tf32", "fp64": "f64"}[args.precision], "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch": BATCH, "precision": args.precision,
                   "l2": f"each step reads a fresh 796 MB increment of a {(args.warmup + args.steps) * BATCH * N * 4 / 1e9:.1f} GB "
                         "pre-generated stream (inputs larger than L2)",
                   "parallelism": f"replicas{ws}"},
        "latency_ms": {"p50": statistics.median(hl["lat"]), "p99": percentile(hl["lat"], 0.99), "max": max(hl["lat"])},
        "increments": {"timed": args.steps, "skipped": sum(s["skipped"] for s in steps),
                       "final_ranks": steps[-1]["ranks"], "new_dirs_last": steps[-1]["new_dirs"],
                       "core_elements": hl["core_elems"], "compression_ratio": hl["n_obs"] * N / max(hl["core_elems"], 1),
                       "capacity_growths": hl["grows"], "device_gb": hl["device_gb"],
                       "krylov_solves": sum(s["krylov"] for s in steps),
                       "krylov_fallbacks": sum(s["krylov_fallbacks"] for s in steps),
                       "eps_check": {"eps": EPS, "rel_err_last": hl["errs"][-1],
                                     "over_eps": hl["errs"][-1] > EPS * (1 + 1e-9)}},
        "roofline": roof,
        "dominant_phase": dom,
        "phase_share": share,
        "phase_roofline": {n: phase_roofline(prof, n, peaks, peak_kind, live) for n in names},
        "peaks": {"hbm_gbs": peaks["hbm_gbs"], "bf16_tflops": peaks["bf16_tflops"], "kind": peak_kind, **live},
        **side,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(hl["launches"]),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
