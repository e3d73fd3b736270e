#!/usr/bin/env python
"""Throughput of the fused 25-point wave step (Gpoint-updates/s, % of HBM roofline).

One bench step = one whole shot of the 512^3 workload (448^3 inner region +
32-point PML, layered velocity model, 10 Hz Ricker source, 12,544 surface
receivers, 1000 time steps) through ``run_shot`` of the C ABI: every row of
the hot path (interior update, fused PML, source injection, receiver
sampling, the time loop) runs in each step.  Inputs are resident in HBM when
the timed region starts; each of the four fields (u^n, u^{n-1}, m, phi) is
~571 MB, far above the 129 MB L2, so no L2 flush is needed between steps.
The same JSON line carries the end-to-end figure (host buffers), the roofline
of the step kernel, the 16-bit storage legs, a serving leg and a gradient leg.

--impl reference times the fp64 CPU oracle on the host cores on bounded
samples of the same workload.  Under torchrun every rank runs its own
replica shot (shots are independent: weak scaling, no collective on the data
path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "25-pt stencil Gpoint-updates/s"
UNIT = "Gpt/s"
HBM_FALLBACK_GBS = 6800.0

# DRAM bytes per launch of the step kernel measured by ncu
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by the sha256 of the
# kernel source it was measured on (comments and whitespace removed); a
# changed kernel reports null.
NCU_TRAFFIC = {
    # ncu on the 512^3 + 32-point-PML step: 1.959 GB read + 0.678 GB written per launch
    "c661d56f6bfa4b42": 2.638e9,
}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["seisgb", "reference"], default="seisgb")
    p.add_argument("--no-cpu-baseline", action="store_true",
                   help="skip the oracle CPU-baseline leg (profiling runs)")
    p.add_argument("--roofline-launches", type=int, default=100)
    p.add_argument("--serve-requests", type=int, default=256,
                   help="shot requests in the serving leg (0: skip)")
    p.add_argument("--grad-shots", type=int, default=16,
                   help="shots of the adjoint-gradient leg (0: skip)")
    p.add_argument("--grad-workers", type=int, default=8,
                   help="gradient shots in flight at once (host threads, one stream each)")
    p.add_argument("--oracle-steps", type=int, default=40,
                   help="time steps per oracle sample (CPU baseline / reference arm)")
    return p.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _workload():
    from paper_2009_04619_gb300 import synth
    return synth.LARGE


def _kernel_hash():
    """sha256 of the step kernel's sources with comments and whitespace removed
    (a comment edit does not change what the counters were measured on)."""
    import re
    h = hashlib.sha256()
    for f in ("step_kernel.cuh", "ptx.cuh", "step_config.cuh"):
        with open(os.path.join(ROOT, "paper_2009_04619_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("".join(src.split()).encode())
    return h.hexdigest()[:16]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def _alg_bytes_per_launch(w, wave_bytes=4, wave_fields=3):
    """Compulsory bytes of one step: read u^n, u^{n-1}, m and write u^{n+1}
    (3 x wave_bytes + 4 B of m per point: 16 B in fp32, 10 B with 16-bit
    wavefields; the difference form reads u^n, d^n and writes u^{n+1}, d^{n+1}:
    wave_fields = 4, 12 B in bf16) plus the fp32 phi read + write (8 B) at PML
    points."""
    N = w.points
    inner = w.nx * w.ny * w.nz
    return (wave_fields * wave_bytes + 4) * N + 8 * (N - inner)


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.uuid], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _time_oracle(w, vel, wav, src, rec, steps, nthreads):
    """Seconds for `steps` oracle time steps of workload w (oracle set-up time of
    the same call with zero steps subtracted)."""
    import oracle
    vmax = float(vel.max())
    dt = float(np.float32(w.cfl_fraction * oracle.cfl_dt(vmax, w.h, w.h, w.h)))
    g = oracle.Grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax=vmax,
                    r0=float(np.float32(1e-3)))
    t = time.perf_counter()
    oracle.run_shot(g, vel, wav, 0, src, rec, nthreads=nthreads, want_state=False)
    t0 = time.perf_counter() - t
    t = time.perf_counter()
    oracle.run_shot(g, vel, wav, steps, src, rec, nthreads=nthreads, want_state=False)
    ts = time.perf_counter() - t
    return max(ts - t0, 1e-9), ts, t0


def _serving(a, seisgb, synth, single_gpts):
    """Continuous-batching leg: Poisson arrivals at 0.8x the capacity implied by
    the single-shot throughput; shots/s and latency percentiles (submit ->
    traces on the host, measured by the server)."""
    import threading

    reqs = synth.serving_requests(a.serve_requests, seed=4)
    work = []
    for r in reqs:
        vmax = float(r["velocity"].max())
        g0 = seisgb.make_grid(r["nx"], r["ny"], r["nz"], r["nb"], r["h"], r["h"], r["h"], 1.0, vmax)
        dt = float(np.float32(0.4 * seisgb.cfl_dt(g0, vmax)))
        g = seisgb.make_grid(r["nx"], r["ny"], r["nz"], r["nb"], r["h"], r["h"], r["h"], dt, vmax)
        work.append((g, r, synth.ricker(r["nt"], dt, r["fp"])))
    pts = [float(np.prod(r["velocity"].shape)) * r["nt"] for r in reqs]
    # single-stream capacity of this mix: each grid size's throughput when it
    # runs alone (run_shot, 300 steps), weighted by the mix's work
    import torch
    solo = {}
    for key in sorted({r["velocity"].shape for r in reqs}):
        g, r, wav = next(x for x in work if x[1]["velocity"].shape == key)
        d_v = torch.from_numpy(r["velocity"]).cuda()
        d_w = torch.from_numpy(wav[:300].copy()).cuda()
        tr = torch.zeros((300, r["rec"].shape[0]), device="cuda")
        seisgb.run_shot(g, d_v, d_w, 300, r["src"], r["rec"], tr)
        torch.cuda.synchronize()
        t = time.perf_counter()
        seisgb.run_shot(g, d_v, d_w, 300, r["src"], r["rec"], tr)
        torch.cuda.synchronize()
        solo[key] = float(np.prod(key)) * 300 / (time.perf_counter() - t) / 1e9
    service = [float(np.prod(r["velocity"].shape)) * r["nt"] / (solo[r["velocity"].shape] * 1e9)
               for r in reqs]
    capacity = 1.0 / float(np.mean(service))  # shots/s, one shot at a time
    rate = 0.8 * capacity
    rng = np.random.default_rng(44)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
    tickets = [None] * len(reqs)
    with seisgb.Server(96 << 30, max_slots=16, steps_per_graph=16) as sv:
        t0 = time.perf_counter()

        def client():
            for i, (g, r, wav) in enumerate(work):
                d = arrivals[i] - (time.perf_counter() - t0)
                if d > 0:
                    time.sleep(d)
                tickets[i] = sv.submit(g, r["velocity"], wav, r["nt"], r["src"], r["rec"])

        th = threading.Thread(target=client)
        th.start()
        lat, queue = [], []
        for i, (g, r, wav) in enumerate(work):
            while tickets[i] is None:
                time.sleep(0.0005)
            rc, res, _ = sv.poll(tickets[i], r["nt"], r["rec"].shape[0], timeout_us=600_000_000)
            lat.append(res.latency_ms)
            queue.append(res.queue_ms)
        th.join()
        total = time.perf_counter() - t0
        st = sv.stats()
    lat = np.array(lat)
    # overload: the first 64 requests submitted at once -> batched capacity
    K = min(64, len(work))
    with seisgb.Server(96 << 30, max_slots=16, steps_per_graph=16) as sv:
        t1 = time.perf_counter()
        tk = [sv.submit(g, r["velocity"], wav, r["nt"], r["src"], r["rec"]) for g, r, wav in work[:K]]
        for t, (g, r, wav) in zip(tk, work[:K]):
            sv.poll(t, r["nt"], r["rec"].shape[0], timeout_us=600_000_000)
        t_over = time.perf_counter() - t1
    overload = {"requests": K, "shots_per_s": K / t_over,
                "gpts_aggregate": sum(pts[:K]) / t_over / 1e9,
                "single_stream_shots_per_s": K / sum(service[:K])}
    return {"requests": len(reqs), "shots_per_s": len(reqs) / total,
            "gpts_aggregate": sum(pts) / total / 1e9, "offered_rate_per_s": rate,
            "single_stream_capacity_per_s": capacity,
            "solo_gpts": {"x".join(str(v) for v in k[::-1]): round(v, 1) for k, v in solo.items()},
            "mean_solo_service_ms": float(np.mean(service)) * 1e3,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_queue_ms": float(np.mean(queue)), "wall_s": total,
            "graph_replays": int(st.graph_replays), "step_launches": int(st.step_launches),
            "overload": overload,
            "config": "Poisson arrivals at 0.8x the single-stream capacity of this mix; grids 128^3, "
                      "192x192x256, 256^3, 384x384x256 (PML 16); 500-2000 steps; seed 4; "
                      "16 slots, 16 steps per graph"}


def _gradient_alg_bytes(w, nt, ckpt, fold=32):
    """Compulsory HBM bytes of one gradient shot: the forward steps (16 B per
    point, +8 B of phi on the PML), the checkpoint saves and restores (3 fields
    read + written each), the recomputed steps (+4 B: g^n written), the adjoint
    steps (w^{k+1}, w^{k+2}, m, g^{k-1}, S read; w^k, S written: 28 B, +8 B of
    mu on the PML) and the fp64 folds of S (24 B per point every `fold` steps)."""
    N = w.points
    P = N - w.nx * w.ny * w.nz
    segs = -(-nt // ckpt)
    return (nt * ((16 + 20 + 28) * N + 24 * P) + 2 * segs * 24 * N
            + -(-nt // fold) * 24 * N)


def _gradient(a, seisgb, synth, peak, uuid=None):
    """Adjoint-gradient leg: 16 shots of the 256^3 / 2000-step workload, misfit
    against traces of the unperturbed model, gradients summed over the shots
    (fp64); shots/s, forward-equivalent Gpt/s and the whole computation's
    algorithmic bytes per second against the HBM peak.  Each rank keeps
    `--grad-workers` shots in flight on as many streams (host threads; 8 by
    default, which divides the 16 shots evenly, ~16 GB of scratch each); under
    torchrun the shots are split across ranks and one fp64 all-reduce sums the
    gradients."""
    import torch
    from paper_2009_04619_gb300 import replicas
    rank, world, _ = _dist()
    w = synth.GRADIENT
    v, v_obs = synth.gradient_models(w)
    vmax = float(max(v.max(), v_obs.max()))
    g0 = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, 1.0, vmax)
    dt = float(np.float32(w.cfl_fraction * seisgb.cfl_dt(g0, vmax)))
    g = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax)
    nt, C = w.nt, w.extra["ckpt_every"]
    wav = synth.ricker(nt, dt, w.fp)
    rec = w.receivers()
    shots = synth.shot_grid(w)[:a.grad_shots]
    mine = replicas.my_shots(len(shots), rank, world)
    d_v = torch.from_numpy(v).cuda()
    d_vo = torch.from_numpy(v_obs).cuda()
    d_w = torch.from_numpy(wav).cuda()
    obs = {}
    for i in mine:
        o = torch.zeros((nt, rec.shape[0]), dtype=torch.float32, device="cuda")
        seisgb.run_shot(g, d_vo, d_w, nt, shots[i], rec, o)
        obs[i] = o
    # several shots in flight on as many streams: their kernels fill each other's
    # partial waves (measured 1.19x over one stream on this workload)
    workers = max(1, a.grad_workers)
    streams = [torch.cuda.Stream() for _ in range(workers)]
    grads = [torch.zeros(v.shape, dtype=torch.float64, device="cuda") for _ in range(workers)]

    def shot_fn(i, k):
        return seisgb.adjoint_shot(g, d_v, d_w, nt, shots[i], rec, obs[i], grads[k], ckpt_every=C,
                                   stream=streams[k]), grads[k]

    # warm-up: one shot on every worker at once, so that each worker's scratch
    # (~16 GB per shot in flight) is allocated and first touched before timing
    replicas.gradient_sum(shot_fn, min(len(shots), workers * world), grads[0], workers=workers,
                          streams=streams)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    sampler = ClockSampler(uuid) if uuid else None
    if sampler:
        sampler.start()
    e0.record(stream)
    J, total = replicas.gradient_sum(shot_fn, len(shots), grads[0], workers=workers,
                                     streams=streams)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = sampler.stop() if sampler else None
    t = replicas.max_over_ranks(e0.elapsed_time(e1) / 1e3, device=grads[0].device)
    tr = torch.zeros((nt, rec.shape[0]), dtype=torch.float32, device="cuda")
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for src in shots[:2]:
        seisgb.run_shot(g, d_v, d_w, nt, src, rec, tr)
    f1.record(stream)
    torch.cuda.synchronize()
    t_fwd = f0.elapsed_time(f1) / 1e3 / min(2, len(shots))
    ns = len(shots)
    alg = _gradient_alg_bytes(w, nt, C)
    gbs = alg * ns / t / 1e9
    return {"workload": w.name, "grid": list(w.shape), "nb": w.nb, "nt": nt, "shots": ns,
            "ranks": world, "collective": "one fp64 all-reduce of the gradient" if world > 1 else None,
            "streams": workers,
            "ckpt_every": C, "nrec": int(rec.shape[0]),
            "shots_per_s": ns / t, "ms_per_shot": t / ns * 1e3,
            "gpts_forward_equivalent": w.points * nt * ns / t / 1e9,
            "forward_ms_per_shot": t_fwd * 1e3, "ratio_to_forward": t / ns / t_fwd,
            "alg_bytes_per_shot": alg, "achieved_gbs": gbs, "frac": gbs / peak,
            "misfit": J, "grad_l2": float(total.norm()), "clocks": clk,
            "grad_finite": bool(torch.isfinite(total).all()),
            "accuracy": "gradient vs the fp64 oracle adjoint (32^3, 50 steps) and the oracle vs "
                        "central differences: tests"}


def _stencil_step_ms(g, fmt, seisgb, dev, d_v, dt, src, d_w, launches, nt):
    """Mean time of one stencil_step launch on 16-bit fields (back to back, CUDA
    events on the launching stream), the per-launch unit of the roofline."""
    import torch
    L = seisgb.layout(g)
    tdt = torch.float16 if fmt == seisgb.FP16_SCALED else torch.bfloat16
    u = [torch.zeros(int(L.elems), dtype=tdt, device=dev) for _ in range(2)]
    phi = torch.zeros(int(L.elems), dtype=torch.float32, device=dev)
    d_m = torch.zeros(int(L.elems), dtype=torch.float32, device=dev)
    g32 = seisgb.make_grid(g.nx, g.ny, g.nz, g.nb, g.dx, g.dy, g.dz, g.dt, g.vmax)
    seisgb.pack(g32, (d_v * dt) ** 2, d_m)
    scale = torch.tensor([1.0] * 4 + [0.0] * 4, dtype=torch.float32, device=dev)
    sc = scale if fmt == seisgb.FP16_SCALED else None
    for n in range(3):
        seisgb.stencil_step(g, u[n % 2], u[(n + 1) % 2], d_m, phi, n, source=(*src, d_w),
                            scale_state=sc)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for n in range(launches):
        seisgb.stencil_step(g, u[n % 2], u[(n + 1) % 2], d_m, phi, (n + 3) % nt,
                            source=(*src, d_w), scale_state=sc)
    r1.record(stream)
    torch.cuda.synchronize()
    seisgb.device_status()
    return r0.elapsed_time(r1) / launches


def _temporal(a, seisgb, w, vel, vmax, dt, src, rec, d_v, d_w, d_tr, dev, barrier, single, world):
    """run_shot with SCHED_PAIRS (temporal blocking) on the benchmark workload (CUDA events around
    a.steps shots after one warm-up shot) and the mean time of one
    stencil_step2 pair (back to back)."""
    import torch
    from paper_2009_04619_gb300 import replicas
    g2 = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax, schedule=seisgb.SCHED_PAIRS)
    seisgb.run_shot(g2, d_v, d_w, w.nt, src, rec, d_tr)
    barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        seisgb.run_shot(g2, d_v, d_w, w.nt, src, rec, d_tr)
    e1.record(stream)
    barrier()
    ms = replicas.max_over_ranks(e0.elapsed_time(e1), device=dev) / a.steps
    val = w.points * w.nt * world / (ms / 1e3) / 1e9
    L = seisgb.layout(g2)
    f = [torch.zeros(int(L.elems), dtype=torch.float32, device=dev) for _ in range(6)]
    seisgb.pack(g2, (d_v * dt) ** 2, f[4])
    M = max(10, a.roofline_launches // 4)
    for k in range(3):
        p = k % 2
        seisgb.stencil_step2(g2, f[2 * p], f[2 * p + 1], f[2 - 2 * p], f[3 - 2 * p], f[4], f[5],
                             2 * k, source=(*src, d_w))
    torch.cuda.synchronize()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for k in range(M):
        p = k % 2
        seisgb.stencil_step2(g2, f[2 * p], f[2 * p + 1], f[2 - 2 * p], f[3 - 2 * p], f[4], f[5],
                             (2 * k) % (w.nt - 1), source=(*src, d_w))
    r1.record(stream)
    torch.cuda.synchronize()
    seisgb.device_status()
    pair_ms = r0.elapsed_time(r1) / M
    del f
    return {"value": val, "unit": UNIT, "ms_per_shot": ms, "vs_single_step": val / single,
            "pair_ms": pair_ms, "ms_per_step_in_pairs": pair_ms / 2,
            "default": "off (SCHED_PAIRS is opt-in); results are bit-identical to one step per launch",
            "design": "two-step kernel on the inner region shrunk by 4 points, two single-step "
                      "shell launches on the rest"}


def _small_case(a, seisgb, synth, dev, barrier):
    """Gpt/s of the small forward-modelling case (64^3 inner + 16-point PML,
    constant 2000 m/s, 100 steps) through run_shot, device-resident inputs,
    CUDA events around `reps` back-to-back shots after a warm-up."""
    import torch
    w = synth.SMALL
    vel = w.velocity()
    g0 = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, 1.0, w.v_const)
    dt = float(np.float32(w.cfl_fraction * seisgb.cfl_dt(g0, w.v_const)))
    g = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, w.v_const)
    rec = w.receivers()
    d_v = torch.from_numpy(vel).to(dev)
    d_w = torch.from_numpy(synth.ricker(w.nt, dt, w.fp)).to(dev)
    tr = torch.zeros((w.nt, rec.shape[0]), dtype=torch.float32, device=dev)
    for _ in range(max(3, a.warmup)):
        seisgb.run_shot(g, d_v, d_w, w.nt, w.source(), rec, tr)
    barrier()
    reps = 20
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        seisgb.run_shot(g, d_v, d_w, w.nt, w.source(), rec, tr)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1) / reps
    return {"workload": w.name, "grid": list(w.shape), "nt": w.nt, "value": w.points * w.nt / ms / 1e6,
            "unit": UNIT, "ms_per_shot": ms,
            "note": "fields fit in L2 (4 x 4.5 MB): no roofline claim; includes run_shot's per-call "
                    "set-up (allocation, m, velocity range check, graph capture)"}


def run_reference(a):
    rank, world, _ = _dist()
    if rank != 0:
        return
    w = _workload()
    vel = w.velocity()
    from paper_2009_04619_gb300 import synth
    import oracle
    oracle.build()
    vmax = float(vel.max())
    dt = float(np.float32(w.cfl_fraction * oracle.cfl_dt(vmax, w.h, w.h, w.h)))
    wav = synth.ricker(w.nt, dt, w.fp)
    rec = w.receivers()
    cores = os.cpu_count() or 1
    S = a.oracle_steps
    for _ in range(a.warmup):
        _time_oracle(w, vel, wav, w.source(), rec, 1, cores)
    tot = 0.0
    for _ in range(a.steps):
        dt_s, _, _ = _time_oracle(w, vel, wav, w.source(), rec, S, cores)
        tot += dt_s
    pts = w.points * S * a.steps
    val = pts / tot / 1e9
    sample = (f"{S} of {w.nt} time steps of the {w.name} workload per bench step "
              f"(oracle set-up time subtracted), fp64 oracle, {cores} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": tot / a.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w.name, "grid": list(w.shape), "nb": w.nb,
                                        "nt_sampled": S},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
        return
    import torch
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2009_04619_gb300 import build, replicas, seisgb, synth
    build.build()
    seisgb.lib()
    w = _workload()
    vel = w.velocity()
    vmax = float(vel.max())
    g0 = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, 1.0, vmax)
    dt = float(np.float32(w.cfl_fraction * seisgb.cfl_dt(g0, vmax)))
    g = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax)
    wav = synth.ricker(w.nt, dt, w.fp)
    src = w.source()
    rec = w.receivers()
    nrec = rec.shape[0]
    d_v = torch.from_numpy(vel).to(dev)
    d_w = torch.from_numpy(wav).to(dev)
    d_tr = torch.zeros((w.nt, nrec), dtype=torch.float32, device=dev)

    for _ in range(a.warmup):
        seisgb.run_shot(g, d_v, d_w, w.nt, src, rec, d_tr)

    uuid = torch.cuda.get_device_properties(dev).uuid
    uuid = "GPU-" + str(uuid) if not str(uuid).startswith("GPU-") else str(uuid)
    clocks = ClockSampler(uuid)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    time.sleep(0.3)
    seisgb.launch_count(reset=True)
    barrier()
    e0.record(stream)
    for _ in range(a.steps):
        seisgb.run_shot(g, d_v, d_w, w.nt, src, rec, d_tr)
    e1.record(stream)
    barrier()
    launches = seisgb.launch_count(reset=True)
    clk = clocks.stop()
    ms = replicas.max_over_ranks(e0.elapsed_time(e1), device=dev)
    ms_per_step = ms / a.steps
    value = replicas.job_rate(w.points * w.nt * a.steps, ms / 1e3, world) / 1e9

    # end to end through the C ABI with pinned host buffers, right after the
    # device-resident timing (same GPU state): velocity and wavelet
    # copied in, traces copied out, every step
    h_v = torch.from_numpy(vel).pin_memory()
    h_w = torch.from_numpy(wav).pin_memory()
    h_tr = torch.zeros((w.nt, nrec), dtype=torch.float32).pin_memory()
    seisgb.run_shot(g, h_v, h_w, w.nt, src, rec, h_tr)
    barrier()
    clocks_e2e = ClockSampler(uuid)
    clocks_e2e.start()
    time.sleep(0.3)
    t = time.perf_counter()
    for _ in range(a.steps):
        seisgb.run_shot(g, h_v, h_w, w.nt, src, rec, h_tr)
    barrier()
    e2e_s = replicas.max_over_ranks(time.perf_counter() - t, device=dev)
    clk_e2e = clocks_e2e.stop()
    e2e_val = replicas.job_rate(w.points * w.nt * a.steps, e2e_s, world) / 1e9
    h2d = vel.nbytes + wav.nbytes + rec.nbytes + 12
    d2h = w.nt * nrec * 4

    # dominant kernel: back-to-back fused steps on the same grid, CUDA events on
    # the launching stream
    L = seisgb.layout(g)
    bufs = [torch.zeros(int(L.elems), dtype=torch.float32, device=dev) for _ in range(3)]
    d_m = torch.zeros(int(L.elems), dtype=torch.float32, device=dev)
    seisgb.pack(g, (d_v * dt) ** 2, d_m)
    M = a.roofline_launches
    for n in range(3):
        seisgb.stencil_step(g, bufs[n % 2], bufs[(n + 1) % 2], d_m, bufs[2], n, source=(*src, d_w))
    torch.cuda.synchronize()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for n in range(M):
        seisgb.stencil_step(g, bufs[n % 2], bufs[(n + 1) % 2], d_m, bufs[2], n % w.nt,
                            source=(*src, d_w))
    r1.record(stream)
    torch.cuda.synchronize()
    kern_ms = r0.elapsed_time(r1) / M
    alg = _alg_bytes_per_launch(w)
    peak, peak_kind = _peaks()
    achieved = alg / (kern_ms / 1e3) / 1e9
    traffic = NCU_TRAFFIC.get(_kernel_hash())
    del bufs, d_m

    # the same shot with 16-bit wavefield storage (fp32 arithmetic); the
    # difference forms (fp16_diff, bf16_diff) are timed inside the shot
    precision = {}
    for fname, fmt in (("fp16_scaled", seisgb.FP16_SCALED), ("bf16", seisgb.BF16),
                       ("fp16_diff", seisgb.FP16_DIFF), ("bf16_diff", seisgb.BF16_DIFF)):
        gp = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax, storage=fmt)
        seisgb.run_shot(gp, d_v, d_w, w.nt, src, rec, d_tr)
        barrier()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(a.steps):
            seisgb.run_shot(gp, d_v, d_w, w.nt, src, rec, d_tr)
        p1.record(stream)
        barrier()
        pms = replicas.max_over_ranks(p0.elapsed_time(p1), device=dev) / a.steps
        diff = fmt in (seisgb.BF16_DIFF, seisgb.FP16_DIFF)
        alg16 = _alg_bytes_per_launch(w, wave_bytes=2, wave_fields=4 if diff else 3)
        if diff:  # no single-step entry point: the step time inside the shot
            kms, kname = pms / w.nt, "diff_step_kernel (in run_shot)"
        else:
            kms = _stencil_step_ms(g=gp, fmt=fmt, seisgb=seisgb, dev=dev, d_v=d_v, dt=dt, src=src,
                                   d_w=d_w, launches=M, nt=w.nt)
            kname = "fused_step_kernel (stencil_step)"
        precision[fname] = {
            "value": w.points * w.nt * world / (pms / 1e3) / 1e9, "unit": UNIT,
            "ms_per_step": pms, "alg_bytes_per_launch": alg16,
            "achieved_gbs": alg16 / (pms / w.nt / 1e3) / 1e9,
            "frac": alg16 / (pms / w.nt / 1e3) / 1e9 / peak,
            "vs_fp32": (w.points * w.nt * world / (pms / 1e3) / 1e9) / value,
            "roofline": {"bound": "hbm", "kernel": kname,
                         "kernel_ms": kms, "achieved": alg16 / (kms / 1e3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": alg16 / (kms / 1e3) / 1e9 / peak,
                         "alg_bytes_per_launch": alg16},
            "error": "relative L2 vs the fp64 oracle: see the 256^3 x 1000-step precision test"}
        if diff:
            precision[fname]["state"] = ("u^n and d^n = u^n - u^{n-1} (difference form), "
                                         + ("fp16 with a scale each" if fmt == seisgb.FP16_DIFF
                                            else "bf16"))

    # temporal blocking: the same shot with SCHED_PAIRS (two steps per HBM
    # pass on the PML-free interior, identical results), and the pair unit
    temporal = _temporal(a, seisgb, w, vel, vmax, dt, src, rec, d_v, d_w, d_tr, dev, barrier,
                         value, world)

    # the small forward-modelling case (64^3 inner + 16-point PML, 100 steps):
    # whole shots through run_shot, device-resident inputs (its four fields fit
    # in L2, so no roofline claim is made for it)
    small = _small_case(a, seisgb, synth, dev, barrier)

    serving = _serving(a, seisgb, synth, value) if a.serve_requests > 0 else None
    gradient = _gradient(a, seisgb, synth, peak, uuid) if a.grad_shots > 0 else None

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "grid": list(w.shape), "inner": [w.nz, w.ny, w.nx],
                   "nb": w.nb, "nt": w.nt, "nrec": nrec, "dt": dt,
                   "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (4 fields x 571 MB), no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "fused_step_kernel", "kernel_ms": kern_ms,
                     "alg_bytes_per_launch": alg, "peak_source": peak_kind,
                     "step_ms_in_shot": ms_per_step / w.nt},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s / a.steps * 1e3,
                "clocks": clk_e2e},
        "gpu_launches": launches,
        "clocks": clk,
        "precision": precision,
        "temporal_blocking": temporal,
        "small_case": small,
        "serving": serving,
        "gradient": gradient,
    }
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        S = a.oracle_steps
        dt_s, ts, t0 = _time_oracle(w, vel, wav, src, rec, S, cores)
        S1 = max(1, S // 20)
        dt_1, _, _ = _time_oracle(w, vel, wav, src, rec, S1, 1)
        ws = synth.SMALL
        vs = ws.velocity()
        dts = float(np.float32(ws.cfl_fraction * oracle.cfl_dt(ws.v_const, ws.h, ws.h, ws.h)))
        wavs = synth.ricker(ws.nt, dts, ws.fp)
        small_all, _, _ = _time_oracle(ws, vs, wavs, ws.source(), ws.receivers(), ws.nt, cores)
        small_1, _, _ = _time_oracle(ws, vs, wavs, ws.source(), ws.receivers(), ws.nt, 1)
        out["cpu_baseline"] = {
            "value": w.points * S / dt_s / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"{S} of {w.nt} time steps of the {w.name} workload "
                       f"({ts:.1f} s call minus {t0:.1f} s oracle set-up), fp64, {cores} threads"),
            "single_thread": {"value": w.points * S1 / dt_1 / 1e9, "unit": UNIT, "cores": 1,
                              "sample": f"{S1} time steps of the same workload, one thread"},
            "small_case": {"workload": ws.name, "unit": UNIT,
                           "value": ws.points * ws.nt / small_all / 1e9, "cores": cores,
                           "value_single_thread": ws.points * ws.nt / small_1 / 1e9,
                           "sample": "the whole 100-step shot, all cores and one thread"}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
