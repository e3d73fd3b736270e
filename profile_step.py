"""Launch the fused step kernel back to back on a synthetic grid and report its
time per launch (CUDA events) -- a small script for timing and for ncu captures.

    python profile_step.py --n 256 --nb 32 --launches 20
    python profile_step.py --adjoint --n 256 --nb 16 --nt 200
    python profile_step.py --storage fp16 --n 512 --nb 32 --nt 40
    python profile_step.py --serve 16
    python profile_step.py --step2 --n 512 --nb 32 --launches 20
    python profile_step.py --shots --n 256 --nb 16 --nt 200 --launches 3

With --adjoint it runs one misfit-gradient shot instead (layered model with a
Gaussian anomaly, observed traces from the model without it) and reports its
time beside a forward shot of the same length.  With --storage fp16 or bf16 it
runs a short run_shot with 16-bit wavefield storage (fp32 arithmetic) and
reports the time per step.  With --serve N it submits the first N requests of
the seeded serving mix at once to a 16-slot server and reports shots/s.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2009_04619_gb300 import build, seisgb, synth  # noqa: E402


def _adjoint(a):
    N, nb = a.n, a.nb
    n_in = N - 2 * nb
    shape = (N, N, N)
    v0 = synth.layered_model(shape, seed=5)
    v = (v0 * synth.gaussian_anomaly(shape, (N / 2, N / 2, N / 2), N / 12, 0.05)).astype(np.float32)
    vmax = float(max(v.max(), v0.max()))
    g0 = seisgb.make_grid(n_in, n_in, n_in, nb, 10.0, 10.0, 10.0, 1.0, vmax)
    dt = float(np.float32(0.4 * seisgb.cfl_dt(g0, vmax)))
    g = seisgb.make_grid(n_in, n_in, n_in, nb, 10.0, 10.0, 10.0, dt, vmax)
    wav = synth.ricker(a.nt, dt, 10.0)
    src = (N // 2, N // 2, nb + 2)
    rec = synth.surface_receivers(n_in, n_in, nb, 4)
    d_v0, d_v = torch.from_numpy(v0).cuda(), torch.from_numpy(v).cuda()
    d_w = torch.from_numpy(wav).cuda()
    obs = torch.zeros((a.nt, rec.shape[0]), device="cuda")
    seisgb.run_shot(g, d_v0, d_w, a.nt, src, rec, obs)
    grad = torch.zeros(shape, dtype=torch.float64, device="cuda")
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    torch.cuda.synchronize()
    e0.record()
    J = seisgb.adjoint_shot(g, d_v, d_w, a.nt, src, rec, obs, grad, ckpt_every=a.ckpt)
    e1.record()
    seisgb.run_shot(g, d_v, d_w, a.nt, src, rec, obs)
    e2.record()
    torch.cuda.synchronize()
    seisgb.device_status()
    ta, tf = e0.elapsed_time(e1), e1.elapsed_time(e2)
    print(json.dumps({"n": N, "nb": nb, "nt": a.nt, "ckpt_every": a.ckpt, "adjoint_ms": ta,
                      "forward_ms": tf, "ratio": ta / tf, "misfit": J,
                      "grad_finite": bool(torch.isfinite(grad).all())}))


def _storage(a):
    n_in = a.n - 2 * a.nb
    v = 3000.0
    fmt = {"fp32": seisgb.FP32, "fp16": seisgb.FP16_SCALED, "bf16": seisgb.BF16,
           "fp32_diff": seisgb.FP32_DIFF, "bf16_diff": seisgb.BF16_DIFF,
           "fp16_diff": seisgb.FP16_DIFF}[a.storage]
    g0 = seisgb.make_grid(n_in, n_in, n_in, a.nb, 10.0, 10.0, 10.0, 1.0, v)
    dt = float(np.float32(0.4 * seisgb.cfl_dt(g0, v)))
    g = seisgb.make_grid(n_in, n_in, n_in, a.nb, 10.0, 10.0, 10.0, dt, v, storage=fmt)
    vel = torch.full(g.shape, v, device="cuda")
    wav = torch.from_numpy(synth.ricker(a.nt, dt, 10.0)).cuda()
    src = (a.n // 2, a.n // 2, a.n // 2)
    rec = synth.surface_receivers(n_in, n_in, a.nb, 8)
    tr = torch.zeros((a.nt, rec.shape[0]), device="cuda")
    seisgb.run_shot(g, vel, wav, a.nt, src, rec, tr)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    seisgb.run_shot(g, vel, wav, a.nt, src, rec, tr)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.nt
    pts = a.n ** 3
    # wavefields read twice and written once (difference form: u^n and d^n read,
    # u^{n+1} and d^{n+1} written), 4 B m, phi read and written at PML points
    wb = 4 if a.storage.startswith("fp32") else 2
    nw = 4 if a.storage.endswith("_diff") else 3
    alg = (nw * wb + 4) * pts + 8 * (pts - n_in ** 3)
    print(json.dumps({"n": a.n, "nb": a.nb, "storage": a.storage, "nt": a.nt, "ms_per_step": ms,
                      "gpts": pts / ms / 1e6, "alg_gbs": alg / ms / 1e6}))


def _serve(a):
    import time
    reqs = synth.serving_requests(256, seed=4)[:a.serve]
    work = []
    for r in reqs:
        vmax = float(r["velocity"].max())
        g0 = seisgb.make_grid(r["nx"], r["ny"], r["nz"], r["nb"], r["h"], r["h"], r["h"], 1.0, vmax)
        dt = float(np.float32(0.4 * seisgb.cfl_dt(g0, vmax)))
        g = seisgb.make_grid(r["nx"], r["ny"], r["nz"], r["nb"], r["h"], r["h"], r["h"], dt, vmax)
        work.append((g, r, synth.ricker(r["nt"], dt, r["fp"])))
    with seisgb.Server(96 << 30, max_slots=a.slots, steps_per_graph=a.spg) as sv:
        t0 = time.perf_counter()
        tk = [sv.submit(g, r["velocity"], wav, r["nt"], r["src"], r["rec"]) for g, r, wav in work]
        for t, (g, r, wav) in zip(tk, work):
            sv.poll(t, r["nt"], r["rec"].shape[0], timeout_us=600_000_000)
        wall = time.perf_counter() - t0
        st = sv.stats()
    import os
    print(json.dumps({"requests": len(work), "slots": a.slots, "steps_per_graph": a.spg,
                      "connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS"),
                      "shots_per_s": len(work) / wall, "wall_s": wall,
                      "graph_replays": int(st.graph_replays), "wait_ms": st.wait_ms,
                      "setup_ms": st.setup_ms, "prepare_ms": st.prepare_ms,
                      "retire_ms": st.retire_ms}))


def _shots(a):
    """run_shot on an n^3 grid (PML nb, layered model, surface receivers every
    4th point, nt steps, device-resident inputs) with each time-loop schedule:
    ms per step (CUDA events around `launches` shots after a warm-up shot)."""
    n_in = a.n - 2 * a.nb
    shape = (a.n, a.n, a.n)
    vel = torch.from_numpy(synth.layered_model(shape, seed=2009)).cuda()
    vmax = float(vel.max())
    g0 = seisgb.make_grid(n_in, n_in, n_in, a.nb, 10.0, 10.0, 10.0, 1.0, vmax)
    dt = float(np.float32(0.4 * seisgb.cfl_dt(g0, vmax)))
    wav = torch.from_numpy(synth.ricker(a.nt, dt, 10.0)).cuda()
    rec = synth.surface_receivers(n_in, n_in, a.nb, 4)
    tr = torch.zeros((a.nt, rec.shape[0]), device="cuda")
    src = (a.n // 2, a.n // 2, a.nb + 2)
    out = {"n": a.n, "nb": a.nb, "nt": a.nt}
    scheds = {"step": seisgb.SCHED_STEP, "flow": seisgb.SCHED_FLOW}
    if a.storage:
        fmt = {"fp32": seisgb.FP32, "fp16": seisgb.FP16_SCALED, "bf16": seisgb.BF16,
           "fp32_diff": seisgb.FP32_DIFF, "bf16_diff": seisgb.BF16_DIFF,
           "fp16_diff": seisgb.FP16_DIFF}[a.storage]
    else:
        fmt = seisgb.FP32
    for name, sched in scheds.items():
        if fmt == seisgb.FP16_SCALED and sched == seisgb.SCHED_FLOW:
            continue
        g = seisgb.make_grid(n_in, n_in, n_in, a.nb, 10.0, 10.0, 10.0, dt, vmax, storage=fmt,
                             schedule=sched)
        seisgb.run_shot(g, vel, wav, a.nt, src, rec, tr)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.launches):
            seisgb.run_shot(g, vel, wav, a.nt, src, rec, tr)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.launches / a.nt
        out[name] = {"ms_per_step": ms, "gpts": a.n ** 3 / ms / 1e6}
    print(json.dumps(out))


def _step2(a):
    """Back-to-back pairs of steps: stencil_step2 (four buffers rotating) against
    two stencil_step launches (in place), CUDA events, same grid and fields."""
    n_in = a.n - 2 * a.nb
    h, v = 10.0, 4500.0
    g0 = seisgb.make_grid(n_in, n_in, n_in, a.nb, h, h, h, 1.0, v)
    dt = 0.4 * seisgb.cfl_dt(g0, v)
    g = seisgb.make_grid(n_in, n_in, n_in, a.nb, h, h, h, dt, v)
    L = seisgb.layout(g)
    f = [torch.zeros(int(L.elems), dtype=torch.float32, device="cuda") for _ in range(6)]
    vel = torch.full(g.shape, 3000.0, device="cuda")
    seisgb.pack(g, (vel * dt) ** 2, f[4])
    w = torch.zeros(2 * (a.warmup + a.launches) + 4, device="cuda")
    src = (a.n // 2, a.n // 2, a.n // 2)
    res = {}
    for mode in ("step2", "step"):
        def run(k, n):
            if mode == "step2":
                p = k % 2  # (f0, f1) -> (f2, f3), then back
                seisgb.stencil_step2(g, f[2 * p], f[2 * p + 1], f[2 - 2 * p], f[3 - 2 * p], f[4], f[5],
                                     n, source=(*src, w))
            else:
                seisgb.stencil_step(g, f[n % 2], f[(n + 1) % 2], f[4], f[5], n, source=(*src, w))
                seisgb.stencil_step(g, f[(n + 1) % 2], f[n % 2], f[4], f[5], n + 1, source=(*src, w))
        for k in range(a.warmup):
            run(k, 2 * k)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(a.launches):
            run(k, 2 * k)
        e1.record()
        torch.cuda.synchronize()
        seisgb.device_status()
        res[mode] = e0.elapsed_time(e1) / (2 * a.launches)
    pts = a.n ** 3
    print(json.dumps({"n": a.n, "nb": a.nb, "ms_per_step_step2": res["step2"],
                      "ms_per_step_single": res["step"], "speedup": res["step"] / res["step2"],
                      "gpts_step2": pts / res["step2"] / 1e6, "gpts_single": pts / res["step"] / 1e6}))


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=256, help="computed points per axis")
    p.add_argument("--nb", type=int, default=32)
    p.add_argument("--launches", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--lib", default=None, help="path of an alternative libseisgb.so build")
    p.add_argument("--adjoint", action="store_true", help="time one misfit-gradient shot")
    p.add_argument("--nt", type=int, default=200, help="time steps of the gradient shot")
    p.add_argument("--ckpt", type=int, default=100, help="checkpoint interval of the gradient shot")
    p.add_argument("--storage", choices=["fp32", "fp16", "bf16", "fp32_diff", "bf16_diff", "fp16_diff"], default=None,
                   help="time a short run_shot with 16-bit wavefield storage")
    p.add_argument("--serve", type=int, default=0,
                   help="submit this many requests of the serving mix to a server at once")
    p.add_argument("--slots", type=int, default=16, help="server slots (--serve)")
    p.add_argument("--spg", type=int, default=16, help="steps per graph replay (--serve)")
    p.add_argument("--shots", action="store_true",
                   help="time whole run_shot calls (layered model) with each time-loop schedule")
    p.add_argument("--step2", action="store_true",
                   help="time stencil_step2 (two steps, temporal blocking) against two stencil_step")
    a = p.parse_args(argv)
    if a.lib:
        seisgb.LIB_PATH = a.lib
    else:
        build.build()
    if a.adjoint:
        _adjoint(a)
        return
    if a.storage:
        _storage(a)
        return
    if a.serve:
        _serve(a)
        return
    if a.step2:
        _step2(a)
        return
    if a.shots:
        _shots(a)
        return
    n_in = a.n - 2 * a.nb  # nb = 0: no PML, every tile takes the interior path
    h, v = 10.0, 4500.0
    g0 = seisgb.make_grid(n_in, n_in, n_in, a.nb, h, h, h, 1.0, v)
    dt = 0.4 * seisgb.cfl_dt(g0, v)
    g = seisgb.make_grid(n_in, n_in, n_in, a.nb, h, h, h, dt, v)
    L = seisgb.layout(g)
    f = [torch.zeros(int(L.elems), dtype=torch.float32, device="cuda") for _ in range(4)]
    vel = torch.full(g.shape, 3000.0, device="cuda")
    seisgb.pack(g, (vel * dt) ** 2, f[2])
    w = torch.zeros(a.warmup + a.launches + 1, device="cuda")
    src = (a.n // 2, a.n // 2, a.n // 2)
    for n in range(a.warmup):
        seisgb.stencil_step(g, f[n % 2], f[(n + 1) % 2], f[2], f[3], n, source=(*src, w))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for n in range(a.launches):
        seisgb.stencil_step(g, f[n % 2], f[(n + 1) % 2], f[2], f[3], n, source=(*src, w))
    e1.record()
    torch.cuda.synchronize()
    seisgb.device_status()
    ms = e0.elapsed_time(e1) / a.launches
    pts = a.n ** 3
    alg = 16 * pts + 8 * (pts - n_in ** 3)
    print(json.dumps({"n": a.n, "nb": a.nb, "ms_per_launch": ms, "gpts": pts / ms / 1e6,
                      "alg_gbs": alg / ms / 1e6, "lib": a.lib or seisgb.LIB_PATH}))


if __name__ == "__main__":
    main()
