"""Parity of the CUDA path (through the C ABI) with the fp64 oracle.

Tolerances:
 - one step from random fields: per point |gpu - oracle| <= 1e-6 * S, S the
   sum of absolute values of the terms the step adds (an fp32 evaluation of
   ~30 terms has error below ~30 * 2^-24 * S = 1.8e-6 S; 1e-6 is what a
   sensible summation order achieves and still catches any wrong term, whose
   size is ~|c_m m u| ~ 1e-2 S);
 - 100 steps of the small forward-modelling case: relative L2 <= 2e-5 over the
   full wavefield and over the traces (the required bound).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_04619_gb300 import seisgb, synth
from gpu_util import abs_term_sum, abs_term_sum_points, ensure_lib, from_padded, padded_zeros, rel_l2, to_padded

pytestmark = pytest.mark.gpu

STEP_CASES = [
    # nx, ny, nz, nb, (dx, dy, dz)
    (13, 17, 11, 5, (10.0, 11.0, 12.0)),
    (90, 37, 29, 5, (10.0, 10.0, 10.0)),   # 2 x-tiles and 3 y-tiles, all ragged
    (6, 5, 7, 3, (8.0, 9.0, 10.0)),
    (130, 20, 9, 8, (10.0, 10.0, 10.0)),   # 3 x-tiles, ragged in x
    (64, 64, 64, 16, (10.0, 10.0, 10.0)),  # the small case's geometry
    (40, 33, 70, 0, (7.0, 7.0, 7.0)),      # no PML: zero walls
    (1, 1, 1, 4, (10.0, 10.0, 10.0)),      # degenerate inner region
]


def _grid_pair(nx, ny, nz, nb, h, vmax=3000.0, r0=1e-3, cfl=0.4):
    dt = float(np.float32(cfl * oracle.cfl_dt(vmax, *h)))
    g = seisgb.make_grid(nx, ny, nz, nb, *h, dt, vmax, r0)
    go = oracle.Grid(nx, ny, nz, nb, float(np.float32(h[0])), float(np.float32(h[1])),
                     float(np.float32(h[2])), dt, vmax=float(np.float32(vmax)),
                     r0=float(np.float32(r0)))
    return g, go


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


@pytest.mark.parametrize("case", STEP_CASES)
def test_single_step_random_fields(case):
    nx, ny, nz, nb, h = case
    g, go = _grid_pair(nx, ny, nz, nb, h)
    rng = np.random.default_rng(nx * 1000 + ny * 10 + nz)
    sh = g.shape
    uc = rng.standard_normal(sh).astype(np.float32)
    up = rng.standard_normal(sh).astype(np.float32)
    ph = (0.1 * rng.standard_normal(sh)).astype(np.float32)
    vel = rng.uniform(1500, 3000, sh).astype(np.float32)
    m = (vel.astype(np.float64) ** 2 * go.dt ** 2).astype(np.float32)
    # oracle: inner points never carry phi; keep phi random only in the PML
    Nz, Ny, Nx = sh
    K, J, I = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    inner = ((I >= nb) & (I < nb + nx) & (J >= nb) & (J < nb + ny) & (K >= nb) & (K < nb + nz))
    ph[inner] = 0.0
    src = (nb + nx // 2, nb + ny // 2, nb + nz // 2)
    wav = np.linspace(-1, 1, 8).astype(np.float32)
    step = 5

    d_uc, d_up, d_m, d_ph = (to_padded(g, a) for a in (uc, up, m, ph))
    d_w = torch.from_numpy(wav).cuda()
    seisgb.stencil_step(g, d_uc, d_up, d_m, d_ph, step, source=(*src, d_w))
    un = from_padded(g, d_up)
    pn = from_padded(g, d_ph)
    seisgb.device_status()

    ref_u, ref_p = oracle.step(go, m, up, uc, ph)
    inv_vol = 1.0 / (go.dx * go.dy * go.dz)
    ref_u[src[2], src[1], src[0]] += float(m[src[2], src[1], src[0]]) * float(wav[step]) * inv_vol
    S = abs_term_sum(go, m, up, uc, ph)
    S[src[2], src[1], src[0]] += abs(float(m[src[2], src[1], src[0]]) * float(wav[step]) * inv_vol)
    err = np.abs(un - ref_u)
    assert np.all(err <= 1e-6 * S + 1e-30), (float((err / S).max()), np.unravel_index(np.argmax(err / S), sh))
    errp = np.abs(pn - ref_p)
    Sp = np.abs(ph) + np.abs(ref_p) + 1e-6 * S
    assert np.all(errp <= 1e-6 * Sp + 1e-30), float((errp / Sp).max())
    # the halo stays zero
    L = seisgb.layout(g)
    full = d_up.cpu().numpy()
    mask = np.ones(int(L.elems), bool)
    k, j, i = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    mask[(L.origin + k * L.stride_z + j * L.sx + i).ravel()] = False
    assert np.all(full[mask] == 0.0)


def _small_case():
    w = synth.SMALL
    vmax = w.v_const
    dt = float(np.float32(w.cfl_fraction * oracle.cfl_dt(vmax, w.h, w.h, w.h)))
    g = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax)
    go = oracle.Grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax=vmax, r0=float(np.float32(1e-3)))
    return w, g, go, dt


def test_small_case_100_steps_rel_l2():
    """Plain FP32 forward modelling, 64^3 + PML 16, 100 steps: full wavefield and
    traces within 2e-5 relative L2 of the fp64 oracle.  Two receiver sets: the
    workload's own, on the inner top face (32 points above the source, which the
    direct wave reaches only after ~0.16 s, so they record the early part), and
    every 4th point of the horizontal plane through the source, which records the
    direct wave within the run."""
    w, g, go, dt = _small_case()
    vel = w.velocity()
    wav = synth.ricker(w.nt, dt, w.fp)
    src = w.source()
    plane = synth.surface_receivers(w.nx, w.ny, w.nb, 4)
    plane[:, 2] = src[2]
    for name, rec in (("top face", w.receivers()), ("source plane", plane)):
        ref = oracle.run_shot(go, vel, wav, w.nt, src, rec)
        tr = torch.zeros((w.nt, rec.shape[0]), dtype=torch.float32, device="cuda")
        u = torch.zeros(g.shape, dtype=torch.float32, device="cuda")
        seisgb.run_shot(g, torch.from_numpy(vel).cuda(), torch.from_numpy(wav).cuda(), w.nt, src,
                        rec, tr, u)
        e_u = rel_l2(u.cpu().numpy(), ref["u"])
        e_t = rel_l2(tr.cpu().numpy(), ref["traces"])
        print(f"small case rel L2 ({name}): wavefield {e_u:.3e} traces {e_t:.3e}")
        assert e_u <= 2e-5 and e_t <= 2e-5
    # the source-plane traces carry the direct wave: their peak is comparable
    # to the wavefield's (not a near-zero precursor)
    assert np.abs(ref["traces"]).max() > 0.1 * np.abs(ref["u"]).max()


def test_run_shot_graph_equals_step_loop():
    """run_shot (CUDA-graph replays + direct tail) gives bit-identical traces and
    wavefield to a loop of stencil_step calls plus receiver gathers."""
    nx, nb, nt = 20, 6, 70
    h = (10.0, 10.0, 10.0)
    g, go = _grid_pair(nx, nx + 3, nx - 2, nb, h, vmax=2500.0)
    rng = np.random.default_rng(1)
    vel = rng.uniform(1500, 2500, g.shape).astype(np.float32)
    wav = synth.ricker(nt, g.dt, 20.0)
    src = (nb + 5, nb + 7, nb + 3)
    rec = np.array([[nb, nb, nb], [nb + 3, nb + 9, nb + 2], [nb + nx - 1, nb + 1, nb + 4]], np.int32)
    tr = torch.zeros((nt, 3), dtype=torch.float32, device="cuda")
    u = torch.zeros(g.shape, dtype=torch.float32, device="cuda")
    d_v = torch.from_numpy(vel).cuda()
    d_w = torch.from_numpy(wav).cuda()
    seisgb.run_shot(g, d_v, d_w, nt, src, rec, tr, u)

    m = (vel.astype(np.float32) * np.float32(g.dt)) ** 2
    d_m = to_padded(g, m)
    a, b, ph = padded_zeros(g), padded_zeros(g), padded_zeros(g)
    tr2 = torch.zeros((nt, 3), dtype=torch.float32, device="cuda")
    cur, prev = a, b
    for n in range(nt):
        seisgb.stencil_step(g, cur, prev, d_m, ph, n, source=(*src, d_w), receivers=(rec, tr2[n]))
        cur, prev = prev, cur
    u2 = from_padded(g, cur)
    assert np.array_equal(tr.cpu().numpy(), tr2.cpu().numpy())
    assert np.array_equal(u.cpu().numpy(), u2)


def test_run_shot_host_buffers_match_device_buffers():
    nx, nb, nt = 24, 4, 40
    g, go = _grid_pair(nx, nx, nx, nb, (10.0, 10.0, 10.0), vmax=2000.0)
    vel = np.full(g.shape, 2000.0, np.float32)
    wav = synth.ricker(nt, g.dt, 25.0)
    src = (nb + 12, nb + 12, nb + 12)
    rec = synth.surface_receivers(nx, nx, nb, 3)
    tr_h = np.zeros((nt, rec.shape[0]), np.float32)
    u_h = np.zeros(g.shape, np.float32)
    seisgb.run_shot(g, vel, wav, nt, src, rec, tr_h, u_h)
    tr_d = torch.zeros((nt, rec.shape[0]), dtype=torch.float32, device="cuda")
    u_d = torch.zeros(g.shape, dtype=torch.float32, device="cuda")
    seisgb.run_shot(g, torch.from_numpy(vel).cuda(), torch.from_numpy(wav).cuda(), nt, src, rec,
                    tr_d, u_d)
    assert np.array_equal(tr_h, tr_d.cpu().numpy()) and np.array_equal(u_h, u_d.cpu().numpy())


def test_run_shot_nt_zero_and_no_receivers():
    g, go = _grid_pair(10, 10, 10, 2, (10.0, 10.0, 10.0))
    vel = np.full(g.shape, 2500.0, np.float32)
    u = np.ones(g.shape, np.float32)
    seisgb.run_shot(g, vel, None, 0, None, np.zeros((0, 3), np.int32), None, u)
    assert np.all(u == 0.0)


def test_run_shot_rejects_dt_above_model_cfl():
    """CFL is checked against the model's actual maximum velocity."""
    g, go = _grid_pair(10, 10, 10, 2, (10.0, 10.0, 10.0), vmax=2000.0, cfl=0.9)
    vel = np.full(g.shape, 2000.0, np.float32)
    vel[5, 5, 5] = 4000.0
    with pytest.raises(seisgb.SeisgbError) as e:
        seisgb.run_shot(g, vel, np.zeros(5, np.float32), 5, (6, 6, 6), np.zeros((0, 3)), None)
    assert e.value.code == seisgb.ERR_UNSTABLE_DT
    vel[5, 5, 5] = float("nan")
    with pytest.raises(seisgb.SeisgbError) as e:
        seisgb.run_shot(g, vel, np.zeros(5, np.float32), 5, (6, 6, 6), np.zeros((0, 3)), None)
    assert e.value.code == seisgb.ERR_INVALID_ARG


def test_run_shot_reports_nonfinite_receivers():
    """A wavelet near the fp32 maximum drives the field to Inf within a few steps;
    the receiver at the source flags it and run_shot returns NONFINITE (float
    overflow only, no device fault involved)."""
    g, go = _grid_pair(12, 12, 12, 3, (1.0, 1.0, 1.0))
    vel = np.full(g.shape, 2500.0, np.float32)
    wav = np.full(40, 3e38, np.float32)
    rec = np.array([[9, 9, 9]], np.int32)
    tr = np.zeros((40, 1), np.float32)
    with pytest.raises(seisgb.SeisgbError) as e:
        seisgb.run_shot(g, vel, wav, 40, (9, 9, 9), rec, tr)
    assert e.value.code == seisgb.ERR_NONFINITE
    assert not np.isfinite(tr).all()
    seisgb.device_status()  # the flag was cleared by run_shot


@pytest.mark.slow
def test_full_size_step_on_sampled_points():
    """512^3 computed domain with the 32-point PML and the layered model, in the
    launch configuration the benchmark times: one step from random fields,
    checked at 40,000 sampled points (plus PML faces, tile seams, corners and the
    source) against the oracle evaluated point by point."""
    w = synth.LARGE
    vel = w.velocity()
    vmax = float(vel.max())
    dt = float(np.float32(w.cfl_fraction * oracle.cfl_dt(vmax, w.h, w.h, w.h)))
    g = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax)
    go = oracle.Grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax=vmax, r0=float(np.float32(1e-3)))
    rng = np.random.default_rng(77)
    sh = g.shape
    uc = rng.standard_normal(sh, dtype=np.float32)
    up = rng.standard_normal(sh, dtype=np.float32)
    ph = (0.1 * rng.standard_normal(sh, dtype=np.float32))
    nb = w.nb
    ph[nb:nb + w.nz, nb:nb + w.ny, nb:nb + w.nx] = 0.0
    m = (vel * np.float32(dt)) ** 2
    d_uc, d_up, d_m, d_ph = (to_padded(g, a) for a in (uc, up, m, ph))
    src = w.source()
    wav = np.linspace(-1, 1, 16).astype(np.float32)
    d_w = torch.from_numpy(wav).cuda()
    seisgb.stencil_step(g, d_uc, d_up, d_m, d_ph, 7, source=(*src, d_w))
    un = from_padded(g, d_up)
    pn = from_padded(g, d_ph)
    seisgb.device_status()
    N = sh[0]
    pts = [rng.integers(0, N, size=3) for _ in range(40000)]
    special = [0, 1, nb - 1, nb, nb + 1, 63, 64, 65, N // 2, N - nb - 1, N - nb, N - 2, N - 1]
    for a in special:
        for b in special[::3]:
            for c in special[::4]:
                pts.append(np.array([a, b, c]))
    pts.append(np.array(src))
    pts = np.array(pts, dtype=np.int32)
    ou, op = oracle.step_points(go, m, up, uc, ph, pts)
    si = np.where((pts == np.array(src)).all(1))[0]
    ou[si] += float(m[src[2], src[1], src[0]]) * float(wav[7]) / (go.dx * go.dy * go.dz)
    gu = un[pts[:, 2], pts[:, 1], pts[:, 0]]
    gp = pn[pts[:, 2], pts[:, 1], pts[:, 0]]
    S = abs_term_sum_points(go, m, up, uc, ph, pts)
    S[si] += abs(float(m[src[2], src[1], src[0]]) * float(wav[7]) / (go.dx * go.dy * go.dz))
    err = np.abs(gu - ou)
    assert np.all(err <= 1e-6 * S + 1e-30), float(np.max(err / S))
    errp = np.abs(gp - op)
    Sp = np.abs(ph[pts[:, 2], pts[:, 1], pts[:, 0]]) + np.abs(op) + 1e-6 * S
    assert np.all(errp <= 1e-6 * Sp + 1e-30), float(np.max(errp / Sp))
