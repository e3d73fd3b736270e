"""Temporal blocking (two time steps per HBM pass on the PML-free interior):
stencil_step2 and run_shot with SCHED_PAIRS against single steps and the fp64
oracle.

The two-step kernel evaluates the interior path's arithmetic operation for
operation, and the shell launches are the single-step kernel itself, so the
results must equal two stencil_step calls (and SCHED_STEP) bit for bit.  Each
of the two steps is also checked against oracle.step at the per-point bound of
the single-step parity tests (1e-6 S)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_04619_gb300 import seisgb, synth
from gpu_util import abs_term_sum, ensure_lib, from_padded, padded_zeros, rel_l2, to_padded

pytestmark = pytest.mark.gpu

CASES = [
    # nx, ny, nz, nb, (dx, dy, dz), source offset from the inner corner
    (90, 37, 29, 5, (10.0, 11.0, 12.0), (45, 18, 14)),   # several two-step tiles, ragged
    (130, 52, 41, 8, (10.0, 10.0, 10.0), (2, 2, 2)),     # source in the band outside the box
    (64, 64, 64, 16, (10.0, 10.0, 10.0), (32, 32, 32)),  # the small case's geometry
    (40, 33, 70, 0, (7.0, 7.0, 7.0), (20, 3, 60)),       # no PML: zero walls
    (9, 7, 6, 3, (10.0, 10.0, 10.0), (4, 3, 3)),         # box empty: shell launches only
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _grid_pair(nx, ny, nz, nb, h, vmax=3000.0, schedule=1):
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, *h)))
    g = seisgb.make_grid(nx, ny, nz, nb, *h, dt, vmax, 1e-3, schedule=schedule)
    go = oracle.Grid(nx, ny, nz, nb, float(np.float32(h[0])), float(np.float32(h[1])),
                     float(np.float32(h[2])), dt, vmax=float(np.float32(vmax)),
                     r0=float(np.float32(1e-3)))
    return g, go


def _oracle_step(go, m, up, uc, ph, src, wav, step):
    ref_u, ref_p = oracle.step(go, m, up, uc, ph)
    inv_vol = 1.0 / (go.dx * go.dy * go.dz)
    S = abs_term_sum(go, m, up, uc, ph)
    term = float(m[src[2], src[1], src[0]]) * float(wav[step]) * inv_vol
    ref_u[src[2], src[1], src[0]] += term
    S[src[2], src[1], src[0]] += abs(term)
    return ref_u, ref_p, S


@pytest.mark.parametrize("case", CASES)
def test_step2_equals_two_steps_and_oracle(case):
    nx, ny, nz, nb, h, so = case
    g, go = _grid_pair(nx, ny, nz, nb, h)
    rng = np.random.default_rng(nx * 7 + ny * 3 + nz)
    sh = g.shape
    uc = rng.standard_normal(sh).astype(np.float32)
    up = rng.standard_normal(sh).astype(np.float32)
    ph = (0.1 * rng.standard_normal(sh)).astype(np.float32)
    Nz, Ny, Nx = sh
    K, J, I = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    inner = ((I >= nb) & (I < nb + nx) & (J >= nb) & (J < nb + ny) & (K >= nb) & (K < nb + nz))
    ph[inner] = 0.0
    vel = rng.uniform(1500, 3000, sh).astype(np.float32)
    m = (vel.astype(np.float64) ** 2 * go.dt ** 2).astype(np.float32)
    src = (nb + so[0], nb + so[1], nb + so[2])
    wav = np.linspace(-1, 1, 12).astype(np.float32)
    step = 5
    d_w = torch.from_numpy(wav).cuda()
    d_m = to_padded(g, m)

    # two stencil_step calls (in place)
    a_up, a_uc, a_ph = to_padded(g, up), to_padded(g, uc), to_padded(g, ph)
    seisgb.stencil_step(g, a_uc, a_up, d_m, a_ph, step, source=(*src, d_w))      # a_up = u^{n+1}
    seisgb.stencil_step(g, a_up, a_uc, d_m, a_ph, step + 1, source=(*src, d_w))  # a_uc = u^{n+2}
    # one stencil_step2 call (four buffers)
    b_up, b_uc, b_ph = to_padded(g, up), to_padded(g, uc), to_padded(g, ph)
    b_n1, b_n2 = padded_zeros(g), padded_zeros(g)
    seisgb.stencil_step2(g, b_up, b_uc, b_n1, b_n2, d_m, b_ph, step, source=(*src, d_w))
    seisgb.device_status()
    torch.cuda.synchronize()
    assert torch.equal(a_up, b_n1) and torch.equal(a_uc, b_n2) and torch.equal(a_ph, b_ph)
    # inputs untouched, halo of the outputs still zero
    assert torch.equal(b_up, to_padded(g, up)) and torch.equal(b_uc, to_padded(g, uc))

    # each step against the oracle: step n from the inputs, step n+1 from the
    # GPU's own u^{n+1} and phi^{n+1}
    u1, p1 = from_padded(g, b_n1), from_padded(g, b_ph)
    ref1, _, S1 = _oracle_step(go, m, up, uc, ph, src, wav, step)
    err1 = np.abs(u1 - ref1)
    assert np.all(err1 <= 1e-6 * S1 + 1e-30), float((err1 / S1).max())
    # phi^{n+1} of the first step is needed for the second: recompute it with
    # the oracle (the GPU keeps only phi^{n+2})
    _, ph1 = oracle.step(go, m, up, uc, ph)
    ph1 = ph1.astype(np.float32)
    u2 = from_padded(g, b_n2)
    ref2, refp2, S2 = _oracle_step(go, m, uc, u1, ph1, src, wav, step + 1)
    # (the GPU's second step used its own fp32 phi^{n+1}, within 1e-6 of ph1:
    # hence 2e-6 S on the second step)
    err2 = np.abs(u2 - ref2)
    assert np.all(err2 <= 2e-6 * S2 + 1e-30), float((err2 / S2).max())
    errp = np.abs(p1 - refp2)
    Sp = np.abs(ph1) + np.abs(refp2) + 1e-6 * S2
    assert np.all(errp <= 2e-6 * Sp + 1e-30), float((errp / Sp).max())


def _shot(g, vel, wav, nt, src, rec):
    tr = torch.zeros((nt, rec.shape[0]), dtype=torch.float32, device="cuda")
    u = torch.zeros(g.shape, dtype=torch.float32, device="cuda")
    seisgb.run_shot(g, torch.from_numpy(vel).cuda(), torch.from_numpy(wav).cuda(), nt, src, rec,
                    tr, u)
    return tr.cpu().numpy(), u.cpu().numpy()


@pytest.mark.parametrize("nt", [100, 71])
def test_run_shot_pairs_small_case(nt):
    """The small forward-modelling case (64^3 + PML 16) with SCHED_PAIRS: the
    same bits as SCHED_STEP (graph replays of 16 pairs, direct pairs, an odd
    last step), and within 2e-5 relative L2 of the fp64 oracle."""
    w = synth.SMALL
    vmax = w.v_const
    dt = float(np.float32(w.cfl_fraction * oracle.cfl_dt(vmax, w.h, w.h, w.h)))
    vel = w.velocity()
    wav = synth.ricker(nt, dt, w.fp)
    src = w.source()
    rec = synth.surface_receivers(w.nx, w.ny, w.nb, 4)
    rec[::2, 2] = src[2]  # half on the source plane: they record the direct wave
    res = {}
    for tb in (seisgb.SCHED_STEP, seisgb.SCHED_PAIRS):
        g = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax, schedule=tb)
        res[tb] = _shot(g, vel, wav, nt, src, rec)
    assert np.array_equal(res[seisgb.SCHED_STEP][0], res[seisgb.SCHED_PAIRS][0]) and np.array_equal(res[seisgb.SCHED_STEP][1], res[seisgb.SCHED_PAIRS][1])
    go = oracle.Grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax=vmax, r0=float(np.float32(1e-3)))
    ref = oracle.run_shot(go, vel, wav, nt, src, rec)
    assert rel_l2(res[seisgb.SCHED_PAIRS][1], ref["u"]) <= 2e-5 and rel_l2(res[seisgb.SCHED_PAIRS][0], ref["traces"]) <= 2e-5


def test_run_shot_pairs_layered_ragged():
    """A ragged anisotropic layered grid, source near a corner of the inner
    region (in the band the shell launches compute): same bits as SCHED_STEP."""
    nx, ny, nz, nb, nt = 101, 45, 38, 7, 67
    shape = (nz + 2 * nb, ny + 2 * nb, nx + 2 * nb)
    vel = synth.layered_model(shape, seed=21, sigma=2.0)
    vmax = float(vel.max())
    h = (10.0, 12.0, 9.0)
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, *h)))
    wav = synth.ricker(nt, dt, 25.0)
    src = (nb + 1, nb + 2, nb + 2)
    rec = synth.surface_receivers(nx, ny, nb, 5)
    res = {}
    for tb in (seisgb.SCHED_STEP, seisgb.SCHED_PAIRS):
        g = seisgb.make_grid(nx, ny, nz, nb, *h, dt, vmax, schedule=tb)
        res[tb] = _shot(g, vel, wav, nt, src, rec)
    assert np.abs(res[seisgb.SCHED_STEP][0]).max() > 0
    assert np.array_equal(res[seisgb.SCHED_STEP][0], res[seisgb.SCHED_PAIRS][0]) and np.array_equal(res[seisgb.SCHED_STEP][1], res[seisgb.SCHED_PAIRS][1])


@pytest.mark.slow
def test_run_shot_pairs_full_size():
    """The 512^3 benchmark grid (448^3 inner + 32-point PML, layered model) in
    the launch configuration the benchmark times, 40 steps (one graph replay of
    16 pairs, then 4 direct pairs): traces and final wavefield bit-identical to
    SCHED_STEP (compared on the device)."""
    w = synth.LARGE
    vel = w.velocity()
    vmax = float(vel.max())
    dt = float(np.float32(w.cfl_fraction * oracle.cfl_dt(vmax, w.h, w.h, w.h)))
    nt = 40
    wav = synth.ricker(nt, dt, w.fp)
    rec = w.receivers()
    d_v, d_w = torch.from_numpy(vel).cuda(), torch.from_numpy(wav).cuda()
    out = {}
    for tb in (seisgb.SCHED_STEP, seisgb.SCHED_PAIRS):
        g = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax, schedule=tb)
        tr = torch.zeros((nt, rec.shape[0]), dtype=torch.float32, device="cuda")
        u = torch.zeros(g.shape, dtype=torch.float32, device="cuda")
        seisgb.run_shot(g, d_v, d_w, nt, w.source(), rec, tr, u)
        out[tb] = (tr, u)
    assert float(out[seisgb.SCHED_STEP][1].abs().max()) > 0
    assert torch.equal(out[seisgb.SCHED_STEP][0], out[seisgb.SCHED_PAIRS][0]) and torch.equal(out[seisgb.SCHED_STEP][1], out[seisgb.SCHED_PAIRS][1])
