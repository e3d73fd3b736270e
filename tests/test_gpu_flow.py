"""The persistent dataflow schedule of run_shot (SCHED_FLOW: one launch for the
whole time loop, CTAs taking (step, tile) items as soon as the neighbouring
tiles have finished the previous step) against one launch per step
(SCHED_STEP) and the fp64 oracle.

The per-point arithmetic is the same plane body in both schedules and the
decomposition does not enter it, so traces and wavefields must be identical bit
for bit; grids range from fewer work units than resident CTAs (many steps in
flight at once) to the 512^3 benchmark grid."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_04619_gb300 import seisgb, synth
from gpu_util import ensure_lib, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _case(nx, ny, nz, nb, nt, seed, h=(10.0, 10.0, 10.0), storage=seisgb.FP32, rec_every=3):
    shape = (nz + 2 * nb, ny + 2 * nb, nx + 2 * nb)
    vel = synth.layered_model(shape, seed=seed, sigma=2.0)
    vmax = float(vel.max())
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, *h)))
    wav = synth.ricker(nt, dt, 25.0)
    rng = np.random.default_rng(seed)
    src = (nb + int(rng.integers(nx)), nb + int(rng.integers(ny)), nb + int(rng.integers(nz)))
    rec = synth.surface_receivers(nx, ny, nb, rec_every)
    # receivers spread over the depth too, so that many work units sample
    rec[:, 2] = nb + rng.integers(0, nz, rec.shape[0])
    return dict(nx=nx, ny=ny, nz=nz, nb=nb, h=h, dt=dt, vmax=vmax, vel=vel, wav=wav, nt=nt,
                src=src, rec=rec.astype(np.int32), storage=storage)


def _run(c, schedule):
    g = seisgb.make_grid(c["nx"], c["ny"], c["nz"], c["nb"], *c["h"], c["dt"], c["vmax"],
                         storage=c["storage"], schedule=schedule)
    tr = torch.zeros((c["nt"], c["rec"].shape[0]), dtype=torch.float32, device="cuda")
    u = torch.zeros(g.shape, dtype=torch.float32, device="cuda")
    seisgb.run_shot(g, torch.from_numpy(c["vel"]).cuda(), torch.from_numpy(c["wav"]).cuda(),
                    c["nt"], c["src"], c["rec"], tr, u)
    return tr.cpu().numpy(), u.cpu().numpy()


CASES = [
    (24, 24, 24, 6, 90, 1),       # fewer units than resident CTAs: many steps in flight
    (90, 37, 29, 5, 61, 2),       # ragged in every axis
    (130, 52, 41, 8, 47, 3),      # several tiles in x
    (40, 33, 70, 0, 33, 4),       # no PML
    (3, 2, 5, 2, 25, 5),          # tiny inner region
    (200, 150, 120, 16, 40, 6),   # mid size, odd step count
]


@pytest.mark.parametrize("case", CASES)
def test_flow_equals_one_launch_per_step(case):
    c = _case(*case)
    a = _run(c, seisgb.SCHED_STEP)
    b = _run(c, seisgb.SCHED_FLOW)
    assert np.abs(a[0]).max() > 0
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_flow_bf16_equals_one_launch_per_step():
    """bf16 storage (stochastic rounding from a hash of point and step): the
    dataflow schedule draws the same random bits, so the same values."""
    c = _case(90, 37, 29, 5, 61, 2, storage=seisgb.BF16)
    a = _run(c, seisgb.SCHED_STEP)
    b = _run(c, seisgb.SCHED_FLOW)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_flow_nt_one_and_zero():
    c = _case(20, 18, 16, 4, 1, 7)
    assert all(np.array_equal(x, y) for x, y in zip(_run(c, seisgb.SCHED_STEP), _run(c, seisgb.SCHED_FLOW)))
    c = _case(20, 18, 16, 4, 0, 7)
    g = seisgb.make_grid(20, 18, 16, 4, 10, 10, 10, c["dt"], c["vmax"], schedule=seisgb.SCHED_FLOW)
    u = np.ones(g.shape, np.float32)
    seisgb.run_shot(g, c["vel"], None, 0, None, np.zeros((0, 3), np.int32), None, u)
    assert np.all(u == 0.0)


def test_flow_small_case_against_oracle():
    """The small forward-modelling case (64^3 + PML 16, 100 steps) with the
    dataflow schedule: within 2e-5 relative L2 of the fp64 oracle."""
    w = synth.SMALL
    dt = float(np.float32(w.cfl_fraction * oracle.cfl_dt(w.v_const, w.h, w.h, w.h)))
    g = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, w.v_const,
                         schedule=seisgb.SCHED_FLOW)
    vel = w.velocity()
    wav = synth.ricker(w.nt, dt, w.fp)
    rec = synth.surface_receivers(w.nx, w.ny, w.nb, 4)
    rec[::2, 2] = w.source()[2]
    tr = torch.zeros((w.nt, rec.shape[0]), dtype=torch.float32, device="cuda")
    u = torch.zeros(g.shape, dtype=torch.float32, device="cuda")
    seisgb.run_shot(g, torch.from_numpy(vel).cuda(), torch.from_numpy(wav).cuda(), w.nt,
                    w.source(), rec, tr, u)
    go = oracle.Grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax=w.v_const,
                     r0=float(np.float32(1e-3)))
    ref = oracle.run_shot(go, vel, wav, w.nt, w.source(), rec)
    assert rel_l2(u.cpu().numpy(), ref["u"]) <= 2e-5
    assert rel_l2(tr.cpu().numpy(), ref["traces"]) <= 2e-5


def test_flow_reports_nonfinite():
    """A receiver that samples Inf inside the dataflow launch sets NONFINITE."""
    dt = float(np.float32(0.4 * oracle.cfl_dt(2500.0, 1.0, 1.0, 1.0)))
    g = seisgb.make_grid(12, 12, 12, 3, 1.0, 1.0, 1.0, dt, 2500.0, schedule=seisgb.SCHED_FLOW)
    vel = np.full(g.shape, 2500.0, np.float32)
    tr = np.zeros((40, 1), np.float32)
    with pytest.raises(seisgb.SeisgbError) as e:
        seisgb.run_shot(g, vel, np.full(40, 3e38, np.float32), 40, (9, 9, 9),
                        np.array([[9, 9, 9]], np.int32), tr)
    assert e.value.code == seisgb.ERR_NONFINITE
    assert not np.isfinite(tr).all()


@pytest.mark.slow
def test_flow_full_size():
    """The 512^3 benchmark grid (448^3 inner + 32-point PML, layered model,
    12,544 surface receivers), 40 steps: dataflow and one-launch-per-step
    schedules give the same traces and wavefield (compared on the device)."""
    w = synth.LARGE
    vel = w.velocity()
    vmax = float(vel.max())
    dt = float(np.float32(w.cfl_fraction * oracle.cfl_dt(vmax, w.h, w.h, w.h)))
    nt = 40
    d_v = torch.from_numpy(vel).cuda()
    d_w = torch.from_numpy(synth.ricker(nt, dt, w.fp)).cuda()
    rec = w.receivers()
    out = {}
    for sched in (seisgb.SCHED_STEP, seisgb.SCHED_FLOW):
        g = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax, schedule=sched)
        tr = torch.zeros((nt, rec.shape[0]), dtype=torch.float32, device="cuda")
        u = torch.zeros(g.shape, dtype=torch.float32, device="cuda")
        seisgb.run_shot(g, d_v, d_w, nt, w.source(), rec, tr, u)
        out[sched] = (tr, u)
    a, b = out[seisgb.SCHED_STEP], out[seisgb.SCHED_FLOW]
    assert float(a[0].abs().max()) > 0
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
