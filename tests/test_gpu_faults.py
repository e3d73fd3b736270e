"""Host-side fault injection, cancellation and resume (no GPU fault involved).

- An allocation that fails (the library's test hook makes chosen pool
  allocations report out of memory, as an exhausted device would) makes
  run_shot return SGB_ERR_OUT_OF_MEMORY with nothing left allocated, and the
  next call gives the same bits as before; a served shot whose set-up fails
  ends with that status while the shots around it run on unchanged.
- serve_cancel ends a queued request at once and retires a resident one at the
  next replay boundary; the other requests' traces are unchanged.
- A shot run as segments with its state (u^n, u^{n-1}, phi^n) passed along gives
  the same bits as one run_shot call."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2009_04619_gb300 import seisgb, synth
from gpu_util import ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()
    yield
    seisgb.debug_fail_allocations(0, 0)


def _request(nx, ny, nz, nb, nt, seed, storage=seisgb.FP32, schedule=seisgb.SCHED_AUTO):
    shape = (nz + 2 * nb, ny + 2 * nb, nx + 2 * nb)
    vel = synth.layered_model(shape, seed=seed, perturb=0.05, sigma=2.0)
    vmax = float(vel.max())
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, 10.0, 10.0, 10.0)))
    g = seisgb.make_grid(nx, ny, nz, nb, 10.0, 10.0, 10.0, dt, vmax, storage=storage,
                         schedule=schedule)
    wav = synth.ricker(nt, dt, 25.0)
    rng = np.random.default_rng(seed)
    src = (nb + int(rng.integers(nx)), nb + int(rng.integers(ny)), nb + 2)
    rec = synth.surface_receivers(nx, ny, nb, 3)
    return g, vel, wav, nt, src, rec


def _alone(g, vel, wav, nt, src, rec, final=False):
    tr = np.zeros((nt, rec.shape[0]), np.float32)
    u = np.zeros(g.shape, np.float32) if final else None
    seisgb.run_shot(g, vel, wav, nt, src, rec, tr, u)
    return (tr, u) if final else tr


def _pool_settled():
    torch.cuda.synchronize()
    return seisgb.pool_used_bytes()


def test_run_shot_allocation_failure_leaves_nothing():
    r = _request(30, 26, 22, 6, 45, 1)
    want_tr, want_u = _alone(*r, final=True)
    base = _pool_settled()
    failures = 0
    for k in range(0, 12):  # fail the k-th allocation of the call
        seisgb.debug_fail_allocations(k, 1)
        try:
            tr, u = _alone(*r, final=True)
            ok = True
        except seisgb.SeisgbError as e:
            assert e.code == seisgb.ERR_OUT_OF_MEMORY and "injected" in str(e)
            ok = False
            failures += 1
        seisgb.debug_fail_allocations(0, 0)
        assert _pool_settled() == base, k  # nothing left allocated
        if ok:  # the hook's number lay beyond the call's allocations
            assert np.array_equal(tr, want_tr) and np.array_equal(u, want_u)
    assert failures >= 5  # every scratch allocation of run_shot was hit once
    tr, u = _alone(*r, final=True)
    assert np.array_equal(tr, want_tr) and np.array_equal(u, want_u)


def test_served_shot_setup_failure_is_isolated():
    reqs = [_request(24, 24, 24, 6, 60, s) for s in (2, 3, 4)]
    want = [_alone(*r) for r in reqs]
    base = _pool_settled()
    with seisgb.Server(8 << 30, max_slots=4, steps_per_graph=8) as sv:
        # one shot's set-up takes 10 pool allocations: the 11th (the second
        # request's first) fails
        seisgb.debug_fail_allocations(10, 1)
        tickets = [sv.submit(*r) for r in reqs]
        got = [sv.poll(t, r[3], r[5].shape[0], timeout_us=60_000_000) for t, r in zip(tickets, reqs)]
        seisgb.debug_fail_allocations(0, 0)
        assert got[1][0] == seisgb.OK and got[1][1].status == seisgb.ERR_OUT_OF_MEMORY
        for i in (0, 2):
            assert got[i][1].status == seisgb.OK
            assert np.array_equal(got[i][2], want[i])
        assert sv.stats().device_bytes == 0
    assert _pool_settled() == base


def test_serve_cancel_queued_and_resident():
    reqs = [_request(24, 24, 24, 6, nt, s) for s, nt in ((5, 400), (6, 400), (7, 60), (8, 60), (9, 60))]
    want = [_alone(*r) for r in reqs]
    base = _pool_settled()
    with seisgb.Server(8 << 30, max_slots=2, steps_per_graph=4) as sv:
        tickets = [sv.submit(*r) for r in reqs]
        sv.cancel(tickets[3])  # queued behind two long shots: ends at once
        rc, res, tr = sv.poll(tickets[3], reqs[3][3], reqs[3][5].shape[0], timeout_us=0)
        assert rc == seisgb.OK and res.status == seisgb.ERR_CANCELLED
        # wait until the first long shot is resident, then cancel it
        for _ in range(2000):
            if sv.stats().resident > 0:
                break
            time.sleep(0.001)
        sv.cancel(tickets[0])
        out = {}
        for i, (t, r) in enumerate(zip(tickets, reqs)):
            if i == 3:
                continue
            out[i] = sv.poll(t, r[3], r[5].shape[0], timeout_us=60_000_000)
        assert out[0][1].status in (seisgb.ERR_CANCELLED, seisgb.OK)
        for i in (1, 2, 4):
            assert out[i][1].status == seisgb.OK
            assert np.array_equal(out[i][2], want[i]), i
        st = sv.stats()
        assert st.cancelled == 1 + int(out[0][1].status == seisgb.ERR_CANCELLED)
        assert st.resident == 0 and st.queued == 0 and st.device_bytes == 0
        with pytest.raises(seisgb.SeisgbError):
            sv.cancel(12345)
    assert _pool_settled() == base


@pytest.mark.parametrize("storage,schedule,cut", [
    (seisgb.FP32, seisgb.SCHED_STEP, 37),
    (seisgb.FP32, seisgb.SCHED_STEP, 64),
    (seisgb.FP32, seisgb.SCHED_FLOW, 41),
    (seisgb.BF16, seisgb.SCHED_STEP, 33),
    (seisgb.BF16, seisgb.SCHED_FLOW, 50),
])
def test_segments_resume_bit_identical(storage, schedule, cut):
    """[0, cut) then [cut, nt) with the state carried in host arrays equals one
    run_shot over [0, nt): traces, final wavefield and phi."""
    g, vel, wav, nt, src, rec = _request(37, 29, 23, 5, 90, 10, storage=storage, schedule=schedule)
    want_tr, want_u = _alone(g, vel, wav, nt, src, rec, final=True)
    state = [np.zeros(g.shape, np.float32) for _ in range(3)]
    tr = np.zeros((nt, rec.shape[0]), np.float32)
    seisgb.run_shot_segment(g, vel, wav, 0, cut, src, rec, tr[:cut], *state)
    saved = [s.copy() for s in state]  # a checkpoint: resume from a copy
    seisgb.run_shot_segment(g, vel, wav, cut, nt, src, rec, tr[cut:], *saved)
    assert np.array_equal(tr, want_tr)
    assert np.array_equal(saved[0], want_u)
    # zero-length segment: the state passes through unchanged
    again = [s.copy() for s in saved]
    seisgb.run_shot_segment(g, vel, wav, nt, nt, src, rec, np.zeros((0, rec.shape[0]), np.float32),
                            *again)
    assert all(np.array_equal(a, b) for a, b in zip(again, saved))


def test_segments_device_state_and_three_pieces():
    g, vel, wav, nt, src, rec = _request(40, 36, 30, 6, 100, 11)
    want_tr, want_u = _alone(g, vel, wav, nt, src, rec, final=True)
    d = [torch.zeros(g.shape, dtype=torch.float32, device="cuda") for _ in range(3)]
    tr = torch.zeros((nt, rec.shape[0]), dtype=torch.float32, device="cuda")
    d_v, d_w = torch.from_numpy(vel).cuda(), torch.from_numpy(wav).cuda()
    for a, b in ((0, 13), (13, 71), (71, nt)):
        seisgb.run_shot_segment(g, d_v, d_w, a, b, src, rec, tr[a:b], *d)
    assert np.array_equal(tr.cpu().numpy(), want_tr)
    assert np.array_equal(d[0].cpu().numpy(), want_u)
