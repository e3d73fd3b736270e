"""Continuous-batching shot server: each result equals run_shot's for the same
request whether it ran alone or in a mix of different grid sizes; admission
respects the HBM budget; over-budget requests are rejected; polls time out."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2009_04619_gb300 import seisgb, synth
from gpu_util import ensure_lib

pytestmark = pytest.mark.gpu

# (inner nx, ny, nz, nb, nt, seed)
MIX = [(24, 24, 24, 6, 90, 1), (40, 28, 20, 8, 150, 2), (18, 36, 30, 4, 60, 3),
       (32, 32, 32, 6, 120, 4), (20, 20, 44, 5, 70, 5), (48, 40, 24, 8, 100, 6)]


def _request(case):
    nx, ny, nz, nb, nt, seed = case
    shape = (nz + 2 * nb, ny + 2 * nb, nx + 2 * nb)
    vel = synth.layered_model(shape, seed=seed, perturb=0.05, sigma=2.0)
    vmax = float(vel.max())
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, 10.0, 10.0, 10.0)))
    g = seisgb.make_grid(nx, ny, nz, nb, 10.0, 10.0, 10.0, dt, vmax)
    wav = synth.ricker(nt, dt, 25.0)
    rng = np.random.default_rng(seed)
    src = (nb + int(rng.integers(nx)), nb + int(rng.integers(ny)), nb + 2)
    rec = synth.surface_receivers(nx, ny, nb, 3)
    return g, vel, wav, nt, src, rec


def _alone(g, vel, wav, nt, src, rec):
    tr = np.zeros((nt, rec.shape[0]), np.float32)
    seisgb.run_shot(g, vel, wav, nt, src, rec, tr)
    return tr


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def test_results_equal_run_shot_alone_and_in_mix():
    reqs = [_request(c) for c in MIX]
    ref = [_alone(*r) for r in reqs]
    for slots in (1, 16):  # one at a time, then all in the mix
        with seisgb.Server(8 << 30, max_slots=slots, steps_per_graph=16) as sv:
            tickets = []
            for i, r in enumerate(reqs):
                tickets.append(sv.submit(*r))
                if i == 2:
                    time.sleep(0.05)  # later requests arrive while earlier ones run
            for t, r, want in zip(tickets, reqs, ref):
                rc, res, tr = sv.poll(t, r[3], r[5].shape[0], timeout_us=60_000_000)
                assert rc == seisgb.OK and res.status == seisgb.OK
                assert np.array_equal(tr, want), (slots, t)
                assert res.latency_ms >= res.queue_ms >= 0
            st = sv.stats()
            assert st.completed == len(reqs) and st.resident == 0 and st.queued == 0


def test_admission_by_budget_and_rejection():
    reqs = [_request(c) for c in MIX[:4]]
    fps = [seisgb.serve_footprint(r[0], r[3], r[5].shape[0]) for r in reqs]
    budget = max(fps) + min(fps) // 2  # never room for two of the larger shots
    with seisgb.Server(budget, max_slots=8, steps_per_graph=8) as sv:
        big = _request((96, 96, 96, 16, 10, 9))
        with pytest.raises(seisgb.SeisgbError) as e:
            sv.submit(*big)
        assert e.value.code == seisgb.ERR_REJECTED
        tickets = [sv.submit(*r) for r in reqs]
        peak = 0
        pending = set(tickets)
        results = {}
        while pending:
            peak = max(peak, sv.stats().device_bytes)
            for t, r in zip(tickets, reqs):
                if t in pending:
                    rc, res, tr = sv.poll(t, r[3], r[5].shape[0], timeout_us=0)
                    if rc == seisgb.OK:
                        pending.discard(t)
                        results[t] = tr
            time.sleep(0.001)
        assert peak <= budget
        assert sv.stats().rejected == 1
        for t, r in zip(tickets, reqs):
            assert np.array_equal(results[t], _alone(*r))


def test_poll_timeout_then_result():
    r = _request((40, 40, 40, 8, 1500, 7))
    with seisgb.Server(8 << 30, max_slots=4, steps_per_graph=32) as sv:
        t = sv.submit(*r)
        rc, res, tr = sv.poll(t, r[3], r[5].shape[0], timeout_us=200)
        assert rc == seisgb.ERR_TIMEOUT
        rc, res, tr = sv.poll(t, r[3], r[5].shape[0], timeout_us=0)
        assert rc in (seisgb.PENDING, seisgb.OK)
        if rc == seisgb.PENDING:
            rc, res, tr = sv.poll(t, r[3], r[5].shape[0], timeout_us=120_000_000)
        assert rc == seisgb.OK and res.status == seisgb.OK
        assert np.array_equal(tr, _alone(*r))
        with pytest.raises(seisgb.SeisgbError):
            sv.poll(t, r[3], r[5].shape[0])  # consumed ticket is unknown now
