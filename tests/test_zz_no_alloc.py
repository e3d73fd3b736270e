"""The allocation-free shot entry point (for callers that cannot allocate device
memory while running, e.g. a process whose memory belongs to another allocator,
or a real-time loop that forbids cudaMalloc/cudaFree after start-up) gives the
same results as run_shot, call after call, without allocating.

Collected last on purpose: it shares one fixed device array across calls."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_04619_gb300 import seisgb, synth
from gpu_util import ensure_lib, rel_l2

pytestmark = pytest.mark.gpu


def _grid(w):
    dt = float(np.float32(w.cfl_fraction * oracle.cfl_dt(w.v_const, w.h, w.h, w.h)))
    return seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, w.v_const), dt


def _both(g, d_v, d_w, nt, src, rec):
    nrec = rec.shape[0]
    tr_a = torch.zeros((nt, nrec), dtype=torch.float32, device="cuda")
    u_a = torch.zeros(g.shape, dtype=torch.float32, device="cuda")
    seisgb.run_shot(g, d_v, d_w, nt, src, rec, tr_a, u_a)
    tr_b = torch.full((nt, nrec), 7.0, dtype=torch.float32, device="cuda")
    u_b = torch.full(g.shape, 7.0, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    seisgb.run_shot_noalloc(g, d_v, d_w, nt, src, rec, tr_b, u_b)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    return tr_a.cpu().numpy(), u_a.cpu().numpy(), tr_b.cpu().numpy(), u_b.cpu().numpy(), free0, free1


def test_noalloc_matches_run_shot_on_consecutive_calls():
    ensure_lib()
    w = synth.SMALL
    g, dt = _grid(w)
    rec = w.receivers()
    d_v = torch.from_numpy(w.velocity()).cuda()
    # first call on this device does the set-up (address of the fixed array)
    cases = [(w.source(), synth.ricker(w.nt, dt, w.fp)),
             ((40, 55, 51), synth.ricker(w.nt, dt, 20.0))]
    for call, (src, wav) in enumerate(cases):
        d_w = torch.from_numpy(wav).cuda()
        tr_a, u_a, tr_b, u_b, free0, free1 = _both(g, d_v, d_w, w.nt, src, rec)
        assert rel_l2(u_b, u_a) <= 2e-5 and rel_l2(tr_b, tr_a) <= 2e-5, call
        assert np.abs(u_a).max() > 0 and np.abs(tr_a).max() > 0
        if call > 0:
            # nothing allocated on the device by the call
            assert free1 == free0, (free0, free1)


def test_noalloc_rejects_grids_above_its_scratch():
    ensure_lib()
    g = seisgb.make_grid(192, 192, 192, 32, 10, 10, 10, 5e-4, 3000)
    d_v = torch.full(g.shape, 2000.0, device="cuda")
    d_w = torch.zeros(4, device="cuda")
    tr = torch.zeros((4, 1), device="cuda")
    with pytest.raises(seisgb.SeisgbError) as e:
        seisgb.run_shot_noalloc(g, d_v, d_w, 4, (100, 100, 100), np.array([[100, 100, 40]]), tr)
    assert e.value.code == seisgb.ERR_INVALID_ARG and "scratch" in str(e.value)
