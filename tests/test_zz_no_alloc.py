"""The allocation-free shot entry point (for callers that cannot allocate device
memory while running, e.g. a process whose memory belongs to another allocator,
or a real-time loop that forbids cudaMalloc/cudaFree after start-up) gives the
same results as run_shot, call after call, without allocating.

run_shot_noalloc launches the same fp32 step kernel with the same decomposition
as run_shot (direct launches instead of CUDA graphs), so traces and the final
wavefield must agree bit for bit; both are also checked against the fp64 oracle.

Collected last on purpose: it shares one fixed device array across calls."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_04619_gb300 import seisgb, synth
from gpu_util import ensure_lib, rel_l2

pytestmark = pytest.mark.gpu


def _case(nx, ny, nz, nb, v, fp, nt, src, rec_every, seed=None):
    shape = (nz + 2 * nb, ny + 2 * nb, nx + 2 * nb)
    vel = (synth.constant_model(shape, v) if seed is None
           else synth.layered_model(shape, seed=seed, vmin=1800.0, vmax=3200.0, sigma=2.0))
    vmax = float(vel.max())
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, 10.0, 10.0, 10.0)))
    g = seisgb.make_grid(nx, ny, nz, nb, 10.0, 10.0, 10.0, dt, vmax)
    go = oracle.Grid(nx, ny, nz, nb, 10.0, 10.0, 10.0, dt, vmax=vmax, r0=float(np.float32(1e-3)))
    rec = synth.surface_receivers(nx, ny, nb, rec_every)
    rec[::2, 2] = src[2]  # half the receivers on the source plane: they record signal early
    return g, go, vel, synth.ricker(nt, dt, fp), nt, src, rec


# The small forward-modelling case twice (two sources, two wavelets), then a
# smaller ragged layered grid: the third call shows that the zeroing at the
# start of a call covers a change of grid layout.
CASES = [
    lambda: _case(64, 64, 64, 16, 2000.0, 15.0, 100, (48, 48, 48), 8),
    lambda: _case(64, 64, 64, 16, 2000.0, 20.0, 100, (40, 55, 51), 8),
    lambda: _case(37, 29, 23, 5, 0.0, 25.0, 80, (20, 17, 9), 3, seed=11),
]


def test_noalloc_matches_run_shot_and_oracle_on_consecutive_calls():
    ensure_lib()
    # set-up call: the first call on a device resolves the fixed array's device
    # address (nothing is checked here; every later call must not allocate)
    g, go, vel, wav, nt, src, rec = CASES[0]()
    d_v = torch.from_numpy(vel).cuda()
    d_w = torch.from_numpy(wav).cuda()
    tr0 = torch.zeros((nt, rec.shape[0]), dtype=torch.float32, device="cuda")
    seisgb.run_shot_noalloc(g, d_v, d_w, nt, src, rec, tr0)
    torch.cuda.synchronize()

    for call, make in enumerate(CASES):
        g, go, vel, wav, nt, src, rec = make()
        nrec = rec.shape[0]
        d_v = torch.from_numpy(vel).cuda()
        d_w = torch.from_numpy(wav).cuda()
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
        assert free1 == free0, (call, free0, free1)  # nothing allocated on the device
        tr_a, u_a, tr_b, u_b = (x.cpu().numpy() for x in (tr_a, u_a, tr_b, u_b))
        assert np.array_equal(tr_b, tr_a) and np.array_equal(u_b, u_a), call
        ref = oracle.run_shot(go, vel, wav, nt, src, rec)
        assert np.abs(ref["traces"]).max() > 0 and np.abs(ref["u"]).max() > 0
        e_u, e_t = rel_l2(u_b, ref["u"]), rel_l2(tr_b, ref["traces"])
        assert e_u <= 2e-5 and e_t <= 2e-5, (call, e_u, e_t)


def test_noalloc_rejects_grids_above_its_scratch():
    ensure_lib()
    g = seisgb.make_grid(192, 192, 192, 32, 10, 10, 10, 5e-4, 3000)
    d_v = torch.full(g.shape, 2000.0, device="cuda")
    d_w = torch.zeros(4, device="cuda")
    tr = torch.zeros((4, 1), device="cuda")
    with pytest.raises(seisgb.SeisgbError) as e:
        seisgb.run_shot_noalloc(g, d_v, d_w, 4, (100, 100, 100), np.array([[100, 100, 40]]), tr)
    assert e.value.code == seisgb.ERR_INVALID_ARG and "scratch" in str(e.value)


def test_noalloc_rejects_outputs_overlapping_inputs():
    ensure_lib()
    g, go, vel, wav, nt, src, rec = CASES[2]()
    N = int(np.prod(g.shape))
    buf = torch.zeros(2 * N, dtype=torch.float32, device="cuda")
    buf[:N] = torch.from_numpy(vel.ravel()).cuda()
    d_w = torch.from_numpy(wav).cuda()
    tr = torch.zeros((nt, rec.shape[0]), dtype=torch.float32, device="cuda")
    with pytest.raises(seisgb.SeisgbError) as e:  # final_u starts inside velocity
        seisgb.run_shot_noalloc(g, buf[:N], d_w, nt, src, rec, tr, buf[N // 2:N // 2 + N])
    assert e.value.code == seisgb.ERR_INVALID_ARG and "overlaps" in str(e.value)
