"""GPU adjoint gradient against the fp64 oracle's (itself pinned by central
differences), checkpoint-interval invariance, and the autograd wrapper."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_04619_gb300 import seisgb, synth
from paper_2009_04619_gb300.autograd import velocity_misfit
from gpu_util import ensure_lib, rel_l2

pytestmark = pytest.mark.gpu


def _case(n_in=16, nb=8, nt=50, seed=3):
    """The 32^3 / 50-step instance: layered model with a Gaussian anomaly,
    observed data from the model without it (halved, so the residual is large)."""
    N = n_in + 2 * nb
    shape = (N, N, N)
    v0 = synth.layered_model(shape, seed=seed, vmin=1800, vmax=3000, perturb=0.0)
    v = (v0 * synth.gaussian_anomaly(shape, (N / 2, N / 2, N / 2 + 3), 3.0, 0.08)).astype(np.float32)
    vmax = float(max(v.max(), v0.max()))
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, 10, 10, 10)))
    wav = synth.ricker(nt, dt, 30.0)
    src = (nb + 1, nb + 2, nb + 2)
    rec = synth.surface_receivers(n_in, n_in, nb, 3)
    go = oracle.Grid(n_in, n_in, n_in, nb, 10.0, 10.0, 10.0, dt, vmax=vmax, r0=float(np.float32(1e-3)))
    obs = (0.5 * oracle.run_shot(go, v0, wav, nt, src, rec, want_state=False)["traces"]).astype(np.float32)
    g = seisgb.make_grid(n_in, n_in, n_in, nb, 10.0, 10.0, 10.0, dt, vmax)
    return g, go, v, wav, nt, src, rec, obs


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def test_gradient_matches_oracle_adjoint():
    """fp32 forward/adjoint with fp64 accumulation vs the fp64 oracle: misfit and
    gradient (bounds: 20x the errors measured when the adjoint was added)."""
    g, go, v, wav, nt, src, rec, obs = _case()
    J_ref, grad_ref = oracle.adjoint_shot(go, v, wav, nt, src, rec, obs.astype(np.float64))
    grad = np.zeros(v.shape)
    J = seisgb.adjoint_shot(g, v, wav, nt, src, rec, obs, grad, ckpt_every=16)
    e_J = abs(J - J_ref) / J_ref
    e_g = rel_l2(grad, grad_ref)
    print(f"adjoint vs oracle: misfit {e_J:.3e}, gradient rel L2 {e_g:.3e}")
    assert e_J <= 1e-4 and e_g <= 1e-3


def test_checkpoint_interval_does_not_change_the_gradient():
    g, go, v, wav, nt, src, rec, obs = _case()
    outs = []
    for c in (7, 16, 50, 0):
        grad = torch.zeros(v.shape, dtype=torch.float64, device="cuda")
        J = seisgb.adjoint_shot(g, torch.from_numpy(v).cuda(), torch.from_numpy(wav).cuda(), nt, src,
                                rec, torch.from_numpy(obs).cuda(), grad, ckpt_every=c)
        outs.append((J, grad.cpu().numpy()))
    for J, grad in outs[1:]:
        assert J == outs[0][0] and np.array_equal(grad, outs[0][1])


def test_autograd_function():
    g, go, v, wav, nt, src, rec, obs = _case()
    vt = torch.from_numpy(v).cuda().requires_grad_(True)
    J = velocity_misfit(vt, g, torch.from_numpy(wav).cuda(), nt, src, rec,
                        torch.from_numpy(obs).cuda(), 10)
    (3.0 * J).backward()
    grad = np.zeros(v.shape)
    J2 = seisgb.adjoint_shot(g, v, wav, nt, src, rec, obs, grad, ckpt_every=10)
    assert float(J) == J2
    np.testing.assert_allclose(vt.grad.cpu().numpy(), (3.0 * grad).astype(np.float32), rtol=1e-6,
                               atol=1e-6 * np.abs(3.0 * grad).max())


def test_gradient_matches_oracle_several_tiles():
    """96^3 (64^3 inner + 16-point PML): tile seams in x and y, several z
    chunks, the PML interface on every face; 120 steps, receivers every 5th
    surface point, source off the tile grid; observed traces = half those of
    the model without the anomaly."""
    n_in, nb, nt = 64, 16, 120
    N = n_in + 2 * nb
    shape = (N, N, N)
    v0 = synth.layered_model(shape, seed=11, vmin=1800, vmax=3200, perturb=0.02)
    v = (v0 * synth.gaussian_anomaly(shape, (50.0, 45.0, 40.0), 6.0, 0.06)).astype(np.float32)
    vmax = float(max(v.max(), v0.max()))
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, 10, 10, 10)))
    wav = synth.ricker(nt, dt, 25.0)
    src = (nb + 21, nb + 30, nb + 3)
    rec = synth.surface_receivers(n_in, n_in, nb, 5)
    go = oracle.Grid(n_in, n_in, n_in, nb, 10.0, 10.0, 10.0, dt, vmax=vmax, r0=float(np.float32(1e-3)))
    # halved: the anomaly's scattering reaches no receiver in 120 steps, so the
    # residual against the unperturbed model's own traces would be rounding noise
    obs = (0.5 * oracle.run_shot(go, v0, wav, nt, src, rec, want_state=False)["traces"]).astype(np.float32)
    J_ref, grad_ref = oracle.adjoint_shot(go, v, wav, nt, src, rec, obs.astype(np.float64))
    g = seisgb.make_grid(n_in, n_in, n_in, nb, 10.0, 10.0, 10.0, dt, vmax)
    grad = np.zeros(shape)
    J = seisgb.adjoint_shot(g, v, wav, nt, src, rec, obs, grad, ckpt_every=32)
    e_J, e_g = abs(J - J_ref) / J_ref, rel_l2(grad, grad_ref)
    print(f"96^3 adjoint vs oracle: misfit {e_J:.3e}, gradient rel L2 {e_g:.3e}")
    assert e_J <= 1e-4 and e_g <= 1e-3


@pytest.mark.slow
def test_full_size_directional_derivative_and_checkpoints():
    """The benchmark's gradient case (256^3, 2000 steps, checkpoints every 100),
    one shot: <dJ/dv, dv> against a central difference of the GPU misfit along
    the anomaly's own shape (fp32 forward runs, so a loose bound), and the
    gradient bit-identical with another checkpoint interval."""
    w = synth.GRADIENT
    v, v_obs = synth.gradient_models(w)
    dv = (v - v_obs).astype(np.float64)  # the anomaly: smooth, localised
    eps = 0.05
    vmax = float(max(v.max(), v_obs.max(), (v + eps * dv).max()))
    g0 = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, 1.0, vmax)
    dt = float(np.float32(w.cfl_fraction * seisgb.cfl_dt(g0, vmax)))
    g = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax)
    nt = w.nt
    wav = torch.from_numpy(synth.ricker(nt, dt, w.fp)).cuda()
    rec = w.receivers()
    src = synth.shot_grid(w)[5]
    obs = torch.zeros((nt, rec.shape[0]), device="cuda")
    seisgb.run_shot(g, torch.from_numpy(v_obs).cuda(), wav, nt, src, rec, obs)
    d_v = torch.from_numpy(v).cuda()
    grad = torch.zeros(v.shape, dtype=torch.float64, device="cuda")
    J = seisgb.adjoint_shot(g, d_v, wav, nt, src, rec, obs, grad, ckpt_every=100)
    grad2 = torch.zeros_like(grad)
    J2 = seisgb.adjoint_shot(g, d_v, wav, nt, src, rec, obs, grad2, ckpt_every=64)
    assert J2 == J and torch.equal(grad, grad2)
    assert bool(torch.isfinite(grad).all())

    def misfit(vv):
        tr = torch.zeros((nt, rec.shape[0]), device="cuda")
        seisgb.run_shot(g, torch.from_numpy(vv.astype(np.float32)).cuda(), wav, nt, src, rec, tr)
        return 0.5 * float(((tr.double() - obs.double()) ** 2).sum())

    assert abs(misfit(v) - J) <= 1e-6 * J  # the adjoint's misfit is run_shot's
    fd = (misfit(v + eps * dv) - misfit(v - eps * dv)) / (2 * eps)
    dd = float((grad * torch.from_numpy(dv).cuda()).sum())
    print(f"256^3 x 2000: <g, dv> {dd:.6e}, central difference {fd:.6e}, rel {abs(dd - fd) / abs(fd):.2e}")
    assert abs(dd - fd) <= 2e-2 * abs(fd)


def test_gradient_matches_oracle_ragged_anisotropic():
    """Inner 45 x 22 x 17 with a 7-point PML (computed 59 x 36 x 31: ragged tiles
    and a phi block that is only partly PML), spacings 10 / 12 / 8 m, 60 steps,
    checkpoints every 13 steps, observed = 0.6 x the traces of the model without
    the anomaly."""
    nx, ny, nz, nb, nt = 45, 22, 17, 7, 60
    dx, dy, dz = 10.0, 12.0, 8.0
    shape = (nz + 2 * nb, ny + 2 * nb, nx + 2 * nb)
    v0 = synth.layered_model(shape, seed=21, vmin=1700, vmax=2900, perturb=0.03)
    v = (v0 * synth.gaussian_anomaly(shape, (30.0, 17.0, 14.0), 4.0, -0.07)).astype(np.float32)
    vmax = float(max(v.max(), v0.max()))
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, dx, dy, dz)))
    wav = synth.ricker(nt, dt, 35.0)
    src = (nb + 40, nb + 5, nb + 2)
    rec = np.array([[nb + i, nb + j, nb + 1] for j in range(0, ny, 4) for i in range(0, nx, 3)],
                   dtype=np.int32)
    go = oracle.Grid(nx, ny, nz, nb, dx, dy, dz, dt, vmax=vmax, r0=float(np.float32(1e-3)))
    obs = (0.6 * oracle.run_shot(go, v0, wav, nt, src, rec, want_state=False)["traces"]).astype(np.float32)
    J_ref, grad_ref = oracle.adjoint_shot(go, v, wav, nt, src, rec, obs.astype(np.float64))
    g = seisgb.make_grid(nx, ny, nz, nb, dx, dy, dz, dt, vmax)
    grad = np.zeros(shape)
    J = seisgb.adjoint_shot(g, v, wav, nt, src, rec, obs, grad, ckpt_every=13)
    e_J, e_g = abs(J - J_ref) / J_ref, rel_l2(grad, grad_ref)
    print(f"ragged anisotropic adjoint vs oracle: misfit {e_J:.3e}, gradient rel L2 {e_g:.3e}")
    assert e_J <= 1e-4 and e_g <= 1e-3


def test_concurrent_calls_on_two_streams_match_sequential():
    """Two shots' gradients computed at once from two host threads on two
    streams (each call has its own scratch and device error word) equal the
    same calls made one after the other, bit for bit."""
    import threading
    g, go, v, wav, nt, src, rec, obs = _case()
    srcs = [src, (src[0] + 5, src[1] + 3, src[2] + 1)]
    d_v, d_w = torch.from_numpy(v).cuda(), torch.from_numpy(wav).cuda()
    d_o = torch.from_numpy(obs).cuda()
    seq = []
    for s in srcs:
        gr = torch.zeros(v.shape, dtype=torch.float64, device="cuda")
        seq.append((seisgb.adjoint_shot(g, d_v, d_w, nt, s, rec, d_o, gr, ckpt_every=10), gr))
    streams = [torch.cuda.Stream() for _ in srcs]
    out = [None, None]
    grads = [torch.zeros(v.shape, dtype=torch.float64, device="cuda") for _ in srcs]
    torch.cuda.synchronize()

    def run(k):
        with torch.cuda.stream(streams[k]):
            out[k] = seisgb.adjoint_shot(g, d_v, d_w, nt, srcs[k], rec, d_o, grads[k], ckpt_every=10,
                                         stream=streams[k])

    threads = [threading.Thread(target=run, args=(k,)) for k in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    for k in range(2):
        assert out[k] == seq[k][0] and torch.equal(grads[k], seq[k][1])
