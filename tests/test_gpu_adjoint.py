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
