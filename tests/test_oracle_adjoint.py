"""Pins of the oracle's adjoint gradient: central finite differences of the
fp64 misfit, in random directions and at single points in the inner region,
the PML and on the inner/PML interface (the 32^3 / 50-step instance)."""
import numpy as np
import pytest

import oracle
from paper_2009_04619_gb300 import synth

EXACT = 1.0 / 16  # velocity steps that are exact in fp32 for v < 2^20


def _case(nb=8, n_in=16, nt=50, seed=3):
    N = n_in + 2 * nb
    shape = (N, N, N)
    v0 = synth.layered_model(shape, seed=seed, vmin=1800, vmax=3000, perturb=0.0)
    v = (v0 * synth.gaussian_anomaly(shape, (N / 2, N / 2, N / 2 + 3), 3.0, 0.08)).astype(np.float32)
    vmax = float(max(v.max(), v0.max()))
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, 10, 10, 10)))
    g = oracle.Grid(n_in, n_in, n_in, nb, 10.0, 10.0, 10.0, dt, vmax=vmax, r0=1e-3)
    wav = synth.ricker(nt, dt, 30.0)
    src = (nb + 1, nb + 2, nb + 2)  # next to a corner: every PML region sees the wave
    rec = synth.surface_receivers(n_in, n_in, nb, 3)
    # observed data: half the unperturbed model's traces, so that the residual
    # is large and the central differences of the misfit are accurate to O(dv^2)
    obs = 0.5 * oracle.run_shot(g, v0, wav, nt, src, rec, want_state=False)["traces"]
    return g, v, wav, nt, src, rec, obs


def _misfit(g, v, wav, nt, src, rec, obs):
    d = oracle.run_shot(g, v, wav, nt, src, rec, want_state=False)["traces"]
    return 0.5 * float(np.sum((d - obs) ** 2))


def test_misfit_matches_forward_traces():
    g, v, wav, nt, src, rec, obs = _case()
    J, _ = oracle.adjoint_shot(g, v, wav, nt, src, rec, obs)
    assert J > 0 and abs(J - _misfit(g, v, wav, nt, src, rec, obs)) <= 1e-12 * J


def test_gradient_vs_central_differences_random_directions():
    g, v, wav, nt, src, rec, obs = _case()
    J, grad = oracle.adjoint_shot(g, v, wav, nt, src, rec, obs)
    rng = np.random.default_rng(0)
    for _ in range(3):
        dv = (rng.integers(-2, 3, size=v.shape) * EXACT).astype(np.float32)
        jp = _misfit(g, (v + dv).astype(np.float32), wav, nt, src, rec, obs)
        jm = _misfit(g, (v - dv).astype(np.float32), wav, nt, src, rec, obs)
        fd = (jp - jm) / 2.0
        ad = float(np.sum(grad * dv))
        assert abs(fd - ad) <= 1e-3 * abs(fd), (fd, ad)


def _region_masks(g, rec, src):
    Nz, Ny, Nx = g.shape
    nb = g.nb
    K, J, I = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    d = lambda q, n_in: np.maximum(np.maximum(nb - q, q - (nb + n_in - 1)), 0)
    dx, dy, dz = d(I, g.nx), d(J, g.ny), d(K, g.nz)
    pml = (dx > 0) | (dy > 0) | (dz > 0)
    near = np.zeros_like(pml)
    for ax in range(3):
        near |= np.roll(pml, 1, ax) | np.roll(pml, -1, ax)
    at_rec = np.zeros_like(pml)
    at_rec[rec[:, 2], rec[:, 1], rec[:, 0]] = True
    at_src = np.zeros_like(pml)
    at_src[src[2], src[1], src[0]] = True
    return {"inner": ~pml & ~near, "pml_one_axis": pml & ((dx > 0) + (dy > 0) + (dz > 0) == 1),
            "pml_corner": (dx > 0) & (dy > 0) & (dz > 0), "interface_inner": ~pml & near,
            "interface_pml": pml & (dx + dy + dz == 1), "receiver": at_rec, "source": at_src}


@pytest.mark.parametrize("where", ["inner", "pml_one_axis", "pml_corner", "interface_inner",
                                   "interface_pml", "receiver", "source"])
def test_gradient_vs_central_differences_single_points(where):
    """At the most sensitive point of each region (PML edges and corners, both
    sides of the inner/PML interface, a receiver, the source), the adjoint
    gradient equals the central difference of the misfit."""
    g, v, wav, nt, src, rec, obs = _case()
    J, grad = oracle.adjoint_shot(g, v, wav, nt, src, rec, obs)
    mask = _region_masks(g, rec, src)[where]
    cand = np.where(mask, np.abs(grad), -1.0)
    k, j, i = np.unravel_index(np.argmax(cand), cand.shape)
    assert abs(grad[k, j, i]) > 1e-6 * np.abs(grad).max()
    dv = np.zeros_like(v)
    dv[k, j, i] = 4 * EXACT
    jp = _misfit(g, (v + dv).astype(np.float32), wav, nt, src, rec, obs)
    jm = _misfit(g, (v - dv).astype(np.float32), wav, nt, src, rec, obs)
    fd = (jp - jm) / 2.0
    ad = float(grad[k, j, i] * dv[k, j, i])
    assert abs(fd - ad) <= 1e-3 * abs(fd), (where, (i, j, k), fd, ad)


def test_gradient_vs_central_differences_anisotropic_ragged():
    """Unequal spacings and extents (a swapped axis or spacing in the adjoint's
    PML terms would show here): inner 9 x 7 x 6, 5-point PML, dx, dy, dz =
    10, 13, 8 m, 40 steps; random directions and the most sensitive PML point
    on each axis."""
    nx, ny, nz, nb, nt = 9, 7, 6, 5, 40
    dxs = (10.0, 13.0, 8.0)
    shape = (nz + 2 * nb, ny + 2 * nb, nx + 2 * nb)
    v0 = synth.layered_model(shape, seed=8, vmin=1800, vmax=2800, perturb=0.0)
    v = (v0 * synth.gaussian_anomaly(shape, (9.0, 8.0, 8.0), 2.0, 0.1)).astype(np.float32)
    vmax = float(max(v.max(), v0.max()))
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, *dxs)))
    g = oracle.Grid(nx, ny, nz, nb, *dxs, dt, vmax=vmax, r0=1e-3)
    wav = synth.ricker(nt, dt, 45.0)
    src = (nb + 1, nb + 5, nb + 1)
    rec = np.array([[nb + i, nb + j, nb] for j in range(0, ny, 2) for i in range(0, nx, 2)],
                   dtype=np.int32)
    obs = 0.5 * oracle.run_shot(g, v0, wav, nt, src, rec, want_state=False)["traces"]
    J, grad = oracle.adjoint_shot(g, v, wav, nt, src, rec, obs)
    rng = np.random.default_rng(2)
    for _ in range(2):
        dv = (rng.integers(-2, 3, size=v.shape) * EXACT).astype(np.float32)
        fd = (_misfit(g, (v + dv).astype(np.float32), wav, nt, src, rec, obs) -
              _misfit(g, (v - dv).astype(np.float32), wav, nt, src, rec, obs)) / 2.0
        assert abs(fd - float(np.sum(grad * dv))) <= 1e-3 * abs(fd)
    # the most sensitive point in the x-only, y-only and z-only PML
    Nz, Ny, Nx = shape
    K, Jj, I = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    depth = lambda q, n: np.maximum(np.maximum(nb - q, q - (nb + n - 1)), 0)
    ddx, ddy, ddz = depth(I, nx), depth(Jj, ny), depth(K, nz)
    for mask in ((ddx > 0) & (ddy == 0) & (ddz == 0), (ddy > 0) & (ddx == 0) & (ddz == 0),
                 (ddz > 0) & (ddx == 0) & (ddy == 0)):
        idx = np.unravel_index(np.argmax(np.where(mask, np.abs(grad), -1.0)), shape)
        dv = np.zeros(shape, np.float32)
        dv[idx] = 4 * EXACT
        fd = (_misfit(g, (v + dv).astype(np.float32), wav, nt, src, rec, obs) -
              _misfit(g, (v - dv).astype(np.float32), wav, nt, src, rec, obs)) / 2.0
        assert abs(fd - float(np.sum(grad * dv))) <= 1e-3 * abs(fd), (idx, fd)
