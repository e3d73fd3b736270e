"""Pins of the fp64 oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed axis, a mis-scaled source, a wrong CFL
constant) fails at least one of them.  None of these tests touches the GPU.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2009_04619_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
# 25-point Laplacian coefficients (section III-A, Eq. 3)
# --------------------------------------------------------------------------

def test_fd2_weights_match_published_table():
    """Oracle's closed-form weights equal Fornberg's published table (golden)."""
    for row in _read_golden("fd2_weights.txt"):
        M = int(row[0])
        exact = [float(Fraction(x)) for x in row[1:]]
        w = oracle.fd2_weights(M)
        np.testing.assert_allclose(w, exact, rtol=1e-14, atol=1e-15)


def test_weight_moments():
    """Moment conditions of an 8th-order 2nd-derivative stencil: sum w = 0,
    2 sum w_m m^2 = 2, 2 sum w_m m^{2p} = 0 (p = 2..4), 2 sum w_m m^10 = -1152."""
    w = oracle.fd2_weights(4)
    assert abs(w[0] + 2 * w[1:].sum()) < 1e-14
    mom = lambda p: 2 * sum(w[m] * m ** (2 * p) for m in range(1, 5))
    assert abs(mom(1) - 2.0) < 1e-13
    for p in (2, 3, 4):
        assert abs(mom(p)) < 1e-9 * 4 ** (2 * p)
    assert abs(mom(5) + 1152.0) < 1e-6


def test_laplacian_coeff_scaling_anisotropic():
    g = oracle.Grid(4, 4, 4, 0, 3.0, 5.0, 7.0, 1e-3)
    c0, cx, cy, cz = oracle.laplacian_coeffs(g)
    w = [float(Fraction(x)) for x in _read_golden("fd2_weights.txt")[3][1:]]
    assert math.isclose(c0, w[0] * (1 / 9 + 1 / 25 + 1 / 49), rel_tol=1e-14)
    for m in range(1, 5):
        assert math.isclose(cx[m], w[m] / 9, rel_tol=1e-14)
        assert math.isclose(cy[m], w[m] / 25, rel_tol=1e-14)
        assert math.isclose(cz[m], w[m] / 49, rel_tol=1e-14)


def _poly_field(g, coeffs, degree_terms):
    """Evaluate sum c x^a y^b z^e on the oracle layout (halo included) at physical
    coordinates x = (i - Nx/2) dx etc.; return the field and its analytic
    Laplacian on the computed points."""
    H = oracle.H
    Nz, Ny, Nx = g.shape
    i = (np.arange(-H, Nx + H) - Nx / 2) * g.dx
    j = (np.arange(-H, Ny + H) - Ny / 2) * g.dy
    k = (np.arange(-H, Nz + H) - Nz / 2) * g.dz
    Z, Y, X = np.meshgrid(k, j, i, indexing="ij")
    u = np.zeros_like(X)
    lap = np.zeros_like(X)
    for c, (a, b, e) in zip(coeffs, degree_terms):
        u += c * X ** a * Y ** b * Z ** e
        if a >= 2:
            lap += c * a * (a - 1) * X ** (a - 2) * Y ** b * Z ** e
        if b >= 2:
            lap += c * b * (b - 1) * X ** a * Y ** (b - 2) * Z ** e
        if e >= 2:
            lap += c * e * (e - 1) * X ** a * Y ** b * Z ** (e - 2)
    return u, oracle.unpad(lap)


def test_laplacian_exact_on_degree9_polynomials():
    """The 8th-order stencil is exact for every polynomial of degree <= 9, and a
    dropped or mis-scaled term on any axis breaks that."""
    rng = np.random.default_rng(7)
    g = oracle.Grid(11, 9, 13, 0, 0.7, 1.3, 1.1, 1e-3)
    terms = [(a, b, e) for a in range(10) for b in range(10) for e in range(10) if a + b + e <= 9]
    coeffs = rng.standard_normal(len(terms))
    u, lap_exact = _poly_field(g, coeffs, terms)
    lap = oracle.laplacian_full(g, u)
    scale = np.abs(lap_exact).max()
    assert np.abs(lap - lap_exact).max() < 1e-10 * scale


def test_laplacian_degree10_truncation_term():
    """On x^10 the stencil's error is exactly (2 sum w_m m^10) h^8 = -1152 h^8."""
    h = 0.5
    g = oracle.Grid(9, 1, 1, 0, h, 1.0, 1.0, 1e-3)
    H = oracle.H
    Nz, Ny, Nx = g.shape
    x = (np.arange(-H, Nx + H) - 4) * h
    u = np.zeros(oracle.full_shape(g))
    u[:, :, :] = x[None, None, :] ** 10
    lap = oracle.laplacian_full(g, u)[0, 0, :]
    xi = x[H:-H]
    err = lap - 90 * xi ** 8
    np.testing.assert_allclose(err, -1152.0 * h ** 8, rtol=1e-6, atol=1e-6 * 1152 * h ** 8)


def test_laplacian_symmetry_group():
    """With equal spacing the star stencil commutes with all 48 axis permutations
    and reflections of a cube."""
    rng = np.random.default_rng(3)
    n = 10
    g = oracle.Grid(n, n, n, 0, 2.0, 2.0, 2.0, 1e-3)
    u = rng.standard_normal((n, n, n))
    lap = oracle.laplacian(g, u)
    for perm in itertools.permutations(range(3)):
        for flips in itertools.product((False, True), repeat=3):
            def T(a):
                a = np.transpose(a, perm)
                for ax, f in enumerate(flips):
                    if f:
                        a = np.flip(a, ax)
                return np.ascontiguousarray(a)
            np.testing.assert_allclose(oracle.laplacian(g, T(u)), T(lap), rtol=0, atol=1e-12)


# --------------------------------------------------------------------------
# Time step, CFL (Eq. 2, Algorithm 1)
# --------------------------------------------------------------------------

def test_cfl_constant_closed_form():
    """Von Neumann limit: dt_max = 2 / (v sqrt(S sum h^-2)), S = 2048/315 at theta = pi."""
    S = 2048 / 315
    for (v, dx, dy, dz) in [(2000, 10, 10, 10), (4500, 10, 7, 12), (1500, 3, 3, 3)]:
        expect = 2.0 / (v * math.sqrt(S * (dx ** -2 + dy ** -2 + dz ** -2)))
        assert math.isclose(oracle.cfl_dt(v, dx, dy, dz), expect, rel_tol=1e-14)
    # the symbol's maximum is at theta = pi
    w = oracle.fd2_weights(4)
    th = np.linspace(0, np.pi, 20001)
    sym = -(w[0] + 2 * sum(w[m] * np.cos(m * th) for m in range(1, 5)))
    assert abs(sym.max() - S) < 1e-12 and np.argmax(sym) == len(th) - 1
    assert math.isclose(oracle.cfl_dt(2000, 10, 10, 10) * 2000 / 10, 0.4528555233184, rel_tol=1e-12)


@pytest.mark.parametrize("factor,stable", [(0.99, True), (1.01, False)])
def test_cfl_blowup(factor, stable):
    """A run slightly above the CFL limit diverges; slightly below stays bounded."""
    n = 40
    v, h = 2000.0, 10.0
    dt = factor * oracle.cfl_dt(v, h, h, h)
    g = oracle.Grid(n, n, n, 0, h, h, h, dt, vmax=v, r0=1.0)
    vel = synth.constant_model(g.shape, v)
    w = synth.ricker(2000, dt, 25.0)
    res = oracle.run_shot(g, vel, w, 2000, (20, 20, 20), np.zeros((0, 3), np.int32))
    peak = np.nanmax(np.abs(res["u"]))
    if stable:
        assert np.isfinite(res["u"]).all() and peak < 1.0
    else:
        assert (not np.isfinite(res["u"]).all()) or peak > 1e10


def test_step_is_eq2_in_inner_region():
    """Away from the PML the update is u^{n+1} = 2u^n - u^{n-1} + m L u^n exactly
    (checked against the oracle's own Laplacian on random data)."""
    rng = np.random.default_rng(11)
    g = oracle.Grid(12, 10, 8, 3, 10.0, 9.0, 8.0, 1e-3, vmax=3000.0, r0=1e-3)
    sh = g.shape
    m = rng.uniform(0.01, 0.1, sh)
    up, uc, ph = rng.standard_normal(sh), rng.standard_normal(sh), np.zeros(sh)
    un, pn = oracle.step(g, m, up, uc, ph)
    L = oracle.laplacian(g, uc)
    nb = g.nb
    inner = (slice(nb, nb + g.nz), slice(nb, nb + g.ny), slice(nb, nb + g.nx))
    np.testing.assert_allclose(un[inner], (2 * uc - up + m * L)[inner], rtol=1e-13, atol=1e-13)
    assert np.all(pn[inner] == 0.0)


def test_pml_step_matches_hand_derivation_at_one_point():
    """At one PML point, recompute a2 from its definition with independent index
    arithmetic (numpy slicing of the compact field)."""
    rng = np.random.default_rng(5)
    g = oracle.Grid(6, 5, 7, 4, 10.0, 12.0, 8.0, 1.3e-3, vmax=3500.0, r0=1e-3)
    sh = g.shape
    m = rng.uniform(0.01, 0.1, sh)
    up, uc, ph = rng.standard_normal(sh), rng.standard_normal(sh), rng.standard_normal(sh) * 0.1
    un, pn = oracle.step(g, m, up, uc, ph)
    w = [float(Fraction(x)) for x in _read_golden("fd2_weights.txt")[3][1:]]
    big = np.zeros(tuple(s + 8 for s in sh))
    big[4:-4, 4:-4, 4:-4] = uc
    for (i, j, k) in [(1, 2, 3), (0, 0, 0), (13, 12, 14), (5, 6, 1), (2, 7, 9)]:
        K, J, I = k + 4, j + 4, i + 4
        L = w[0] * (g.dx ** -2 + g.dy ** -2 + g.dz ** -2) * big[K, J, I]
        for mm in range(1, 5):
            L += w[mm] * ((big[K, J, I + mm] + big[K, J, I - mm]) / g.dx ** 2 +
                          (big[K, J + mm, I] + big[K, J - mm, I]) / g.dy ** 2 +
                          (big[K + mm, J, I] + big[K - mm, J, I]) / g.dz ** 2)

        def prof(n_in, q, h):
            d = max(g.nb - q, q - (g.nb + n_in - 1), 0)
            return -3 * g.vmax * math.log(g.r0) / (2 * g.nb * h) * (d / g.nb) ** 2
        e = prof(g.nx, i, g.dx) + prof(g.ny, j, g.dy) + prof(g.nz, k, g.dz)
        gde = ((prof(g.nx, i + 1, g.dx) - prof(g.nx, i - 1, g.dx)) * (big[K, J, I + 1] - big[K, J, I - 1]) / (4 * g.dx ** 2)
               + (prof(g.ny, j + 1, g.dy) - prof(g.ny, j - 1, g.dy)) * (big[K, J + 1, I] - big[K, J - 1, I]) / (4 * g.dy ** 2)
               + (prof(g.nz, k + 1, g.dz) - prof(g.nz, k - 1, g.dz)) * (big[K + 1, J, I] - big[K - 1, J, I]) / (4 * g.dz ** 2))
        ed = e * g.dt
        u_exp = ((2 - ed ** 2) * uc[k, j, i] - (1 - ed) * up[k, j, i] + m[k, j, i] * (L + ph[k, j, i])) / (1 + ed)
        p_exp = (ph[k, j, i] - g.dt * gde) / (1 + ed)
        assert oracle.is_pml(g, i, j, k)
        assert math.isclose(un[k, j, i], u_exp, rel_tol=1e-12, abs_tol=1e-12)
        assert math.isclose(pn[k, j, i], p_exp, rel_tol=1e-12, abs_tol=1e-14)


# --------------------------------------------------------------------------
# Green's function (source scaling and recurrence), before any reflection
# --------------------------------------------------------------------------

def _green_case(scale):
    w = synth.SMALL
    h = w.h / scale
    n_in, nb = 64 * scale, 16 * scale
    nt = w.nt * scale
    dt = np.float32(0.4 * oracle.cfl_dt(w.v_const, w.h, w.h, w.h) / scale)
    g = oracle.Grid(n_in, n_in, n_in, nb, np.float32(h), np.float32(h), np.float32(h), float(dt),
                    vmax=w.v_const, r0=1e-3)
    N = n_in + 2 * nb
    c = N // 2
    # delay 1.2/fp so the wavelet starts from ~2e-5 of its peak: a start-up jump
    # would add an error that does not shrink under refinement
    wav = synth.ricker(nt, float(dt), w.fp, t0=1.2 / w.fp)
    offs = [5, 10, 15]
    rec = []
    for r in offs:
        rs = r * scale
        rec += [(c + rs, c, c), (c, c - rs, c), (c, c, c + rs)]
        d = int(round(rs / math.sqrt(3)))
        rec += [(c + d, c + d, c + d)]
    rec = np.array(rec, dtype=np.int32)
    res = oracle.run_shot(g, synth.constant_model(g.shape, w.v_const), wav, nt, (c, c, c), rec)
    return g, res, rec, c, float(dt), wav


def _green_exact(r_m, t, v, fp):
    tau = t - r_m / v - 1.2 / fp
    a = (np.pi * fp * tau) ** 2
    return (1 - 2 * a) * np.exp(-a) / (4 * np.pi * r_m)


@pytest.mark.slow
def test_green_function_and_refinement():
    """Homogeneous 3D Green's function u = w(t - r/v) / (4 pi r) (Eq. 1 with a point
    source), compared on 4 <= r <= 17 points at step 100 of the 64^3 + PML 16 case,
    and again after halving h and dt at fixed physical geometry."""
    errs = []
    for scale in (1, 2):
        g, res, rec, c, dt, wav = _green_case(scale)
        nt = res["traces"].shape[0]
        u = res["u"]
        Nz, Ny, Nx = g.shape
        K, J, I = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
        r_pts = np.sqrt((I - c) ** 2 + (J - c) ** 2 + (K - c) ** 2) / scale
        sel = (r_pts >= 4) & (r_pts <= 17)
        r_m = r_pts[sel] * 10.0
        ex = _green_exact(r_m, nt * dt, 2000.0, 15.0)
        err = np.linalg.norm(u[sel] - ex) / np.linalg.norm(ex)
        # traces along axes and diagonals
        t = (np.arange(nt) + 1) * dt
        rr = np.sqrt(((rec - c) ** 2).sum(axis=1)) / scale * 10.0
        ex_tr = _green_exact(rr[None, :], t[:, None], 2000.0, 15.0)
        err_tr = np.linalg.norm(res["traces"] - ex_tr) / np.linalg.norm(ex_tr)
        errs.append((err, err_tr))
        print("green rel L2 (wavefield, traces):", errs[-1])
    assert errs[0][0] < 3e-2 and errs[0][1] < 3e-2, errs
    assert errs[1][0] < errs[0][0] / 3 and errs[1][1] < errs[0][1] / 3, errs


def test_green_far_field_symmetry_small():
    """Centred source in a cube with a PML: the wavefield is invariant under the
    48 symmetries of the cube (Eq. 3 and the PML are both isotropic)."""
    n, nb = 15, 5
    v, h = 2000.0, 10.0
    dt = np.float32(0.4 * oracle.cfl_dt(v, h, h, h))
    g = oracle.Grid(n, n, n, nb, h, h, h, float(dt), vmax=v, r0=1e-3)
    N = n + 2 * nb
    c = N // 2
    wav = synth.ricker(60, float(dt), 25.0)
    res = oracle.run_shot(g, synth.constant_model(g.shape, v), wav, 60, (c, c, c), np.zeros((0, 3), np.int32))
    u, ph = res["u"], res["phi"]
    sc = np.abs(u).max()
    for perm in itertools.permutations(range(3)):
        for flips in itertools.product((False, True), repeat=3):
            a, b = np.transpose(u, perm), np.transpose(ph, perm)
            for ax, f in enumerate(flips):
                if f:
                    a, b = np.flip(a, ax), np.flip(b, ax)
            assert np.abs(a - u).max() <= 1e-12 * sc
            assert np.abs(b - ph).max() <= 1e-12 * max(np.abs(ph).max(), 1e-300)


# --------------------------------------------------------------------------
# PML invariants (parity of the PML itself is pinned by invariants only)
# --------------------------------------------------------------------------

def test_pml_with_zero_damping_is_the_interior_update():
    """eta = 0 (r0 = 1) turns the PML update into Eq. 2 bit for bit and keeps phi = 0:
    compare with the same computed domain declared as all-inner (nb = 0)."""
    n, nb = 10, 4
    v, h = 2500.0, 10.0
    dt = float(np.float32(0.4 * oracle.cfl_dt(v, h, h, h)))
    rng = np.random.default_rng(2)
    N = n + 2 * nb
    vel = rng.uniform(1500, 2500, (N, N, N)).astype(np.float32)
    wav = synth.ricker(40, dt, 20.0)
    rec = np.array([[3, 4, 5], [9, 9, 9], [0, 17, 2]], dtype=np.int32)
    a = oracle.run_shot(oracle.Grid(n, n, n, nb, h, h, h, dt, vmax=v, r0=1.0), vel, wav, 40, (8, 9, 7), rec)
    b = oracle.run_shot(oracle.Grid(N, N, N, 0, h, h, h, dt, vmax=v, r0=1.0), vel, wav, 40, (8, 9, 7), rec)
    assert np.array_equal(a["u"], b["u"]) and np.array_equal(a["traces"], b["traces"])
    assert np.all(a["phi"] == 0.0)


def _absorb_runs():
    v, h, fp = 2000.0, 10.0, 15.0
    dt = float(np.float32(0.4 * oracle.cfl_dt(v, h, h, h)))
    nt = int(0.30 / dt)
    wav = synth.ricker(nt, dt, fp)
    n_win, nb = 40, 16
    out = {}
    for tag, n_in in (("small", n_win), ("big", n_win + 64)):
        g = oracle.Grid(n_in, n_in, n_in, nb, h, h, h, dt, vmax=v, r0=1e-3)
        N = n_in + 2 * nb
        c = N // 2
        # receivers fill the inner window of the small case (every 2nd point)
        lo = c - n_win // 2
        ii = np.arange(lo, lo + n_win, 2)
        K, J, I = np.meshgrid(ii, ii, ii, indexing="ij")
        rec = np.stack([I.ravel(), J.ravel(), K.ravel()], 1).astype(np.int32)
        res = oracle.run_shot(g, synth.constant_model(g.shape, v), wav, nt, (c, c, c), rec,
                              want_state=False)
        out[tag] = res["traces"]
    return out, dt


@pytest.mark.slow
def test_pml_absorbs_and_energy_decays():
    """The PML reflects little: inside the inner window the run with a 16-point
    PML stays within 1% of the peak incident amplitude of a run on a domain 64
    points wider per side (whose own boundary is too far to be seen), and the
    window empties once the wave has left."""
    out, dt = _absorb_runs()
    small, big = out["small"], out["big"]
    peak = np.abs(big).max()
    diff = np.abs(small - big).max() / peak
    # measured when first written: 1.4e-3 and 2.3e-3
    assert diff < 5e-3, diff
    late = np.abs(small[-20:]).max() / peak
    assert late < 1e-2, late


# --------------------------------------------------------------------------
# Domain decomposition geometry (section III-B, Table III)
# --------------------------------------------------------------------------

def test_seven_regions_partition_the_domain():
    """Regions 0..6 cover every computed point once; region 0 is exactly the
    non-PML set; top/bottom span full x-y, front/back full x and inner z,
    left/right inner y and inner z."""
    g = oracle.Grid(5, 6, 7, 3, 1.0, 1.0, 1.0, 1e-3)
    Nz, Ny, Nx = g.shape
    reg = np.zeros(g.shape, dtype=int)
    for k in range(Nz):
        for j in range(Ny):
            for i in range(Nx):
                reg[k, j, i] = oracle.region(g, i, j, k)
                assert (reg[k, j, i] == 0) == (not oracle.is_pml(g, i, j, k))
    nb = g.nb
    counts = np.bincount(reg.ravel(), minlength=7)
    assert counts[0] == g.nx * g.ny * g.nz
    assert counts[1] == counts[2] == nb * Ny * Nx
    assert counts[3] == counts[4] == g.nz * nb * Nx
    assert counts[5] == counts[6] == g.nz * g.ny * nb
    assert counts.sum() == Nz * Ny * Nx


def _region_extent(g, r, probe):
    """Extent of region r along each axis through a probe point inside it."""
    Nz, Ny, Nx = g.shape
    i0, j0, k0 = probe
    ex = sum(oracle.region(g, i, j0, k0) == r for i in range(Nx))
    ey = sum(oracle.region(g, i0, j, k0) == r for j in range(Ny))
    ez = sum(oracle.region(g, i0, j0, k) == r for k in range(Nz))
    return ex, ey, ez


def test_table3_grid_sizes_fix_the_geometry():
    """Table III's block counts on the 1000^3 V100 run equal ceil(extent/block)
    products of this region geometry with 946 inner points and a 27-point PML."""
    g = oracle.Grid(946, 946, 946, 27, 1.0, 1.0, 1.0, 1e-3)
    probes = {"inner": (500, 500, 500), "top": (500, 500, 3), "front": (500, 3, 500),
              "left": (3, 500, 500)}
    ids = {"inner": 0, "top": 1, "front": 3, "left": 5}
    for row in _read_golden("table3_grid_sizes.txt"):
        name, bx, by, bz, reg, blocks = row[0], int(row[1]), int(row[2]), int(row[3]), row[4], int(row[5])
        ex, ey, ez = _region_extent(g, ids[reg], probes[reg])
        got = math.ceil(ex / bx) * math.ceil(ey / by) * math.ceil(ez / bz)
        assert got == blocks, (name, reg, got, blocks)


def test_step_points_equals_full_step():
    """The per-point entry (used for full-size GPU parity on samples) gives the
    same numbers as the whole-grid step, bit for bit, on fp32-representable data."""
    rng = np.random.default_rng(9)
    g = oracle.Grid(9, 7, 6, 4, 10.0, 12.0, 9.0, 1.1e-3, vmax=3000.0, r0=1e-3)
    sh = g.shape
    f = lambda s=1.0: (rng.standard_normal(sh) * s).astype(np.float32)
    m = rng.uniform(0.01, 0.1, sh).astype(np.float32)
    up, uc, ph = f(), f(), f(0.1)
    un, pn = oracle.step(g, m, up, uc, ph)
    Nz, Ny, Nx = sh
    pts = np.array([(i, j, k) for k in range(Nz) for j in range(Ny) for i in range(Nx)
                    if (i * 7 + j * 3 + k) % 5 == 0], dtype=np.int32)
    ou, op = oracle.step_points(g, m, up, uc, ph, pts)
    assert np.array_equal(ou, un[pts[:, 2], pts[:, 1], pts[:, 0]])
    assert np.array_equal(op, pn[pts[:, 2], pts[:, 1], pts[:, 0]])
