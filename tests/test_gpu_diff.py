"""The difference form of the leapfrog step (stencil_step_diff, storage
SGB_FP32_DIFF / SGB_BF16_DIFF): the state is u^n and d^n = u^n - u^{n-1}.

In exact arithmetic one step equals Eq. 2 (and the PML update) with
u^{n-1} = u^n - d^n, so the fp64 oracle's step from (u^{n-1}, u^n) gives the
expected u^{n+1}, and d^{n+1} = u^{n+1} - u^n.  Per point the GPU's d^{n+1} is
held to 1e-6 S, S an upper bound of the absolute terms the difference form
adds (|d^n| + |u^n| + |m| (sum of the Laplacian's |terms| + |phi|) + |phi|:
the |u^n| covers the e^2 u^n term of the PML form); u^{n+1} = u^n + d^{n+1}
adds one fp32 rounding.  bf16 stores each of the two with stochastic rounding,
within one bf16 spacing of the fp32 value.  run_shot in difference form must
equal a loop of stencil_step_diff calls bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_04619_gb300 import seisgb, synth
from gpu_util import abs_term_sum, ensure_lib, from_padded, padded_zeros, to_padded

pytestmark = pytest.mark.gpu

CASES = [
    # nx, ny, nz, nb, (dx, dy, dz), source offset from the inner corner
    (90, 37, 29, 5, (10.0, 11.0, 12.0), (45, 18, 14)),   # several tiles, ragged, anisotropic
    (40, 33, 70, 0, (7.0, 7.0, 7.0), (20, 3, 60)),       # no PML
    (9, 7, 6, 3, (10.0, 10.0, 10.0), (4, 3, 3)),         # tiny inner region, PML corners
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _ulp_bf16(x):
    """Spacing of the bf16 grid around |x| (8 significant bits)."""
    ax = np.maximum(np.abs(x), 1e-30)
    return np.exp2(np.floor(np.log2(ax)) - 7)


def _bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def _setup(case, bf16):
    nx, ny, nz, nb, h, so = case
    vmax = 3000.0
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, *h)))
    storage = seisgb.BF16_DIFF if bf16 else seisgb.FP32_DIFF
    g = seisgb.make_grid(nx, ny, nz, nb, *h, dt, vmax, 1e-3, storage)
    go = oracle.Grid(nx, ny, nz, nb, float(np.float32(h[0])), float(np.float32(h[1])),
                     float(np.float32(h[2])), dt, vmax=float(np.float32(vmax)),
                     r0=float(np.float32(1e-3)))
    rng = np.random.default_rng(nx * 13 + ny + 7 * nz + int(bf16))
    sh = g.shape
    uc = rng.standard_normal(sh).astype(np.float32)
    dn = (0.3 * rng.standard_normal(sh)).astype(np.float32)
    if bf16:
        uc, dn = _bf16(uc), _bf16(dn)
    ph = (0.1 * rng.standard_normal(sh)).astype(np.float32)
    Nz, Ny, Nx = sh
    K, J, I = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    inner = ((I >= nb) & (I < nb + nx) & (J >= nb) & (J < nb + ny) & (K >= nb) & (K < nb + nz))
    ph[inner] = 0.0
    vel = rng.uniform(1500, 3000, sh).astype(np.float32)
    m = (vel.astype(np.float64) ** 2 * dt ** 2).astype(np.float32)
    src = (nb + so[0], nb + so[1], nb + so[2])
    wav = np.linspace(-1, 1, 12).astype(np.float32)
    return g, go, uc, dn, ph, m, src, wav


@pytest.mark.parametrize("bf16", [False, True], ids=["fp32", "bf16"])
@pytest.mark.parametrize("case", CASES)
def test_stencil_step_diff_vs_oracle(case, bf16):
    g, go, uc, dn, ph, m, src, wav = _setup(case, bf16)
    step = 5
    sh = g.shape
    cast = (lambda t: t.to(torch.bfloat16)) if bf16 else (lambda t: t)
    d_uc, d_d = cast(to_padded(g, uc)), cast(to_padded(g, dn))
    d_un = cast(padded_zeros(g))
    d_m, d_ph = to_padded(g, m), to_padded(g, ph)
    d_w = torch.from_numpy(wav).cuda()
    seisgb.stencil_step_diff(g, d_uc, d_un, d_d, d_m, d_ph, step, source=(*src, d_w))
    seisgb.device_status()
    torch.cuda.synchronize()
    un, dd = from_padded(g, d_un.float()), from_padded(g, d_d.float())
    pn = from_padded(g, d_ph)
    # the halo of the written fields stays zero
    L = seisgb.layout(g)
    mask = torch.ones(int(L.elems), dtype=torch.bool, device="cuda")
    inside = padded_zeros(g)
    seisgb.pack(g, torch.ones(sh, device="cuda"), inside)
    mask &= inside == 0
    assert not bool(d_un.float()[mask].any()) and not bool(d_d.float()[mask].any())

    up = uc.astype(np.float64) - dn.astype(np.float64)  # u^{n-1}, exact in fp64
    ref_u, ref_p = oracle.step(go, m, up, uc, ph)
    inv_vol = 1.0 / (go.dx * go.dy * go.dz)
    term = float(m[src[2], src[1], src[0]]) * float(wav[step]) * inv_vol
    ref_u[src[2], src[1], src[0]] += term
    ref_d = ref_u - uc.astype(np.float64)
    S = abs_term_sum(go, m, up, uc, ph) - np.abs(uc) - np.abs(up) + np.abs(dn)
    S[src[2], src[1], src[0]] += abs(term)
    tol_d = 1e-6 * S + 1e-30
    tol_u = tol_d + 2.0 ** -24 * np.abs(ref_u)
    if bf16:  # each stored value is one of the two bf16 neighbours of its fp32 value
        tol_d = tol_d + _ulp_bf16(ref_d) * (1 + 1e-3)
        tol_u = tol_u + _ulp_bf16(ref_u) * (1 + 1e-3)
    err_d, err_u = np.abs(dd - ref_d), np.abs(un - ref_u)
    assert np.all(err_d <= tol_d), (float((err_d / tol_d).max()), np.unravel_index(np.argmax(err_d / tol_d), sh))
    assert np.all(err_u <= tol_u), (float((err_u / tol_u).max()), np.unravel_index(np.argmax(err_u / tol_u), sh))
    errp = np.abs(pn - ref_p)
    Sp = np.abs(ph) + np.abs(ref_p) + 1e-6 * S
    assert np.all(errp <= 1e-6 * Sp + 1e-30), float((errp / Sp).max())
    big = np.abs(ref_d) > 1e-3
    if bf16 and big.sum() > 20000:  # stochastic rounding is unbiased: mean error ~ 0 spacings
        z = (dd - ref_d)[big] / _ulp_bf16(ref_d[big])
        assert abs(float(z.mean())) < 0.02, float(z.mean())


@pytest.mark.parametrize("storage", [seisgb.FP32_DIFF, seisgb.BF16_DIFF], ids=["fp32", "bf16"])
def test_run_shot_equals_stencil_step_diff_loop(storage):
    """run_shot in difference form (graph replays of 32 steps and direct
    launches) equals a loop of stencil_step_diff calls with the same buffers'
    roles, receivers sampling u^{n+1} after each step: traces and final
    wavefield bit for bit (bf16 included: the random bits depend only on the
    point and the step)."""
    nx, ny, nz, nb, nt = 61, 30, 27, 6, 70
    shape = (nz + 2 * nb, ny + 2 * nb, nx + 2 * nb)
    vel = synth.layered_model(shape, seed=12, sigma=2.0)
    vmax = float(vel.max())
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, 10.0, 10.0, 10.0)))
    g = seisgb.make_grid(nx, ny, nz, nb, 10.0, 10.0, 10.0, dt, vmax, storage=storage)
    wav = synth.ricker(nt, dt, 25.0)
    src = (nb + 30, nb + 15, nb + 13)
    rec = synth.surface_receivers(nx, ny, nb, 4).astype(np.int32)
    rec[:, 2] = src[2]
    d_v, d_w = torch.from_numpy(vel).cuda(), torch.from_numpy(wav).cuda()
    tr = torch.zeros((nt, rec.shape[0]), dtype=torch.float32, device="cuda")
    u = torch.zeros(g.shape, dtype=torch.float32, device="cuda")
    seisgb.run_shot(g, d_v, d_w, nt, src, rec, tr, u)

    wdt = torch.bfloat16 if storage == seisgb.BF16_DIFF else torch.float32
    bufs = [padded_zeros(g).to(wdt) for _ in range(3)]  # u^{n}, u^{n+1} alternate; d in place
    d_m = to_padded(g, (vel.astype(np.float32) * np.float32(g.dt)) ** 2)  # as run_shot forms m
    d_ph = padded_zeros(g)
    tr2 = torch.zeros_like(tr)
    for n in range(nt):
        seisgb.stencil_step_diff(g, bufs[n & 1], bufs[(n + 1) & 1], bufs[2], d_m, d_ph, n,
                                 source=(*src, d_w), receivers=(rec, tr2[n]))
    seisgb.device_status()
    u2 = from_padded(g, bufs[nt & 1].float())
    assert float(tr.abs().max()) > 0
    assert torch.equal(tr, tr2)
    assert np.array_equal(u.cpu().numpy(), u2)
