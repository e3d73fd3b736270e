"""16-bit wavefield storage (fp16 with a per-field power-of-two scale, bf16,
and the difference-form state u^n, u^n - u^{n-1}) with fp32 arithmetic: error
against the fp64 oracle, stated per format."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_04619_gb300 import seisgb, synth
from gpu_util import ensure_lib, rel_l2

pytestmark = pytest.mark.gpu

FORMATS = {"fp32": seisgb.FP32, "fp16": seisgb.FP16_SCALED, "bf16": seisgb.BF16}


def _source_plane_receivers(w, every=4):
    """Receivers on the horizontal plane through the source, so that they record
    the direct wave within a short run."""
    rec = synth.surface_receivers(w.nx, w.ny, w.nb, every)
    rec[:, 2] = w.source()[2]
    return rec


def _run(w, vel, storage, nt, rec=None):
    vmax = float(vel.max())
    dt = float(np.float32(w.cfl_fraction * oracle.cfl_dt(vmax, w.h, w.h, w.h)))
    g = seisgb.make_grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax, storage=storage)
    wav = synth.ricker(nt, dt, w.fp)
    rec = w.receivers() if rec is None else rec
    tr = torch.zeros((nt, rec.shape[0]), dtype=torch.float32, device="cuda")
    u = torch.zeros(g.shape, dtype=torch.float32, device="cuda")
    seisgb.run_shot(g, torch.from_numpy(vel).cuda(), torch.from_numpy(wav).cuda(), nt,
                    w.source(), rec, tr, u)
    return tr.cpu().numpy(), u.cpu().numpy(), dt, wav, rec


def _oracle(w, vel, dt, wav, rec, nt):
    go = oracle.Grid(w.nx, w.ny, w.nz, w.nb, w.h, w.h, w.h, dt, vmax=float(vel.max()),
                     r0=float(np.float32(1e-3)))
    return oracle.run_shot(go, vel, wav, nt, w.source(), rec)


def test_small_case_error_per_format():
    """64^3 + PML 16, 100 steps, receivers on the source plane.  fp16 with scaling
    keeps 11 significant bits per stored value, bf16 8.  Measured when written
    (wavefield, traces): fp16 2.7e-3 / 1.1e-3, bf16 2.3e-2 / 1.5e-2; the bounds
    are about 3x those."""
    ensure_lib()
    w = synth.SMALL
    vel = w.velocity()
    errs = {}
    ref = None
    for name, fmt in FORMATS.items():
        tr, u, dt, wav, rec = _run(w, vel, fmt, w.nt, _source_plane_receivers(w))
        if ref is None:
            ref = _oracle(w, vel, dt, wav, rec, w.nt)
        errs[name] = (rel_l2(u, ref["u"]), rel_l2(tr, ref["traces"]))
    print("small case rel L2 (wavefield, traces):", errs)
    assert errs["fp32"][0] <= 2e-5 and errs["fp32"][1] <= 2e-5
    assert errs["fp16"][0] <= 1e-2 and errs["fp16"][1] <= 1e-2
    assert errs["bf16"][0] <= 8e-2 and errs["bf16"][1] <= 8e-2
    assert errs["fp16"][0] < errs["bf16"][0]


def test_difference_form_small_case():
    """The difference-form formats (state u^n, d^n = u^n - u^{n-1}) on the small
    case, 64^3 + PML 16, 100 steps, receivers on the source plane.  In fp32 the
    form is the same scheme as the leapfrog up to rounding, so it meets the
    fp32 bound (2e-5) against the oracle, PML included (measured 2.7e-6 /
    5.2e-7).  In bf16 a stored rounding error of u no longer enters the time
    difference: measured 1.0e-2 / 5.4e-3 against 2.4e-2 / 1.1e-2 for the bf16
    leapfrog state; scaled fp16 in difference form 1.1e-3 / 4.6e-4 against 2.8e-3 /
    9.8e-4 for the fp16 leapfrog state.  The bounds are about 3x the measured
    errors."""
    ensure_lib()
    w = synth.SMALL
    vel = w.velocity()
    rec = _source_plane_receivers(w)
    errs = {}
    ref = None
    for name, fmt in (("fp32_diff", seisgb.FP32_DIFF), ("bf16_diff", seisgb.BF16_DIFF),
                      ("bf16", seisgb.BF16), ("fp16_diff", seisgb.FP16_DIFF)):
        tr, u, dt, wav, rec = _run(w, vel, fmt, w.nt, rec)
        if ref is None:
            ref = _oracle(w, vel, dt, wav, rec, w.nt)
        assert np.abs(tr).max() > 0
        errs[name] = (rel_l2(u, ref["u"]), rel_l2(tr, ref["traces"]))
    print("difference form, small case rel L2 (wavefield, traces):", errs)
    assert errs["fp32_diff"][0] <= 2e-5 and errs["fp32_diff"][1] <= 2e-5
    assert errs["bf16_diff"][0] <= 3e-2 and errs["bf16_diff"][1] <= 1.6e-2
    assert errs["bf16_diff"][0] < 0.7 * errs["bf16"][0]
    assert errs["fp16_diff"][0] <= 3.5e-3 and errs["fp16_diff"][1] <= 1.5e-3


def test_fp32_difference_form_ragged_layered_vs_oracle():
    """FP32_DIFF on a ragged anisotropic layered grid (several tiles, PML 7,
    source near a PML corner, receivers spread over the depth) against the fp64
    oracle: the fp32 bound of the leapfrog path (2e-5 relative L2)."""
    ensure_lib()
    nx, ny, nz, nb, nt = 101, 45, 38, 7, 90
    shape = (nz + 2 * nb, ny + 2 * nb, nx + 2 * nb)
    vel = synth.layered_model(shape, seed=33, sigma=2.0)
    vmax = float(vel.max())
    h = (10.0, 12.0, 9.0)
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, *h)))
    wav = synth.ricker(nt, dt, 25.0)
    src = (nb + 3, nb + ny - 4, nb + 5)
    rng = np.random.default_rng(5)
    rec = synth.surface_receivers(nx, ny, nb, 5)
    rec[:, 2] = nb + rng.integers(0, nz, rec.shape[0])
    rec = rec.astype(np.int32)
    g = seisgb.make_grid(nx, ny, nz, nb, *h, dt, vmax, storage=seisgb.FP32_DIFF)
    tr = torch.zeros((nt, rec.shape[0]), dtype=torch.float32, device="cuda")
    u = torch.zeros(g.shape, dtype=torch.float32, device="cuda")
    seisgb.run_shot(g, torch.from_numpy(vel).cuda(), torch.from_numpy(wav).cuda(), nt, src, rec,
                    tr, u)
    go = oracle.Grid(nx, ny, nz, nb, *h, dt, vmax=vmax, r0=float(np.float32(1e-3)))
    ref = oracle.run_shot(go, vel, wav, nt, src, rec)
    assert np.abs(ref["traces"]).max() > 0
    assert rel_l2(u.cpu().numpy(), ref["u"]) <= 2e-5
    assert rel_l2(tr.cpu().numpy(), ref["traces"]) <= 2e-5


@pytest.mark.slow
def test_256_cube_1000_steps_error_per_format():
    """The reduced-precision error check on the layered model at 256^3 computed
    (192^3 inner + 32-point PML), 1000 steps, against the fp64 oracle.  Measured
    when written (wavefield, traces): fp32 1.8e-4 / 9.9e-5, fp16 2.2e-2 / 1.3e-2,
    bf16 1.8e-1 / 1.1e-1 (stochastic rounding; with round-to-nearest fp16 was
    1.4e-1 / 6.9e-2 and bf16 diverged).  fp32 error grows with the step count:
    2.7e-6 after 100 steps of the small case, 1.8e-4 after 1000 here.  The
    difference form brings bf16 below 1e-1: measured 5.1e-2 / 2.6e-2
    (BF16_DIFF), and 1.1e-4 / 2.8e-5 for FP32_DIFF; scaled fp16 in difference form
    6.4e-3 / 3.1e-3 (FP16_DIFF) against 2.2e-2 / 1.3e-2."""
    ensure_lib()
    w = synth.scaled(synth.LARGE, 192, 32, 1000, name="fwd256_pml32_layered_ricker10_nt1000")
    vel = w.velocity()
    errs = {}
    ref = None
    formats = dict(FORMATS, fp32_diff=seisgb.FP32_DIFF, bf16_diff=seisgb.BF16_DIFF,
                   fp16_diff=seisgb.FP16_DIFF)
    for name, fmt in formats.items():
        tr, u, dt, wav, rec = _run(w, vel, fmt, w.nt)
        if ref is None:
            ref = _oracle(w, vel, dt, wav, rec, w.nt)
        errs[name] = (rel_l2(u, ref["u"]), rel_l2(tr, ref["traces"]))
    print("256^3 x 1000 rel L2 (wavefield, traces):", errs)
    assert errs["fp32"][0] <= 5e-4 and errs["fp32"][1] <= 5e-4
    assert errs["fp16"][0] <= 5e-2 and errs["fp16"][1] <= 4e-2
    assert errs["bf16"][0] <= 4e-1 and errs["bf16"][1] <= 3e-1
    assert errs["fp32_diff"][0] <= 5e-4 and errs["fp32_diff"][1] <= 5e-4
    assert errs["bf16_diff"][0] <= 1e-1 and errs["bf16_diff"][1] <= 8e-2
    assert errs["fp16_diff"][0] <= 2e-2 and errs["fp16_diff"][1] <= 1e-2


# Stored mantissa bits of the 16-bit formats: fp16 keeps 10, bf16 7.
MANT = {"fp16": 10, "bf16": 7}
TORCH16 = {"fp16": torch.float16, "bf16": torch.bfloat16}


def _padded16(g, stored, fmt):
    """Padded device field of 16-bit values from compact fp32 values that are
    already representable in the format (the conversion is exact)."""
    from gpu_util import to_padded
    return to_padded(g, stored).to(TORCH16[fmt])


def _ulp16(x, p):
    """Spacing of the 16-bit grid around |x| (normal range)."""
    ax = np.maximum(np.abs(x), 1e-30)
    return np.exp2(np.floor(np.log2(ax)) - p)


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_stencil_step_16bit_single_step_vs_oracle(fmt):
    """One step of stencil_step on 16-bit fields from random inputs (ragged grid
    over several tiles, anisotropic spacing, PML), against oracle.step.  The fp32
    evaluation has error <= 1e-6 S (S = sum of |terms|, the fp32 bound of the
    other parity tests); stochastic rounding then picks one of the two 16-bit
    neighbours of the fp32 value, within one spacing 2^-p |x| of it (p = 10 for
    fp16, 7 for bf16).  The rounding must also be unbiased: the mean signed error
    in units of the spacing is ~0."""
    from gpu_util import abs_term_sum, from_padded, to_padded
    ensure_lib()
    nx, ny, nz, nb, h = 90, 37, 29, 5, (10.0, 11.0, 12.0)
    vmax = 3000.0
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, *h)))
    storage = FORMATS[fmt]
    g = seisgb.make_grid(nx, ny, nz, nb, *h, dt, vmax, 1e-3, storage)
    g32 = seisgb.make_grid(nx, ny, nz, nb, *h, dt, vmax, 1e-3)
    go = oracle.Grid(nx, ny, nz, nb, *h, dt, vmax=vmax, r0=float(np.float32(1e-3)))
    rng = np.random.default_rng(16 + len(fmt))
    sh = g.shape
    q = lambda a: torch.from_numpy(a.astype(np.float32)).to(TORCH16[fmt]).float().numpy()
    st_c, st_p = q(rng.standard_normal(sh)), q(rng.standard_normal(sh))
    s_c, s_p = (2.0 ** -3, 2.0 ** -2) if fmt == "fp16" else (1.0, 1.0)
    uc, up = st_c * np.float32(s_c), st_p * np.float32(s_p)
    ph = (0.1 * rng.standard_normal(sh)).astype(np.float32)
    Nz, Ny, Nx = sh
    K, J, I = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    inner = ((I >= nb) & (I < nb + nx) & (J >= nb) & (J < nb + ny) & (K >= nb) & (K < nb + nz))
    ph[inner] = 0.0
    vel = rng.uniform(1500, 3000, sh).astype(np.float32)
    m = (vel.astype(np.float64) ** 2 * dt ** 2).astype(np.float32)
    src = (nb + nx // 2, nb + ny // 2, nb + nz // 2)
    wav = np.linspace(-1, 1, 8).astype(np.float32)
    step = 5

    d_uc, d_up = _padded16(g, st_c, fmt), _padded16(g, st_p, fmt)
    d_m, d_ph = to_padded(g, m), to_padded(g, ph)
    d_w = torch.from_numpy(wav).cuda()
    scale = torch.tensor([1.0] * 4 + [0.0] * 4, dtype=torch.float32, device="cuda")
    scale[step & 3], scale[(step - 1) & 3] = s_c, s_p
    scale[4 + (step & 3)] = float(np.abs(uc).max())
    scale[4 + ((step - 1) & 3)] = float(np.abs(up).max())
    seisgb.stencil_step(g, d_uc, d_up, d_m, d_ph, step, source=(*src, d_w),
                        scale_state=scale if fmt == "fp16" else None)
    seisgb.device_status()
    s_n = float(scale[(step + 1) & 3]) if fmt == "fp16" else 1.0
    un = from_padded(g32, d_up.float()) * np.float32(s_n)
    pn = from_padded(g32, d_ph)

    ref_u, ref_p = oracle.step(go, m, up, uc, ph)
    inv_vol = 1.0 / (go.dx * go.dy * go.dz)
    ref_u[src[2], src[1], src[0]] += float(m[src[2], src[1], src[0]]) * float(wav[step]) * inv_vol
    S = abs_term_sum(go, m, up, uc, ph)
    S[src[2], src[1], src[0]] += abs(float(m[src[2], src[1], src[0]]) * float(wav[step]) * inv_vol)
    p = MANT[fmt]
    err = np.abs(un - ref_u)
    bound = 1.01e-6 * S + 2.0 ** -p * (np.abs(ref_u) + 1e-6 * S) + 1e-30
    if fmt == "fp16":
        bound += 2.0 ** -24 * s_n  # subnormal spacing of the scaled grid
        assert s_n == 2.0 ** np.round(np.log2(s_n))  # a power of two
        assert np.abs(un).max() / s_n < 65504.0  # no stored value overflowed
    assert np.all(err <= bound), float((err / bound).max())
    # unbiased rounding: mean signed error ~ 0 in units of the 16-bit spacing
    big = np.abs(ref_u) > 1e3 * 1e-6 * S
    d = ((un - ref_u) / _ulp16(ref_u, p))[big]
    assert d.size > 10000 and abs(float(d.mean())) < 0.02, float(d.mean())
    assert float(np.abs(d).mean()) > 0.2  # the values really were rounded to 16 bits
    errp = np.abs(pn - ref_p)
    Sp = np.abs(ph) + np.abs(ref_p) + 1e-6 * S
    assert np.all(errp <= 1e-6 * Sp + 1e-30), float((errp / Sp).max())


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_run_shot_16bit_equals_stencil_step_loop(fmt):
    """run_shot with 16-bit storage (CUDA-graph replays) gives bit-identical
    traces and wavefield to a loop of stencil_step calls on 16-bit fields (the
    fp16 scale state starting from unit scales and zero maxima)."""
    from gpu_util import from_padded, to_padded
    ensure_lib()
    nx, nb, nt = 20, 6, 70
    vmax = 2500.0
    dt = float(np.float32(0.4 * oracle.cfl_dt(vmax, 10.0, 10.0, 10.0)))
    g = seisgb.make_grid(nx, nx + 3, nx - 2, nb, 10.0, 10.0, 10.0, dt, vmax, 1e-3, FORMATS[fmt])
    g32 = seisgb.make_grid(nx, nx + 3, nx - 2, nb, 10.0, 10.0, 10.0, dt, vmax)
    rng = np.random.default_rng(1)
    vel = rng.uniform(1500, 2500, g.shape).astype(np.float32)
    wav = synth.ricker(nt, dt, 20.0)
    src = (nb + 5, nb + 7, nb + 3)
    rec = np.array([[nb, nb, nb], [nb + 3, nb + 9, nb + 2], [nb + nx - 1, nb + 1, nb + 4]], np.int32)
    tr = torch.zeros((nt, 3), dtype=torch.float32, device="cuda")
    u = torch.zeros(g.shape, dtype=torch.float32, device="cuda")
    d_v, d_w = torch.from_numpy(vel).cuda(), torch.from_numpy(wav).cuda()
    seisgb.run_shot(g, d_v, d_w, nt, src, rec, tr, u)

    m = (vel * np.float32(dt)) ** 2
    d_m = to_padded(g32, m)
    L = seisgb.layout(g)
    a, b = (torch.zeros(int(L.elems), dtype=TORCH16[fmt], device="cuda") for _ in range(2))
    ph = torch.zeros(int(L.elems), dtype=torch.float32, device="cuda")
    scale = torch.tensor([1.0] * 4 + [0.0] * 4, dtype=torch.float32, device="cuda")
    tr2 = torch.zeros((nt, 3), dtype=torch.float32, device="cuda")
    cur, prev = a, b
    for n in range(nt):
        seisgb.stencil_step(g, cur, prev, d_m, ph, n, source=(*src, d_w), receivers=(rec, tr2[n]),
                            scale_state=scale if fmt == "fp16" else None)
        cur, prev = prev, cur
    s_final = float(scale[nt & 3]) if fmt == "fp16" else 1.0
    u2 = from_padded(g32, cur.float()) * np.float32(s_final)
    assert np.array_equal(tr.cpu().numpy(), tr2.cpu().numpy())
    assert np.array_equal(u.cpu().numpy(), u2)
