"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol its header declares; host-side validation and layout work on CPU."""
import ctypes
import glob
import math
import os
import re

import numpy as np
import pytest

from paper_2009_04619_gb300 import build, seisgb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for stmt in src.split(";"):
            stmt = " ".join(stmt.split())
            if not stmt or stmt.startswith("typedef") or "#" in stmt.split("(")[0]:
                continue
            m = re.search(r"(\w+)\s*\([^()]*(\([^()]*\)[^()]*)*\)\s*$", stmt)
            if m and "{" not in stmt:
                names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return seisgb.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("stencil_step", "run_shot", "sgb_layout", "sgb_cfl_dt", "sgb_last_error"):
        assert n in names, names


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps exactly the declared functions
    assert set(seisgb.SIGNATURES) == names


def test_layout_geometry(lib):
    g = seisgb.make_grid(13, 17, 11, 5, 10, 11, 12, 1e-3, 3000)
    L = seisgb.layout(g)
    assert (L.Nx, L.Ny, L.Nz) == (23, 27, 21)
    assert L.halo_lo_x == 8 and L.halo == 4
    assert L.sx % 32 == 0 and L.sx >= 8 + 23 + 4
    assert (L.sy, L.sz) == (27 + 8, 21 + 8)
    assert L.stride_z == L.sx * L.sy
    assert L.origin == 4 * L.stride_z + 4 * L.sx + 8
    assert L.elems == L.sx * L.sy * L.sz
    assert (L.origin * 4) % 16 == 0 and (L.sx * 4) % 16 == 0


def test_cfl_dt_closed_form(lib):
    g = seisgb.make_grid(8, 8, 8, 2, 10, 7, 12, 1e-3, 3000)
    got = seisgb.cfl_dt(g, 4500.0)
    want = 2.0 / (4500.0 * math.sqrt(2048 / 315 * (10 ** -2 + 7 ** -2 + 12 ** -2)))
    assert math.isclose(got, want, rel_tol=1e-6)


@pytest.mark.parametrize("field,value", [("nx", 0), ("nb", -1), ("dx", 0.0), ("dt", -1.0),
                                         ("pml_r0", 0.0), ("pml_r0", 1.5), ("storage", 7),
                                         ("vmax", float("nan")), ("schedule", 4),
                                         ("schedule", -1)])
def test_bad_grid_rejected_without_gpu(lib, field, value):
    g = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000)
    setattr(g, field, value)
    with pytest.raises(seisgb.SeisgbError) as e:
        seisgb.layout(g)
    assert e.value.code == seisgb.ERR_INVALID_ARG


def test_step_argument_checks_precede_any_gpu_work(lib):
    """Invalid calls return their code from host-side validation alone (these run
    on a machine without a GPU)."""
    g = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000)
    st = 0
    L = seisgb.lib()
    buf = (ctypes.c_float * 64)()
    a = ctypes.addressof(buf)
    a16 = a + (16 - a % 16) % 16
    # NULL field
    assert L.stencil_step(ctypes.byref(g), None, a16, a16, a16, 0, None, None, st) == seisgb.ERR_INVALID_ARG
    # misaligned pointer
    assert L.stencil_step(ctypes.byref(g), a16 + 4, a16 + 16, a16, a16, 0, None, None, st) == seisgb.ERR_INVALID_ARG
    # aliasing u_cur and u_prev_to_next
    assert L.stencil_step(ctypes.byref(g), a16, a16, a16, a16, 0, None, None, st) == seisgb.ERR_INVALID_ARG
    # phi required with a PML
    assert L.stencil_step(ctypes.byref(g), a16, a16 + 16, a16, None, 0, None, None, st) == seisgb.ERR_INVALID_ARG
    # source outside the inner region
    src = seisgb.Source(0, 0, 0, a16)
    assert L.stencil_step(ctypes.byref(g), a16, a16 + 16, a16, a16 + 32, 0, ctypes.byref(src), None, st) == seisgb.ERR_INVALID_ARG
    # dt above the CFL limit
    g2 = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1.0, 3000)
    assert L.stencil_step(ctypes.byref(g2), a16, a16 + 16, a16, a16 + 32, 0, None, None, st) == seisgb.ERR_UNSTABLE_DT
    assert "CFL" in seisgb.last_error()
    # negative step
    assert L.stencil_step(ctypes.byref(g), a16, a16 + 16, a16, a16 + 32, -1, None, None, st) == seisgb.ERR_INVALID_ARG


def test_run_shot_argument_checks_without_gpu(lib):
    g = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000)
    L = seisgb.lib()
    v = np.full(g.shape, 2000, np.float32)
    w = np.zeros(10, np.float32)
    src = np.array([0, 0, 0], np.int32)  # in the PML: rejected
    rc = L.run_shot(ctypes.byref(g), v.ctypes.data, w.ctypes.data, 10, src.ctypes.data, None, 0,
                    None, None, None)
    assert rc == seisgb.ERR_INVALID_ARG
    rec = np.array([[5, 5, 1]], np.int32)  # receiver in the PML
    tr = np.zeros(10, np.float32)
    src = np.array([5, 5, 5], np.int32)
    rc = L.run_shot(ctypes.byref(g), v.ctypes.data, w.ctypes.data, 10, src.ctypes.data,
                    rec.ctypes.data, 1, tr.ctypes.data, None, None)
    assert rc == seisgb.ERR_INVALID_ARG
    rc = L.run_shot(ctypes.byref(g), v.ctypes.data, w.ctypes.data, -1, src.ctypes.data, None, 0,
                    None, None, None)
    assert rc == seisgb.ERR_INVALID_ARG


@pytest.mark.parametrize("entry", ["run_shot", "run_shot_noalloc"])
def test_outputs_overlapping_inputs_rejected_without_gpu(lib, entry):
    """traces and final_u may overlap neither velocity, wavelet nor each other
    (checked before any GPU work, for both shot entry points)."""
    g = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000)
    f = getattr(seisgb.lib(), entry)
    N = int(np.prod(g.shape))
    nt = 10
    big = np.zeros(4 * N, np.float32)
    v = big[:N]
    v[:] = 2000.0
    w = np.zeros(nt, np.float32)
    src = np.array([5, 5, 5], np.int32)
    rec = np.array([[5, 5, 2]], np.int32)
    tr = np.zeros(nt, np.float32)
    base = big.ctypes.data

    def call(tr_ptr, u_ptr, w_ptr=w.ctypes.data):
        rc = f(ctypes.byref(g), base, w_ptr, nt, src.ctypes.data, rec.ctypes.data, 1, tr_ptr, u_ptr,
               None)
        return rc, seisgb.last_error()

    rc, msg = call(tr.ctypes.data, base + 4 * (N // 2))  # final_u inside velocity
    assert rc == seisgb.ERR_INVALID_ARG and "final_u overlaps velocity" in msg
    rc, msg = call(base + 4 * (N - 1), None)  # traces start on velocity's last element
    assert rc == seisgb.ERR_INVALID_ARG and "traces overlaps velocity" in msg
    rc, msg = call(base + 4 * (2 * N), base + 4 * (2 * N + 5))  # traces inside final_u
    assert rc == seisgb.ERR_INVALID_ARG and "overlaps" in msg
    rc, msg = call(base + 4 * N, None, w_ptr=base + 4 * N + 8)  # traces over the wavelet
    assert rc == seisgb.ERR_INVALID_ARG and "traces overlaps wavelet" in msg


def test_serve_footprint_arithmetic(lib):
    """Four padded fp32 fields + velocity upload + wavelet + receiver table + traces."""
    g = seisgb.make_grid(20, 24, 16, 6, 10, 10, 10, 1e-3, 3000)
    L = seisgb.layout(g)
    nt, nrec = 300, 17
    Nz, Ny, Nx = g.shape
    want = 4 * L.elems * 4 + Nz * Ny * Nx * 4 + nt * 4 + nrec * 8 + nt * nrec * 4
    assert seisgb.serve_footprint(g, nt, nrec) == want
    with pytest.raises(seisgb.SeisgbError):
        seisgb.serve_footprint(g, 0, nrec)


@pytest.mark.parametrize("budget,slots,steps", [(0, 4, 16), (1 << 30, 0, 16), (1 << 30, 65, 16),
                                                (1 << 30, 4, 0), (1 << 30, 4, 257)])
def test_serve_config_rejected_without_gpu(lib, budget, slots, steps):
    cfg = seisgb.ServeConfig(budget, slots, steps)
    h = ctypes.c_void_p()
    assert seisgb.lib().serve_create(ctypes.byref(cfg), ctypes.byref(h)) == seisgb.ERR_INVALID_ARG


@pytest.mark.parametrize("limit_us", [0, -5, 2000001])
def test_wait_selftest_arguments_checked_without_gpu(lib, limit_us):
    st = ctypes.c_int32(7)
    assert lib.sgb_selftest_wait_timeout(limit_us, ctypes.byref(st), None) == seisgb.ERR_INVALID_ARG
    assert st.value == 7
    assert lib.sgb_selftest_wait_timeout(1000, None, None) == seisgb.ERR_INVALID_ARG


def test_binding_checks_buffers_before_the_c_call(lib):
    """Element type, contiguity, size and (for device-only calls) residency are
    checked in Python: the C ABI takes plain pointers and cannot."""
    g = seisgb.make_grid(8, 8, 8, 2, 10.0, 10.0, 10.0, 1e-3, 2000.0)
    N = int(np.prod(g.shape))
    nt, rec = 4, np.array([[4, 4, 2]], dtype=np.int32)
    v = np.full(g.shape, 2000.0, dtype=np.float32)
    w = np.zeros(nt, dtype=np.float32)
    tr = np.zeros((nt, 1), dtype=np.float32)
    with pytest.raises(ValueError, match="float32"):
        seisgb.run_shot(g, v.astype(np.float64), w, nt, (4, 4, 4), rec, tr)
    with pytest.raises(ValueError, match="at least"):
        seisgb.run_shot(g, v.ravel()[:N - 1], w, nt, (4, 4, 4), rec, tr)
    with pytest.raises(ValueError, match="contiguous"):
        seisgb.run_shot(g, np.asfortranarray(v), w, nt, (4, 4, 4), rec, tr)
    with pytest.raises(ValueError, match="at least"):
        seisgb.run_shot(g, v, w[:2], nt, (4, 4, 4), rec, tr)
    with pytest.raises(ValueError, match="at least"):
        seisgb.run_shot(g, v, w, nt, (4, 4, 4), rec, tr[:2])
    with pytest.raises(ValueError, match="float64"):
        seisgb.adjoint_shot(g, v, w, nt, (4, 4, 4), rec, tr, np.zeros(g.shape, np.float32))
    E = int(seisgb.layout(g).elems)
    f = np.zeros(E, dtype=np.float32)
    with pytest.raises(ValueError, match="CUDA"):
        seisgb.stencil_step(g, f, f.copy(), f.copy(), f.copy(), 0)
    with pytest.raises(ValueError, match="CUDA"):
        seisgb.pack(g, v, f)


def test_schedules_check_storage(lib):
    """Temporal blocking needs fp32 fields; the dataflow schedule has no per-step
    fp16 scale (fp32 and bf16 only)."""
    for storage, sched in ((seisgb.BF16, seisgb.SCHED_PAIRS), (seisgb.FP16_SCALED, seisgb.SCHED_PAIRS),
                           (seisgb.FP16_SCALED, seisgb.SCHED_FLOW)):
        g = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000, storage=storage, schedule=sched)
        with pytest.raises(seisgb.SeisgbError) as e:
            seisgb.layout(g)
        assert e.value.code == seisgb.ERR_INVALID_ARG and "SCHED" in str(e.value)
    g = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000, storage=seisgb.BF16,
                         schedule=seisgb.SCHED_FLOW)
    seisgb.layout(g)


def test_difference_form_storage_checks(lib):
    """The difference-form formats run through run_shot with one launch per
    step and through stencil_step_diff: the other schedules, stencil_step,
    segments, the allocation-free entry point and the server reject them, and
    stencil_step_diff rejects other formats and aliased or misaligned fields,
    all before any GPU work; unknown storage codes are rejected."""
    L = seisgb.lib()
    for storage in (seisgb.FP32_DIFF, seisgb.BF16_DIFF):
        for sched in (seisgb.SCHED_AUTO, seisgb.SCHED_STEP):
            seisgb.layout(seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000, storage=storage,
                                           schedule=sched))
        for sched in (seisgb.SCHED_PAIRS, seisgb.SCHED_FLOW):
            g = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000, storage=storage, schedule=sched)
            with pytest.raises(seisgb.SeisgbError) as e:
                seisgb.layout(g)
            assert e.value.code == seisgb.ERR_INVALID_ARG and "SCHED" in str(e.value)
        g = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000, storage=storage)
        E = int(seisgb.layout(g).elems)
        buf = np.zeros(5 * E + 16, np.float32)
        b = buf.ctypes.data + (16 - buf.ctypes.data % 16) % 16
        fld = [b + 4 * E * q for q in range(4)]
        assert L.stencil_step(ctypes.byref(g), fld[0], fld[1], fld[2], fld[3], 0, None, None,
                              None) == seisgb.ERR_INVALID_ARG
        assert "stencil_step_diff" in seisgb.last_error()
        sd = lambda u, un, d, gg=g: L.stencil_step_diff(ctypes.byref(gg), u, un, d, fld[3], fld[3],
                                                        0, None, None, None)
        assert sd(fld[0], fld[1], None) == seisgb.ERR_INVALID_ARG      # no d
        assert sd(fld[0], fld[1], fld[0]) == seisgb.ERR_INVALID_ARG    # d = u_cur
        assert sd(fld[0], fld[1], fld[1]) == seisgb.ERR_INVALID_ARG    # d = u_next
        assert sd(fld[0], fld[0], fld[2]) == seisgb.ERR_INVALID_ARG    # u_next = u_cur
        assert sd(fld[0], fld[1], fld[2] + 4) == seisgb.ERR_INVALID_ARG  # misaligned d
        g_plain = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000)
        assert sd(fld[0], fld[1], fld[2], g_plain) == seisgb.ERR_INVALID_ARG
        assert "SGB_FP32_DIFF or SGB_BF16_DIFF" in seisgb.last_error()
        N = int(np.prod(g.shape))
        v = np.full(g.shape, 2000, np.float32)
        w = np.zeros(10, np.float32)
        src = np.array([5, 5, 5], np.int32)
        st = [np.zeros(N, np.float32) for _ in range(3)]
        assert L.run_shot_segment(ctypes.byref(g), v.ctypes.data, w.ctypes.data, 0, 4,
                                  src.ctypes.data, None, 0, None, *[x.ctypes.data for x in st],
                                  None) == seisgb.ERR_INVALID_ARG
        assert "segments need SGB_FP32 or SGB_BF16" in seisgb.last_error()
    g = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000, storage=seisgb.FP16_DIFF)
    seisgb.layout(g)
    E = int(seisgb.layout(g).elems)
    buf = np.zeros(5 * E + 16, np.float32)
    b = buf.ctypes.data + (16 - buf.ctypes.data % 16) % 16
    fld = [b + 4 * E * q for q in range(4)]
    assert L.stencil_step_diff(ctypes.byref(g), fld[0], fld[1], fld[2], fld[3], fld[3], 0, None,
                               None, None) == seisgb.ERR_INVALID_ARG
    assert "run_shot only" in seisgb.last_error()
    for sched in (seisgb.SCHED_PAIRS, seisgb.SCHED_FLOW):
        with pytest.raises(seisgb.SeisgbError):
            seisgb.layout(seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000,
                                           storage=seisgb.FP16_DIFF, schedule=sched))
    for bad in (-1, 6):
        g = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000, storage=bad)
        with pytest.raises(seisgb.SeisgbError):
            seisgb.layout(g)


def test_step2_argument_checks_without_gpu(lib):
    """stencil_step2 validates before any GPU work: four distinct aligned
    buffers, fp32 storage, phi with a PML, the CFL limit."""
    g = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000)
    E = int(seisgb.layout(g).elems)
    buf = np.zeros(7 * E + 16, np.float32)
    b = buf.ctypes.data + (16 - buf.ctypes.data % 16) % 16
    fld = [b + 4 * E * q for q in range(6)]
    L = seisgb.lib()
    f = lambda *a: L.stencil_step2(ctypes.byref(g), *a, 0, None, None)
    assert f(fld[0], fld[1], fld[1], fld[3], fld[4], fld[5]) == seisgb.ERR_INVALID_ARG  # out = in
    assert "overlaps" in seisgb.last_error()
    assert f(fld[0], fld[1], fld[2], fld[2], fld[4], fld[5]) == seisgb.ERR_INVALID_ARG  # outs equal
    assert f(fld[0], fld[1], fld[2], fld[3], fld[4], None) == seisgb.ERR_INVALID_ARG    # no phi
    assert f(fld[0] + 4, fld[1], fld[2], fld[3], fld[4], fld[5]) == seisgb.ERR_INVALID_ARG
    g16 = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000, storage=seisgb.BF16)
    assert L.stencil_step2(ctypes.byref(g16), *fld, 0, None, None) == seisgb.ERR_INVALID_ARG
    g2 = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1.0, 3000)
    assert L.stencil_step2(ctypes.byref(g2), *fld, 0, None, None) == seisgb.ERR_UNSTABLE_DT


def test_segment_argument_checks_without_gpu(lib):
    """run_shot_segment validates before any GPU work: 0 <= n_begin <= n_end,
    three state arrays, no fp16-scaled storage, no overlap of the state with
    the inputs."""
    g = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000)
    L = seisgb.lib()
    N = int(np.prod(g.shape))
    v = np.full(g.shape, 2000, np.float32)
    w = np.zeros(10, np.float32)
    src = np.array([5, 5, 5], np.int32)
    st = [np.zeros(N, np.float32) for _ in range(3)]
    f = lambda gg, a, b, s0, s1, s2, vel=v: L.run_shot_segment(
        ctypes.byref(gg), vel.ctypes.data, w.ctypes.data, a, b, src.ctypes.data, None, 0, None,
        s0, s1, s2, None)
    p = [x.ctypes.data for x in st]
    assert f(g, 5, 4, *p) == seisgb.ERR_INVALID_ARG
    assert f(g, -1, 4, *p) == seisgb.ERR_INVALID_ARG
    assert f(g, 0, 4, p[0], None, p[2]) == seisgb.ERR_INVALID_ARG
    assert f(g, 0, 4, p[0], p[0], p[2]) == seisgb.ERR_INVALID_ARG  # state arrays overlap
    assert "overlaps" in seisgb.last_error()
    assert f(g, 0, 4, v.ctypes.data, p[1], p[2]) == seisgb.ERR_INVALID_ARG  # state over velocity
    g16 = seisgb.make_grid(8, 8, 8, 2, 10, 10, 10, 1e-3, 3000, storage=seisgb.FP16_SCALED)
    assert f(g16, 0, 4, *p) == seisgb.ERR_INVALID_ARG
    assert "segments need SGB_FP32 or SGB_BF16" in seisgb.last_error()


def test_fault_hook_arguments(lib):
    assert lib.sgb_debug_fail_allocations(-1, 1) == seisgb.ERR_INVALID_ARG
    assert lib.sgb_debug_fail_allocations(0, -1) == seisgb.ERR_INVALID_ARG
    assert lib.sgb_debug_fail_allocations(3, 0) == seisgb.OK  # disarmed
