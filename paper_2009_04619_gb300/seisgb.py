"""Thin Python binding of ``libseisgb.so`` (the C ABI in ``include/seisgb.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Tensors are torch tensors (device memory and streams come from
PyTorch); host buffers may be numpy arrays or CPU tensors where the C entry
point accepts host pointers.  When the library is missing or fails to load
every call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libseisgb.so")

OK = 0
PENDING = 1
ERR_INVALID_ARG = -1
ERR_OUT_OF_MEMORY = -2
ERR_UNSTABLE_DT = -3
ERR_CUDA = -4
ERR_TIMEOUT = -5
ERR_NONFINITE = -6
ERR_REJECTED = -7
ERR_CANCELLED = -8

FP32 = 0
FP16_SCALED = 1
BF16 = 2
# difference form: the state (u^n, u^n - u^{n-1}) instead of (u^n, u^{n-1});
# a third wavefield: run_shot and stencil_step_diff
FP32_DIFF = 3
BF16_DIFF = 4
FP16_DIFF = 5  # scaled fp16 in difference form: run_shot only

# run_shot time-loop schedules (sgb_grid.schedule)
SCHED_AUTO = 0
SCHED_STEP = 1
SCHED_PAIRS = 2
SCHED_FLOW = 3


class SeisgbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"seisgb error {code}: {msg}")
        self.code = code


class Grid(ctypes.Structure):
    """``sgb_grid``: inner extents, PML width, spacing, dt, PML damping inputs,
    storage format."""
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("nb", ctypes.c_int32), ("dx", ctypes.c_float), ("dy", ctypes.c_float),
                ("dz", ctypes.c_float), ("dt", ctypes.c_float), ("vmax", ctypes.c_float),
                ("pml_r0", ctypes.c_float), ("storage", ctypes.c_int32),
                ("schedule", ctypes.c_int32)]

    @property
    def shape(self):
        """Computed domain as (Nz, Ny, Nx)."""
        return (self.nz + 2 * self.nb, self.ny + 2 * self.nb, self.nx + 2 * self.nb)


class LayoutInfo(ctypes.Structure):
    _fields_ = [("Nx", ctypes.c_int32), ("Ny", ctypes.c_int32), ("Nz", ctypes.c_int32),
                ("halo_lo_x", ctypes.c_int32), ("halo", ctypes.c_int32),
                ("sx", ctypes.c_int64), ("sy", ctypes.c_int64), ("sz", ctypes.c_int64),
                ("stride_y", ctypes.c_int64), ("stride_z", ctypes.c_int64),
                ("origin", ctypes.c_int64), ("elems", ctypes.c_int64)]


class Source(ctypes.Structure):
    _fields_ = [("i", ctypes.c_int32), ("j", ctypes.c_int32), ("k", ctypes.c_int32),
                ("wavelet", ctypes.c_void_p)]


class Receivers(ctypes.Structure):
    _fields_ = [("nrec", ctypes.c_int32), ("ijk", ctypes.c_void_p), ("traces", ctypes.c_void_p)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_slots", ctypes.c_int32),
                ("steps_per_graph", ctypes.c_int32)]


class ShotRequest(ctypes.Structure):
    _fields_ = [("grid", Grid), ("velocity", ctypes.c_void_p), ("wavelet", ctypes.c_void_p),
                ("nt", ctypes.c_int32), ("src_ijk", ctypes.c_int32 * 3),
                ("rec_ijk", ctypes.c_void_p), ("nrec", ctypes.c_int32)]


class ShotResult(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("nt", ctypes.c_int32),
                ("nrec", ctypes.c_int32), ("traces", ctypes.c_void_p),
                ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("resident", ctypes.c_int32),
                ("queued", ctypes.c_int32), ("graph_replays", ctypes.c_uint64),
                ("step_launches", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("setup_ms", ctypes.c_double), ("prepare_ms", ctypes.c_double),
                ("retire_ms", ctypes.c_double), ("wait_ms", ctypes.c_double),
                ("cancelled", ctypes.c_uint64)]


_lib = None

# name -> (restype, argtypes); every symbol declared in include/seisgb.h
SIGNATURES = {
    "sgb_layout": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(LayoutInfo)]),
    "sgb_cfl_dt": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_float,
                                  ctypes.POINTER(ctypes.c_float)]),
    "stencil_step": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                    ctypes.POINTER(Source), ctypes.POINTER(Receivers),
                                    ctypes.c_void_p]),
    "stencil_step_diff": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int32, ctypes.POINTER(Source),
                                         ctypes.POINTER(Receivers), ctypes.c_void_p]),
    "stencil_step_scaled": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int32, ctypes.POINTER(Source),
                                           ctypes.POINTER(Receivers), ctypes.c_void_p]),
    "stencil_step2": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(Source),
                                     ctypes.c_void_p]),
    "run_shot": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "run_shot_segment": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "adjoint_shot": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_double), ctypes.c_void_p,
                                    ctypes.c_void_p]),
    "run_shot_noalloc": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "sgb_pack": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p]),
    "sgb_unpack": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    "serve_footprint": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_int32, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_uint64)]),
    "serve_create": (ctypes.c_int, [ctypes.POINTER(ServeConfig), ctypes.POINTER(ctypes.c_void_p)]),
    "serve_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ShotRequest),
                                    ctypes.POINTER(ctypes.c_uint64)]),
    "serve_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ShotResult),
                                  ctypes.c_int32]),
    "serve_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServeStats)]),
    "serve_cancel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "sgb_debug_fail_allocations": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64]),
    "sgb_pool_used_bytes": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64)]),
    "serve_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "sgb_device_status": (ctypes.c_int, [ctypes.c_void_p]),
    "sgb_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                                 ctypes.c_void_p]),
    "sgb_launch_count": (ctypes.c_int64, [ctypes.c_int]),
    "sgb_last_error": (ctypes.c_char_p, []),
}


def lib():
    """Load ``libseisgb.so`` (raises if it is missing: build it with
    ``paper_2009_04619_gb300.build.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"seisgb CUDA library not built: {LIB_PATH} is missing "
                               "(run paper_2009_04619_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != OK:
        raise SeisgbError(rc, lib().sgb_last_error().decode())
    return rc


def make_grid(nx, ny, nz, nb, dx, dy, dz, dt, vmax, pml_r0=1e-3, storage=FP32,
              schedule=0) -> Grid:
    return Grid(int(nx), int(ny), int(nz), int(nb), float(dx), float(dy), float(dz), float(dt),
                float(vmax), float(pml_r0), int(storage), int(schedule))


def layout(g: Grid) -> LayoutInfo:
    out = LayoutInfo()
    _check(lib().sgb_layout(ctypes.byref(g), ctypes.byref(out)))
    return out


def cfl_dt(g: Grid, vmax: float) -> float:
    out = ctypes.c_float()
    _check(lib().sgb_cfl_dt(ctypes.byref(g), float(vmax), ctypes.byref(out)))
    return out.value


def _ptr(x):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _desc(x):
    """(dtype name, C-contiguous, element count, on a CUDA device) of a numpy
    array or torch tensor."""
    if isinstance(x, np.ndarray):
        return x.dtype.name, bool(x.flags.c_contiguous), int(x.size), False
    return (str(x.dtype).replace("torch.", ""), bool(x.is_contiguous()), int(x.numel()),
            bool(x.is_cuda))


def _buf(x, name: str, dtype: str, min_numel: int, optional: bool = False, cuda: bool = False):
    """Address of `x` after checking what the C side cannot: element type,
    C-contiguity, at least `min_numel` elements, and (cuda=True) that it lives
    on the GPU.  Raises ValueError otherwise."""
    if x is None:
        if optional:
            return None
        raise ValueError(f"{name} is required")
    dt, contiguous, numel, on_cuda = _desc(x)
    if dt != dtype:
        raise ValueError(f"{name}: expected {dtype} elements, got {dt}")
    if not contiguous:
        raise ValueError(f"{name} must be contiguous")
    if numel < min_numel:
        raise ValueError(f"{name}: {numel} elements, at least {min_numel} needed")
    if cuda and not on_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    return _ptr(x)


def _points(g: Grid) -> int:
    a, b, c = g.shape
    return a * b * c


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


_WAVE_DTYPE = {FP32: "float32", FP16_SCALED: "float16", BF16: "bfloat16",
               FP32_DIFF: "float32", BF16_DIFF: "bfloat16", FP16_DIFF: "float16"}


def stencil_step(g: Grid, u_cur, u_prev_to_next, m, phi, step: int = 0, source=None,
                 receivers=None, stream=None, scale_state=None):
    """One fused step.  Fields: CUDA tensors in the padded layout; u_cur and
    u_prev_to_next hold g.storage elements (float32, bfloat16, or float16 for
    FP16_SCALED, which also needs scale_state: a float32 CUDA tensor of 8 values,
    see stencil_step_scaled in the C header); m and phi are float32.
    source: (i, j, k, wavelet_cuda_tensor) or None.
    receivers: (ijk int32 numpy [nrec, 3], traces_row cuda tensor [nrec]) or None."""
    E = int(layout(g).elems)
    wdt = _WAVE_DTYPE.get(int(g.storage), "float32")
    src = None
    if source is not None:
        i, j, k, w = source
        src = Source(int(i), int(j), int(k), _buf(w, "wavelet", "float32", int(step) + 1, cuda=True))
    rec = None
    keep = None
    if receivers is not None:
        ijk, row = receivers
        keep = np.ascontiguousarray(np.asarray(ijk, dtype=np.int32).reshape(-1, 3))
        rec = Receivers(keep.shape[0], keep.ctypes.data,
                        _buf(row, "traces row", "float32", keep.shape[0], cuda=True))
    fields = [_buf(u_cur, "u_cur", wdt, E, cuda=True),
              _buf(u_prev_to_next, "u_prev_to_next", wdt, E, cuda=True),
              _buf(m, "m", "float32", E, cuda=True)]
    srcp = ctypes.byref(src) if src is not None else None
    recp = ctypes.byref(rec) if rec is not None else None
    php = _buf(phi, "phi", "float32", E, cuda=True)
    if int(g.storage) == FP16_SCALED:
        sc = _buf(scale_state, "scale_state", "float32", 8, cuda=True)
        rc = lib().stencil_step_scaled(ctypes.byref(g), *fields, php, sc, int(step), srcp, recp,
                                       _stream(stream))
    else:
        rc = lib().stencil_step(ctypes.byref(g), *fields, php, int(step), srcp, recp,
                                _stream(stream))
    del keep
    _check(rc)


def stencil_step_diff(g: Grid, u_cur, u_next, d, m, phi, step: int = 0, source=None,
                      receivers=None, stream=None):
    """One step in difference form (g.storage FP32_DIFF or BF16_DIFF): reads
    u_cur = u^n and d = u^n - u^{n-1}, writes u^{n+1} into u_next and d^{n+1}
    over d.  Fields: CUDA tensors in the padded layout (u_cur, u_next, d of
    g.storage elements; m, phi float32); source and receivers as for
    stencil_step."""
    E = int(layout(g).elems)
    wdt = _WAVE_DTYPE.get(int(g.storage), "float32")
    src = None
    if source is not None:
        i, j, k, w = source
        src = Source(int(i), int(j), int(k), _buf(w, "wavelet", "float32", int(step) + 1, cuda=True))
    rec = None
    keep = None
    if receivers is not None:
        ijk, row = receivers
        keep = np.ascontiguousarray(np.asarray(ijk, dtype=np.int32).reshape(-1, 3))
        rec = Receivers(keep.shape[0], keep.ctypes.data,
                        _buf(row, "traces row", "float32", keep.shape[0], cuda=True))
    fields = [_buf(u_cur, "u_cur", wdt, E, cuda=True), _buf(u_next, "u_next", wdt, E, cuda=True),
              _buf(d, "d", wdt, E, cuda=True), _buf(m, "m", "float32", E, cuda=True),
              _buf(phi, "phi", "float32", E, cuda=True)]
    rc = lib().stencil_step_diff(ctypes.byref(g), *fields, int(step),
                                 ctypes.byref(src) if src is not None else None,
                                 ctypes.byref(rec) if rec is not None else None, _stream(stream))
    del keep
    _check(rc)


def stencil_step2(g: Grid, u_prev, u_cur, u_next, u_next2, m, phi, step: int = 0, source=None,
                  stream=None):
    """Two steps with temporal blocking on the PML-free interior: reads u^{n-1}
    (u_prev) and u^n (u_cur), writes u^{n+1} (u_next) and u^{n+2} (u_next2);
    phi is updated in place.  fp32 CUDA tensors in the padded layout.
    source: (i, j, k, wavelet_cuda_tensor) or None (samples step and step + 1)."""
    E = int(layout(g).elems)
    src = None
    if source is not None:
        i, j, k, w = source
        src = Source(int(i), int(j), int(k), _buf(w, "wavelet", "float32", int(step) + 2, cuda=True))
    f = [_buf(x, nm, "float32", E, cuda=True) for x, nm in
         ((u_prev, "u_prev"), (u_cur, "u_cur"), (u_next, "u_next"), (u_next2, "u_next2"),
          (m, "m"), (phi, "phi"))]
    _check(lib().stencil_step2(ctypes.byref(g), *f, int(step),
                               ctypes.byref(src) if src is not None else None, _stream(stream)))


def run_shot(g: Grid, velocity, wavelet, nt: int, src_ijk, rec_ijk, traces, final_u=None,
             stream=None):
    """Whole shot.  velocity, wavelet, traces, final_u: torch tensors (CUDA or
    CPU) or numpy arrays; src_ijk / rec_ijk: host int sequences."""
    s = None if src_ijk is None else np.ascontiguousarray(np.asarray(src_ijk, dtype=np.int32))
    r = np.ascontiguousarray(np.asarray(rec_ijk, dtype=np.int32).reshape(-1, 3))
    nrec = r.shape[0]
    N, nt = _points(g), int(nt)
    _check(lib().run_shot(ctypes.byref(g), _buf(velocity, "velocity", "float32", N),
                          _buf(wavelet, "wavelet", "float32", nt, optional=s is None), nt,
                          None if s is None else s.ctypes.data,
                          r.ctypes.data if nrec else None, nrec,
                          _buf(traces, "traces", "float32", nt * nrec) if nrec else None,
                          _buf(final_u, "final_u", "float32", N, optional=True), _stream(stream)))


def run_shot_segment(g: Grid, velocity, wavelet, n_begin: int, n_end: int, src_ijk, rec_ijk,
                     traces, u_cur, u_prev, phi, stream=None):
    """Steps n_begin .. n_end-1 of a shot from the state (u_cur = u^{n_begin},
    u_prev = u^{n_begin-1}, phi; float32 arrays of the grid's shape, host or
    device), which is overwritten with the state at n_end; traces receives
    n_end - n_begin rows."""
    s = None if src_ijk is None else np.ascontiguousarray(np.asarray(src_ijk, dtype=np.int32))
    r = np.ascontiguousarray(np.asarray(rec_ijk, dtype=np.int32).reshape(-1, 3))
    nrec = r.shape[0]
    N, nb_, ne_ = _points(g), int(n_begin), int(n_end)
    _check(lib().run_shot_segment(ctypes.byref(g), _buf(velocity, "velocity", "float32", N),
                                  _buf(wavelet, "wavelet", "float32", ne_, optional=s is None),
                                  nb_, ne_, None if s is None else s.ctypes.data,
                                  r.ctypes.data if nrec else None, nrec,
                                  _buf(traces, "traces", "float32", (ne_ - nb_) * nrec)
                                  if nrec else None,
                                  _buf(u_cur, "u_cur", "float32", N), _buf(u_prev, "u_prev", "float32", N),
                                  _buf(phi, "phi", "float32", N), _stream(stream)))


def adjoint_shot(g: Grid, velocity, wavelet, nt: int, src_ijk, rec_ijk, observed, grad_velocity,
                 ckpt_every: int = 0, stream=None) -> float:
    """Trace misfit J = 1/2 sum (d - observed)^2 and, into grad_velocity (fp64,
    the velocity's shape, host or device), dJ/dv by the discrete adjoint with
    checkpoints every ckpt_every steps (0: 100).  Returns J."""
    s = np.ascontiguousarray(np.asarray(src_ijk, dtype=np.int32))
    r = np.ascontiguousarray(np.asarray(rec_ijk, dtype=np.int32).reshape(-1, 3))
    J = ctypes.c_double()
    N, nt, nrec = _points(g), int(nt), r.shape[0]
    _check(lib().adjoint_shot(ctypes.byref(g), _buf(velocity, "velocity", "float32", N),
                              _buf(wavelet, "wavelet", "float32", nt), nt,
                              s.ctypes.data, r.ctypes.data, nrec,
                              _buf(observed, "observed", "float32", nt * nrec),
                              int(ckpt_every), ctypes.byref(J),
                              _buf(grad_velocity, "grad_velocity", "float64", N), _stream(stream)))
    return J.value


def run_shot_noalloc(g: Grid, velocity, wavelet, nt: int, src_ijk, rec_ijk, traces,
                     final_u=None, stream=None):
    """run_shot for callers that cannot allocate device memory: same arguments
    (device tensors only for velocity / wavelet / traces / final_u); scratch comes
    from a fixed device array inside the library (small grids only, see the C
    header).  Calls must not overlap on the GPU."""
    s = None if src_ijk is None else np.ascontiguousarray(np.asarray(src_ijk, dtype=np.int32))
    r = np.ascontiguousarray(np.asarray(rec_ijk, dtype=np.int32).reshape(-1, 3))
    nrec = r.shape[0]
    N, nt = _points(g), int(nt)
    _check(lib().run_shot_noalloc(ctypes.byref(g), _buf(velocity, "velocity", "float32", N),
                                  _buf(wavelet, "wavelet", "float32", nt, optional=s is None),
                                  nt, None if s is None else s.ctypes.data,
                                  r.ctypes.data if nrec else None, nrec,
                                  _buf(traces, "traces", "float32", nt * nrec) if nrec else None,
                                  _buf(final_u, "final_u", "float32", N, optional=True),
                                  _stream(stream)))


def pack(g: Grid, compact, padded, stream=None):
    E = int(layout(g).elems)
    _check(lib().sgb_pack(ctypes.byref(g), _buf(compact, "compact", "float32", _points(g), cuda=True),
                          _buf(padded, "padded", "float32", E, cuda=True), _stream(stream)))


def unpack(g: Grid, padded, compact, stream=None):
    E = int(layout(g).elems)
    _check(lib().sgb_unpack(ctypes.byref(g), _buf(padded, "padded", "float32", E, cuda=True),
                            _buf(compact, "compact", "float32", _points(g), cuda=True),
                            _stream(stream)))


def device_status(stream=None):
    _check(lib().sgb_device_status(_stream(stream)))


def selftest_wait_timeout(limit_us: int, stream=None) -> int:
    """Run the bounded-wait self-test; returns the status the host read from the
    device error word (ERR_TIMEOUT when failure detection works)."""
    st = ctypes.c_int32(0)
    _check(lib().sgb_selftest_wait_timeout(int(limit_us), ctypes.byref(st), _stream(stream)))
    return int(st.value)


def debug_fail_allocations(after: int, count: int = 1):
    """Test hook: the library's pool allocations numbered after .. after +
    count - 1 (counted from this call) fail with ERR_OUT_OF_MEMORY; count 0
    disarms.  Process-wide."""
    _check(lib().sgb_debug_fail_allocations(int(after), int(count)))


def pool_used_bytes() -> int:
    """Bytes currently allocated from the current device's library pool."""
    out = ctypes.c_int64()
    _check(lib().sgb_pool_used_bytes(ctypes.byref(out)))
    return int(out.value)


def launch_count(reset: bool = False) -> int:
    return int(lib().sgb_launch_count(1 if reset else 0))


def last_error() -> str:
    return lib().sgb_last_error().decode()


def serve_footprint(g: Grid, nt: int, nrec: int) -> int:
    out = ctypes.c_uint64()
    _check(lib().serve_footprint(ctypes.byref(g), int(nt), int(nrec), ctypes.byref(out)))
    return out.value


class Server:
    """Continuous-batching shot server on the current device (the C API's
    serve_create / serve_submit / serve_poll / serve_destroy)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 16, steps_per_graph: int = 16):
        cfg = ServeConfig(int(hbm_budget_bytes), int(max_slots), int(steps_per_graph))
        h = ctypes.c_void_p()
        _check(lib().serve_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h

    def submit(self, g: Grid, velocity: np.ndarray, wavelet: np.ndarray, nt: int, src_ijk,
               rec_ijk) -> int:
        v = np.ascontiguousarray(velocity, dtype=np.float32)
        w = np.ascontiguousarray(wavelet, dtype=np.float32)
        r = np.ascontiguousarray(np.asarray(rec_ijk, dtype=np.int32).reshape(-1, 3))
        req = ShotRequest(g, v.ctypes.data, w.ctypes.data, int(nt),
                          (ctypes.c_int32 * 3)(*[int(x) for x in src_ijk]), r.ctypes.data,
                          r.shape[0])
        t = ctypes.c_uint64()
        _check(lib().serve_submit(self.h, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int, nt: int, nrec: int, timeout_us: int = 0):
        """(code, result, traces): code OK with traces [nt, nrec], PENDING or
        ERR_TIMEOUT (traces None)."""
        tr = np.zeros((nt, nrec), dtype=np.float32)
        res = ShotResult(0, 0, 0, 0, tr.ctypes.data, 0.0, 0.0)
        rc = lib().serve_poll(self.h, int(ticket), ctypes.byref(res), int(timeout_us))
        if rc in (PENDING, ERR_TIMEOUT):
            return rc, None, None
        _check(rc)
        return rc, res, tr

    def cancel(self, ticket: int):
        _check(lib().serve_cancel(self.h, int(ticket)))

    def stats(self) -> ServeStats:
        out = ServeStats()
        _check(lib().serve_stats(self.h, ctypes.byref(out)))
        return out

    def close(self):
        if self.h:
            _check(lib().serve_destroy(self.h))
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
