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

FP32 = 0
FP16_SCALED = 1
BF16 = 2


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
                ("pml_r0", ctypes.c_float), ("storage", ctypes.c_int32)]

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
    "run_shot": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "run_shot_noalloc": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "sgb_pack": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p]),
    "sgb_unpack": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    "sgb_device_status": (ctypes.c_int, [ctypes.c_void_p]),
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


def make_grid(nx, ny, nz, nb, dx, dy, dz, dt, vmax, pml_r0=1e-3, storage=FP32) -> Grid:
    return Grid(int(nx), int(ny), int(nz), int(nb), float(dx), float(dy), float(dz), float(dt),
                float(vmax), float(pml_r0), int(storage))


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


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def stencil_step(g: Grid, u_cur, u_prev_to_next, m, phi, step: int = 0, source=None,
                 receivers=None, stream=None):
    """One fused step.  Fields: CUDA tensors in the padded layout.
    source: (i, j, k, wavelet_cuda_tensor) or None.
    receivers: (ijk int32 numpy [nrec, 3], traces_row cuda tensor [nrec]) or None."""
    src = None
    if source is not None:
        i, j, k, w = source
        src = Source(int(i), int(j), int(k), _ptr(w))
    rec = None
    keep = None
    if receivers is not None:
        ijk, row = receivers
        keep = np.ascontiguousarray(np.asarray(ijk, dtype=np.int32).reshape(-1, 3))
        rec = Receivers(keep.shape[0], keep.ctypes.data, _ptr(row))
    rc = lib().stencil_step(ctypes.byref(g), _ptr(u_cur), _ptr(u_prev_to_next), _ptr(m), _ptr(phi),
                            int(step), ctypes.byref(src) if src is not None else None,
                            ctypes.byref(rec) if rec is not None else None, _stream(stream))
    del keep
    _check(rc)


def run_shot(g: Grid, velocity, wavelet, nt: int, src_ijk, rec_ijk, traces, final_u=None,
             stream=None):
    """Whole shot.  velocity, wavelet, traces, final_u: torch tensors (CUDA or
    CPU) or numpy arrays; src_ijk / rec_ijk: host int sequences."""
    s = None if src_ijk is None else np.ascontiguousarray(np.asarray(src_ijk, dtype=np.int32))
    r = np.ascontiguousarray(np.asarray(rec_ijk, dtype=np.int32).reshape(-1, 3))
    nrec = r.shape[0]
    _check(lib().run_shot(ctypes.byref(g), _ptr(velocity), _ptr(wavelet), int(nt),
                          None if s is None else s.ctypes.data,
                          r.ctypes.data if nrec else None, nrec,
                          _ptr(traces) if nrec else None, _ptr(final_u), _stream(stream)))


def run_shot_noalloc(g: Grid, velocity, wavelet, nt: int, src_ijk, rec_ijk, traces,
                     final_u=None, stream=None):
    """run_shot for callers that cannot allocate device memory: same arguments
    (device tensors only for velocity / wavelet / traces / final_u); scratch comes
    from a fixed device array inside the library (small grids only, see the C
    header).  Calls must not overlap on the GPU."""
    s = None if src_ijk is None else np.ascontiguousarray(np.asarray(src_ijk, dtype=np.int32))
    r = np.ascontiguousarray(np.asarray(rec_ijk, dtype=np.int32).reshape(-1, 3))
    nrec = r.shape[0]
    _check(lib().run_shot_noalloc(ctypes.byref(g), _ptr(velocity), _ptr(wavelet), int(nt),
                                  None if s is None else s.ctypes.data,
                                  r.ctypes.data if nrec else None, nrec,
                                  _ptr(traces) if nrec else None, _ptr(final_u),
                                  _stream(stream)))


def pack(g: Grid, compact, padded, stream=None):
    _check(lib().sgb_pack(ctypes.byref(g), _ptr(compact), _ptr(padded), _stream(stream)))


def unpack(g: Grid, padded, compact, stream=None):
    _check(lib().sgb_unpack(ctypes.byref(g), _ptr(padded), _ptr(compact), _stream(stream)))


def device_status(stream=None):
    _check(lib().sgb_device_status(_stream(stream)))


def launch_count(reset: bool = False) -> int:
    return int(lib().sgb_launch_count(1 if reset else 0))


def last_error() -> str:
    return lib().sgb_last_error().decode()
