"""fp64 CPU oracle for the 25-point acoustic wave step with PML (arXiv 2009.04619).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package.  The product
path (``paper_2009_04619_gb300``) never imports it and fails loudly when its
CUDA library is missing.

The arithmetic lives in ``oracle.c`` (plain C, fp64, OpenMP over z-planes);
this module only marshals numpy arrays through ctypes and converts between the
oracle's own layout (halo of 4 on every side, no padding) and compact
``(Nz, Ny, Nx)`` arrays.

Parity status: interior update, recurrence, source scaling and CFL limit are
pinned by closed forms; the PML update is pinned by invariants only and is
"parity unpinned" against the paper, which prints no PML formulas.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
H = 4  # halo width = stencil radius

_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liboracle.so`` with gcc (fp contraction off,
    so x86 and Arm give the same roundings)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("nb", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.c_double), ("dt", ctypes.c_double), ("vmax", ctypes.c_double),
                ("r0", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        gp = ctypes.POINTER(_Grid)
        L.ora_fd2_weights.argtypes = [ctypes.c_int, dp]
        L.ora_laplacian_coeffs.argtypes = [gp, dp, dp, dp, dp]
        L.ora_cfl_dt.argtypes = [ctypes.c_double] * 4
        L.ora_cfl_dt.restype = ctypes.c_double
        L.ora_field_len.argtypes = [gp]
        L.ora_field_len.restype = ctypes.c_size_t
        L.ora_is_pml.argtypes = [gp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.ora_region.argtypes = [gp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.ora_eta_axis.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int]
        L.ora_eta_axis.restype = ctypes.c_double
        L.ora_eta_max.argtypes = [gp, ctypes.c_double]
        L.ora_eta_max.restype = ctypes.c_double
        L.ora_eta.argtypes = [gp, dp]
        L.ora_laplacian.argtypes = [gp, dp, dp, ctypes.c_int]
        L.ora_step.argtypes = [gp, dp, dp, dp, dp, dp, dp, dp, ctypes.c_int]
        fp = ctypes.POINTER(ctypes.c_float)
        ip = ctypes.POINTER(ctypes.c_int)
        L.ora_step_points.argtypes = [gp, fp, fp, fp, fp, ip, ctypes.c_int, dp, dp, ctypes.c_int]
        L.ora_run_shot.argtypes = [gp, fp, fp, ctypes.c_int, ip, ip, ctypes.c_int, dp, dp, dp, dp,
                                   ctypes.c_int]
        L.ora_run_shot.restype = ctypes.c_int
        L.ora_adjoint_shot.argtypes = [gp, fp, fp, ctypes.c_int, ip, ip, ctypes.c_int, dp, dp, dp,
                                       ctypes.c_int]
        L.ora_adjoint_shot.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a, ctype=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


@dataclass
class Grid:
    """Problem statement of section III-B: inner extents, PML width, spacing, dt,
    plus the two numbers that set the PML damping profile."""
    nx: int
    ny: int
    nz: int
    nb: int
    dx: float
    dy: float
    dz: float
    dt: float
    vmax: float = 0.0
    r0: float = 1e-3

    @property
    def shape(self):
        """Computed domain as (Nz, Ny, Nx)."""
        return (self.nz + 2 * self.nb, self.ny + 2 * self.nb, self.nx + 2 * self.nb)

    def c(self) -> _Grid:
        return _Grid(self.nx, self.ny, self.nz, self.nb, float(self.dx), float(self.dy),
                     float(self.dz), float(self.dt), float(self.vmax), float(self.r0))


def fd2_weights(M: int = 4) -> np.ndarray:
    w = np.zeros(M + 1)
    lib().ora_fd2_weights(M, _ptr(w))
    return w


def laplacian_coeffs(g: Grid):
    c0 = np.zeros(1)
    cx, cy, cz = np.zeros(5), np.zeros(5), np.zeros(5)
    lib().ora_laplacian_coeffs(ctypes.byref(g.c()), _ptr(c0), _ptr(cx), _ptr(cy), _ptr(cz))
    return float(c0[0]), cx, cy, cz


def cfl_dt(vmax: float, dx: float, dy: float, dz: float) -> float:
    return float(lib().ora_cfl_dt(vmax, dx, dy, dz))


def is_pml(g: Grid, i: int, j: int, k: int) -> bool:
    return bool(lib().ora_is_pml(ctypes.byref(g.c()), i, j, k))


def region(g: Grid, i: int, j: int, k: int) -> int:
    return int(lib().ora_region(ctypes.byref(g.c()), i, j, k))


def eta_max(g: Grid, h: float) -> float:
    return float(lib().ora_eta_max(ctypes.byref(g.c()), h))


def eta_axis(n_inner: int, nb: int, emax: float, i: int) -> float:
    return float(lib().ora_eta_axis(n_inner, nb, emax, i))


def full_shape(g: Grid):
    Nz, Ny, Nx = g.shape
    return (Nz + 2 * H, Ny + 2 * H, Nx + 2 * H)


def pad(a: np.ndarray, g: Grid) -> np.ndarray:
    """Compact (Nz, Ny, Nx) -> oracle layout with a zero halo, float64."""
    out = np.zeros(full_shape(g), dtype=np.float64)
    out[H:-H, H:-H, H:-H] = a
    return out


def unpad(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a[H:-H, H:-H, H:-H])


def eta(g: Grid) -> np.ndarray:
    e = np.zeros(full_shape(g))
    lib().ora_eta(ctypes.byref(g.c()), _ptr(e))
    return e


def laplacian(g: Grid, u: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """25-point Laplacian of a compact field (zero outside), compact result."""
    uf = pad(np.asarray(u, dtype=np.float64), g)
    out = np.zeros_like(uf)
    lib().ora_laplacian(ctypes.byref(g.c()), _ptr(uf), _ptr(out), nthreads)
    return unpad(out)


def laplacian_full(g: Grid, ufull: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """25-point Laplacian of a field given in the oracle layout, halo included (the
    halo values are used as they are); compact result."""
    uf = np.ascontiguousarray(ufull, dtype=np.float64)
    assert uf.shape == full_shape(g)
    out = np.zeros_like(uf)
    lib().ora_laplacian(ctypes.byref(g.c()), _ptr(uf), _ptr(out), nthreads)
    return unpad(out)


def step(g: Grid, m, u_prev, u_cur, phi_cur, nthreads: int = 0):
    """One step from compact fields; returns compact (u_next, phi_next)."""
    mf, up, uc, ph = (pad(np.asarray(a, dtype=np.float64), g) for a in (m, u_prev, u_cur, phi_cur))
    e = eta(g)
    un = np.zeros_like(uc)
    pn = np.zeros_like(uc)
    lib().ora_step(ctypes.byref(g.c()), _ptr(mf), _ptr(e), _ptr(up), _ptr(uc), _ptr(ph),
                   _ptr(un), _ptr(pn), nthreads)
    return unpad(un), unpad(pn)


def step_points(g: Grid, m, u_prev, u_cur, phi, pts, nthreads: int = 0):
    """One step evaluated only at the listed points (int [npts, 3] rows (i, j, k)),
    reading float32 compact fields; returns (u_next, phi_next) at those points."""
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (m, u_prev, u_cur, phi)]
    for a in arrs:
        assert a.shape == g.shape
    pts = np.ascontiguousarray(np.asarray(pts, dtype=np.int32).reshape(-1, 3))
    n = pts.shape[0]
    ou, op = np.zeros(n), np.zeros(n)
    lib().ora_step_points(ctypes.byref(g.c()), *(_ptr(a, ctypes.c_float) for a in arrs),
                          _ptr(pts, ctypes.c_int), n, _ptr(ou), _ptr(op), nthreads)
    return ou, op


def run_shot(g: Grid, velocity: np.ndarray, wavelet: np.ndarray, nt: int, src, rec,
             nthreads: int = 0, want_state: bool = True):
    """Algorithm 1 with source and receivers.  velocity: compact float32 (Nz,Ny,Nx);
    wavelet: float32 [nt]; src: (i,j,k) or None; rec: int array [nrec,3].
    Returns dict with traces [nt,nrec] and (optionally) u, u_prev, phi compact."""
    vel = np.ascontiguousarray(velocity, dtype=np.float32)
    assert vel.shape == g.shape
    w = np.ascontiguousarray(wavelet, dtype=np.float32)
    assert w.shape[0] >= nt
    rec = np.ascontiguousarray(np.asarray(rec, dtype=np.int32).reshape(-1, 3))
    nrec = rec.shape[0]
    traces = np.zeros((max(nt, 0), nrec))
    u = np.zeros(g.shape) if want_state else None
    up = np.zeros(g.shape) if want_state else None
    ph = np.zeros(g.shape) if want_state else None
    s = None if src is None else np.ascontiguousarray(np.asarray(src, dtype=np.int32))
    rc = lib().ora_run_shot(ctypes.byref(g.c()), _ptr(vel, ctypes.c_float), _ptr(w, ctypes.c_float),
                            nt, _ptr(s, ctypes.c_int), _ptr(rec, ctypes.c_int), nrec, _ptr(traces),
                            _ptr(u), _ptr(up), _ptr(ph), nthreads)
    if rc != 0:
        raise RuntimeError("oracle run_shot failed")
    return {"traces": traces, "u": u, "u_prev": up, "phi": ph}


def adjoint_shot(g: Grid, velocity: np.ndarray, wavelet: np.ndarray, nt: int, src, rec,
                 observed: np.ndarray, nthreads: int = 0):
    """Misfit J = 1/2 sum (d - obs)^2 of a shot and its gradient dJ/dv (compact
    (Nz, Ny, Nx), float64) by the discrete adjoint; observed: [nt, nrec]."""
    vel = np.ascontiguousarray(velocity, dtype=np.float32)
    w = np.ascontiguousarray(wavelet, dtype=np.float32)
    rec = np.ascontiguousarray(np.asarray(rec, dtype=np.int32).reshape(-1, 3))
    obs = np.ascontiguousarray(observed, dtype=np.float64)
    assert obs.shape == (nt, rec.shape[0])
    s = np.ascontiguousarray(np.asarray(src, dtype=np.int32))
    J = np.zeros(1)
    grad = np.zeros(g.shape)
    rc = lib().ora_adjoint_shot(ctypes.byref(g.c()), _ptr(vel, ctypes.c_float),
                                _ptr(w, ctypes.c_float), nt, _ptr(s, ctypes.c_int),
                                _ptr(rec, ctypes.c_int), rec.shape[0], _ptr(obs), _ptr(J),
                                _ptr(grad), nthreads)
    if rc != 0:
        raise RuntimeError("oracle adjoint_shot failed")
    return float(J[0]), grad
