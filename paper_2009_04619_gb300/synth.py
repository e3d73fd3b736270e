"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds input recipes only (velocity models, the source wavelet,
source/receiver positions and the workload definitions); none of the stencil,
boundary or time-stepping arithmetic lives here.  Everything is numpy, seeded,
and returns float32 arrays in the compact ``(Nz, Ny, Nx)`` layout (x fastest,
z = depth).

The paper runs bare cubes (1000^3 on V100, section V-A) with an unstated Earth
model and no public dataset; these layered models stand in for it.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def ricker(nt: int, dt: float, fp: float, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet samples w(n dt), n = 0..nt-1, peak frequency fp, delay t0
    (default 1/fp).  The paper's source f is unspecified; this is the usual
    seismic choice."""
    if t0 is None:
        t0 = 1.0 / fp
    t = np.arange(nt, dtype=np.float64) * float(dt) - t0
    a = (np.pi * fp * t) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float32)


def constant_model(shape, v: float) -> np.ndarray:
    return np.full(shape, v, dtype=np.float32)


def _smooth_noise(shape, rng, sigma: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter1d

    p = rng.standard_normal(shape, dtype=np.float32)
    for ax in range(3):
        if shape[ax] > 1:
            p = gaussian_filter1d(p, sigma, axis=ax, truncate=3.0, mode="nearest")
    mx = float(np.max(np.abs(p)))
    if mx > 0:
        p /= mx
    return p


def layered_model(shape, seed: int = 2009, vmin: float = 1500.0, vmax: float = 4500.0,
                  layers=(8, 20), perturb: float = 0.05, sigma: float = 4.0) -> np.ndarray:
    """Horizontal layers along z (depth): L ~ U{8..20} layers, L-1 distinct
    interface depths, per-layer velocity ~ U(vmin, vmax); then a multiplicative
    perturbation v (1 + perturb * p), p = Gaussian-smoothed white noise
    (sigma points, seed + 1) normalised to max |p| = 1."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    L = int(rng.integers(layers[0], layers[1] + 1))
    L = max(1, min(L, nz))
    cuts = np.sort(rng.choice(np.arange(1, max(nz, 2)), size=min(L - 1, max(nz - 1, 0)),
                              replace=False)) if L > 1 else np.zeros(0, dtype=np.int64)
    vel_layers = rng.uniform(vmin, vmax, size=len(cuts) + 1)
    layer_of_k = np.searchsorted(cuts, np.arange(nz), side="right")
    v_k = vel_layers[layer_of_k].astype(np.float32)
    v = np.broadcast_to(v_k[:, None, None], shape).astype(np.float32)
    if perturb:
        p = _smooth_noise(shape, np.random.default_rng(seed + 1), sigma)
        v *= (1.0 + perturb * p)
    return np.ascontiguousarray(v, dtype=np.float32)


def gaussian_anomaly(shape, center, radius: float, amplitude: float) -> np.ndarray:
    """Multiplicative factor 1 + amplitude * exp(-r^2 / (2 radius^2))."""
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r2 = (i - center[0]) ** 2 + (j - center[1]) ** 2 + (k - center[2]) ** 2
    return (1.0 + amplitude * np.exp(-r2 / (2.0 * radius ** 2))).astype(np.float32)


def surface_receivers(nx: int, ny: int, nb: int, every: int = 4, depth: int = 0) -> np.ndarray:
    """Receivers on the top face of the inner region (k = nb + depth), every
    ``every``-th inner point in x and y; int32 [nrec, 3] rows (i, j, k)."""
    ii = np.arange(nb, nb + nx, every)
    jj = np.arange(nb, nb + ny, every)
    J, I = np.meshgrid(jj, ii, indexing="ij")
    K = np.full_like(I, nb + depth)
    return np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1).astype(np.int32)


@dataclass
class Workload:
    """One forward-modelling workload: inner extents, PML width, spacing, model
    recipe, source, receivers, number of steps, dt as a fraction of the CFL
    limit."""
    name: str
    nx: int
    ny: int
    nz: int
    nb: int
    h: float
    nt: int
    fp: float
    model: str  # "constant" or "layered"
    v_const: float = 2000.0
    seed: int = 2009
    src: tuple | None = None  # (i, j, k) in computed coordinates
    rec_every: int = 4
    cfl_fraction: float = 0.4
    extra: dict = field(default_factory=dict)

    @property
    def shape(self):
        return (self.nz + 2 * self.nb, self.ny + 2 * self.nb, self.nx + 2 * self.nb)

    @property
    def points(self) -> int:
        a, b, c = self.shape
        return a * b * c

    def velocity(self) -> np.ndarray:
        if self.model == "constant":
            return constant_model(self.shape, self.v_const)
        return layered_model(self.shape, seed=self.seed)

    def source(self):
        if self.src is not None:
            return tuple(int(s) for s in self.src)
        Nz, Ny, Nx = self.shape
        return (Nx // 2, Ny // 2, Nz // 2)

    def receivers(self) -> np.ndarray:
        return surface_receivers(self.nx, self.ny, self.nb, self.rec_every)


# Plain FP32 forward modelling, parity case: 64^3 inner + 16-point PML
# (96^3 computed), h = 10 m, v = 2000 m/s, 15 Hz Ricker at the centre, 100 steps.
SMALL = Workload(name="fwd64_pml16_const2000_ricker15_nt100", nx=64, ny=64, nz=64, nb=16,
                 h=10.0, nt=100, fp=15.0, model="constant", v_const=2000.0, src=(48, 48, 48),
                 rec_every=8)

# Single large shot: 512^3 computed (448^3 inner + 32-point PML), h = 10 m,
# layered model (seed 2009), 10 Hz Ricker at 20 m depth below the inner top
# face, 1000 steps, receivers on every 4th inner surface point (112^2).
LARGE = Workload(name="fwd512_pml32_layered_ricker10_nt1000", nx=448, ny=448, nz=448, nb=32,
                 h=10.0, nt=1000, fp=10.0, model="layered", seed=2009, src=(256, 256, 34),
                 rec_every=4)


def scaled(w: Workload, n_inner: int, nb: int, nt: int, name: str | None = None) -> Workload:
    """Same recipe at another size (source kept at the centre column, same depth
    below the top face)."""
    N = n_inner + 2 * nb
    s = w.src
    src = None if s is None else (N // 2, N // 2, nb + (s[2] - w.nb) if s[2] != (w.nz + 2 * w.nb) // 2
                                  else N // 2)
    return Workload(name=name or f"{w.name}@{N}", nx=n_inner, ny=n_inner, nz=n_inner, nb=nb, h=w.h,
                    nt=nt, fp=w.fp, model=w.model, v_const=w.v_const, seed=w.seed, src=src,
                    rec_every=w.rec_every, cfl_fraction=w.cfl_fraction)


# Gradient workload: 256^3 computed (224^3 inner + 16-point PML), h = 10 m, the
# layered model (seed 2009) times a seeded Gaussian anomaly, 10 Hz Ricker,
# 2000 steps, 16 shots on a 4 x 4 grid of surface positions 20 m deep,
# receivers on every 4th inner surface point, checkpoints every 100 steps.
GRADIENT = Workload(name="grad256_pml16_layered_anomaly_ricker10_nt2000_16shots", nx=224, ny=224,
                    nz=224, nb=16, h=10.0, nt=2000, fp=10.0, model="layered", seed=2009,
                    rec_every=4, extra={"shots": 16, "ckpt_every": 100, "anomaly_seed": 5})


def anomaly_params(w: Workload, seed: int):
    """Seeded Gaussian anomaly inside the inner region: centre uniform in its
    middle half, radius U(8, 24) points, amplitude U(5%, 10%) with a random
    sign.  Returns (centre (i, j, k), radius, amplitude)."""
    rng = np.random.default_rng(seed)
    lo = [w.nb + n // 4 for n in (w.nx, w.ny, w.nz)]
    hi = [w.nb + 3 * n // 4 for n in (w.nx, w.ny, w.nz)]
    c = tuple(float(rng.uniform(a, b)) for a, b in zip(lo, hi))
    radius = float(rng.uniform(8.0, 24.0))
    amp = float(rng.uniform(0.05, 0.10)) * (1.0 if rng.random() < 0.5 else -1.0)
    return c, radius, amp


def gradient_models(w: Workload):
    """(v, v_obs): the layered model with the anomaly, where the gradient is
    taken, and the unperturbed layered model that generates the observed data."""
    v0 = w.velocity()
    c, radius, amp = anomaly_params(w, w.extra.get("anomaly_seed", 5))
    v = (v0 * gaussian_anomaly(v0.shape, c, radius, amp)).astype(np.float32)
    return v, v0


def shot_grid(w: Workload, per_side: int = 4, depth: int = 2):
    """per_side^2 source positions on a regular grid over the inner surface,
    `depth` points below it."""
    xs = [w.nb + int((q + 0.5) * w.nx / per_side) for q in range(per_side)]
    ys = [w.nb + int((q + 0.5) * w.ny / per_side) for q in range(per_side)]
    return [(x, y, w.nb + depth) for y in ys for x in xs]


# Serving workload: shot requests over four grid sizes (computed x, y, z; PML 16).
SERVE_GRIDS = [(128, 128, 128), (192, 192, 256), (256, 256, 256), (384, 384, 256)]


def serving_requests(n: int = 256, seed: int = 4, nb: int = 16, h: float = 10.0, fp: float = 10.0,
                     nt_range=(500, 2000), models_per_grid: int = 8, rec_every: int = 8):
    """Seeded shot requests: grid uniform over SERVE_GRIDS, nt uniform in
    nt_range, a layered model (1500-4500 m/s, drawn from a pool of
    models_per_grid seeded models per grid), source uniform over the inner
    top surface 20 m deep, receivers on every rec_every-th inner surface point.
    Returns a list of dicts (the velocity arrays are shared within a pool)."""
    rng = np.random.default_rng(seed)
    pool = {}
    out = []
    for i in range(n):
        gx, gy, gz = SERVE_GRIDS[int(rng.integers(len(SERVE_GRIDS)))]
        nt = int(rng.integers(nt_range[0], nt_range[1] + 1))
        mseed = int(rng.integers(models_per_grid))
        key = (gx, gy, gz, mseed)
        if key not in pool:
            pool[key] = layered_model((gz, gy, gx), seed=seed * 1000 + 17 * len(pool) + mseed,
                                      perturb=0.0)
        nx, ny, nz = gx - 2 * nb, gy - 2 * nb, gz - 2 * nb
        src = (nb + int(rng.integers(nx)), nb + int(rng.integers(ny)), nb + 2)
        out.append({"nx": nx, "ny": ny, "nz": nz, "nb": nb, "h": h, "nt": nt, "fp": fp,
                    "velocity": pool[key], "src": src,
                    "rec": surface_receivers(nx, ny, nb, rec_every)})
    return out
