"""Shared helpers for the GPU tests: device fields in the library's padded layout,
built and read back through the C ABI's own pack/unpack entry points."""
import numpy as np
import torch

from paper_2009_04619_gb300 import build, seisgb

_built = False


def ensure_lib():
    global _built
    if not _built:
        build.build()
        seisgb.lib()
        _built = True


def padded_zeros(g):
    L = seisgb.layout(g)
    return torch.zeros(int(L.elems), dtype=torch.float32, device="cuda")


def to_padded(g, compact: np.ndarray):
    t = torch.from_numpy(np.ascontiguousarray(compact, dtype=np.float32)).cuda()
    out = padded_zeros(g)
    seisgb.pack(g, t, out)
    return out


def from_padded(g, padded) -> np.ndarray:
    out = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    seisgb.unpack(g, padded, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def abs_term_sum(g, m, up, uc, ph):
    """Per point, the sum of absolute values of the terms one step adds up
    (scale for a rounding-error bound of an fp32 evaluation)."""
    w = np.array([205 / 72, 8 / 5, 1 / 5, 8 / 315, 1 / 560])
    h2 = [g.dx ** 2, g.dy ** 2, g.dz ** 2]
    Nz, Ny, Nx = g.shape
    P = np.zeros((Nz + 8, Ny + 8, Nx + 8))
    P[4:-4, 4:-4, 4:-4] = np.abs(uc)
    S = w[0] * (1 / h2[0] + 1 / h2[1] + 1 / h2[2]) * np.abs(uc)
    for m_ in range(1, 5):
        S = S + w[m_] / h2[0] * (P[4:-4, 4:-4, 4 + m_:Nx + 4 + m_] + P[4:-4, 4:-4, 4 - m_:Nx + 4 - m_])
        S = S + w[m_] / h2[1] * (P[4:-4, 4 + m_:Ny + 4 + m_, 4:-4] + P[4:-4, 4 - m_:Ny + 4 - m_, 4:-4])
        S = S + w[m_] / h2[2] * (P[4 + m_:Nz + 4 + m_, 4:-4, 4:-4] + P[4 - m_:Nz + 4 - m_, 4:-4, 4:-4])
    return 2 * np.abs(uc) + np.abs(up) + np.abs(m) * (S + np.abs(ph)) + np.abs(ph)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def abs_term_sum_points(g, m, up, uc, ph, pts):
    """abs_term_sum at listed points (i, j, k) only, for full-size fields."""
    w = np.array([205 / 72, 8 / 5, 1 / 5, 8 / 315, 1 / 560])
    h2 = [g.dx ** 2, g.dy ** 2, g.dz ** 2]
    Nz, Ny, Nx = g.shape
    i, j, k = pts[:, 0].astype(np.int64), pts[:, 1].astype(np.int64), pts[:, 2].astype(np.int64)

    def au(ii, jj, kk):
        ok = (ii >= 0) & (ii < Nx) & (jj >= 0) & (jj < Ny) & (kk >= 0) & (kk < Nz)
        out = np.zeros(len(ii))
        out[ok] = np.abs(uc[kk[ok], jj[ok], ii[ok]])
        return out

    S = w[0] * (1 / h2[0] + 1 / h2[1] + 1 / h2[2]) * au(i, j, k)
    for q in range(1, 5):
        S += w[q] / h2[0] * (au(i + q, j, k) + au(i - q, j, k))
        S += w[q] / h2[1] * (au(i, j + q, k) + au(i, j - q, k))
        S += w[q] / h2[2] * (au(i, j, k + q) + au(i, j, k - q))
    a = lambda f: np.abs(f[k, j, i]).astype(np.float64)
    return 2 * a(uc) + a(up) + a(m) * (S + a(ph)) + a(ph)
