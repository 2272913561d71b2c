"""ORACLE -- test infrastructure only (see oracle/__init__.py).

Plain numpy FP64 restatement of the correction plumbing of arXiv 2201.13191
Sec. II-E: line integrals a = -ln(I/I0); FDK for a circular orbit (cosine
pre-weighting, discrete Ram-Lak ramp filter in the isocentre plane,
voxel-driven backprojection with bilinear interpolation and the (D/(D-x.n))^2
weight, dbeta/2 for a full orbit); multi-level Otsu thresholds by exhaustive
search of the between-class variance; and eq. (Correction).
"""

from __future__ import annotations

import numpy as np


def ramlak(n, tau):
    """Discrete Ram-Lak kernel h[k], k = -(n-1)..(n-1)."""
    k = np.arange(-(n - 1), n)
    h = np.zeros(len(k))
    h[k == 0] = 1.0 / (4.0 * tau * tau)
    odd = (k % 2) != 0
    h[odd] = -1.0 / (np.pi * k[odd] * tau) ** 2
    return h


def fdk(p, angles, pu, pv, sod, sdd, grid):
    """p [n_proj][nv][nu] line integrals; grid = (nx, ny, nz, dx, dy, dz); returns vol [nz][ny][nx] (mm^-1)."""
    n_proj, nv, nu = p.shape
    nx, ny, nz, dx, dy, dz = grid
    du, dv = pu * sod / sdd, pv * sod / sdd
    u = (np.arange(nu) - 0.5 * (nu - 1)) * du
    v = (np.arange(nv) - 0.5 * (nv - 1)) * dv
    wgt = sod / np.sqrt(sod**2 + u[None, :] ** 2 + v[:, None] ** 2)
    h = ramlak(nu, du)
    q = np.zeros_like(p, dtype=np.float64)
    for k in range(n_proj):
        pw = p[k] * wgt
        for r in range(nv):
            q[k, r] = np.convolve(pw[r], h, mode="full")[nu - 1 : 2 * nu - 1] * du
    x = (np.arange(nx) - 0.5 * (nx - 1)) * dx
    y = (np.arange(ny) - 0.5 * (ny - 1)) * dy
    z = (np.arange(nz) - 0.5 * (nz - 1)) * dz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    vol = np.zeros((nz, ny, nx))
    for k, b in enumerate(np.asarray(angles, dtype=np.float64)):
        c, s = np.cos(b), np.sin(b)
        depth = sod - (X * c + Y * s)
        mag = sod / depth
        fu = (-X * s + Y * c) * mag / du + 0.5 * (nu - 1)
        fv = Z * mag / dv + 0.5 * (nv - 1)
        u0 = np.floor(fu).astype(int)
        v0 = np.floor(fv).astype(int)
        au, av = fu - u0, fv - v0
        ok = (u0 >= 0) & (u0 + 1 < nu) & (v0 >= 0) & (v0 + 1 < nv)
        u0c, v0c = np.clip(u0, 0, nu - 2), np.clip(v0, 0, nv - 2)
        qk = q[k]
        val = (1 - av) * ((1 - au) * qk[v0c, u0c] + au * qk[v0c, u0c + 1]) + av * (
            (1 - au) * qk[v0c + 1, u0c] + au * qk[v0c + 1, u0c + 1]
        )
        vol += np.where(ok, mag * mag * val, 0.0)
    return vol * np.pi / n_proj


def otsu(hist, classes):
    """Thresholds (bin indices) maximising the between-class variance; ties to the smallest."""
    hist = np.asarray(hist, dtype=np.float64)
    nb = len(hist)
    centers = np.arange(nb) + 0.5
    N = hist.sum()
    mu = (hist * centers).sum() / max(N, 1.0)

    def term(a, b):
        w = hist[a:b].sum()
        if w <= 0:
            return 0.0
        m = (hist[a:b] * centers[a:b]).sum() / w
        return w * (m - mu) ** 2

    best, arg = -1.0, (1, nb)
    if classes == 2:
        for a in range(1, nb):
            v = term(0, a) + term(a, nb)
            if v > best:
                best, arg = v, (a, nb)
    else:
        for a in range(1, nb):
            for b in range(a + 1, nb):
                v = term(0, a) + term(a, b) + term(b, nb)
                if v > best:
                    best, arg = v, (a, b)
    return arg


def correct(a, ip, is_):
    """Eq. (Correction): c = a - ln(Ip / (Ip + Is))."""
    return a - np.log(ip / (ip + is_))
