"""ORACLE -- test infrastructure only (see oracle/__init__.py).

Plain numpy FP64 restatement of the correction plumbing of arXiv 2201.13191
Sec. II-E: line integrals a = -ln(I/I0); FDK for a circular orbit (cosine
pre-weighting, discrete Ram-Lak ramp filter in the isocentre plane,
voxel-driven backprojection with bilinear interpolation and the (D/(D-x.n))^2
weight, dbeta/2 for a full orbit); the histogram of the reconstruction,
multi-level Otsu thresholds by exhaustive search of the between-class
variance and the class -> material / density map; eq. (Correction); and the
down-sampling of the segmented volume for the Monte Carlo step (Sec. II-C.2,
Sec. II-E).
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


def histogram(vol, lo, hi, nbins=256):
    """Histogram of mu over [lo, hi) in nbins bins, values outside clamped to the end bins.

    The bin of a value is an integer decided by floating point, so it is taken
    in the precision the library takes it in (FP32): b = trunc((mu - lo) *
    (nbins / (hi - lo))), each operation rounded to FP32, then clamped."""
    f = np.float32
    v = np.asarray(vol, dtype=f).ravel()
    sc = f(nbins) / (f(hi) - f(lo))
    x = (v - f(lo)) * sc
    b = np.clip(np.trunc(x), 0, nbins - 1).astype(np.int64)
    return np.bincount(b, minlength=nbins), b


def segment(vol, lo, hi, classes, class_material, murho_cls, class_density0, rho_max=30.0, nbins=256):
    """Segmentation of a reconstruction (Sec. II-E): Otsu thresholds on the
    histogram, class 0 -> class_material[0] at class_density0, class k >= 1 ->
    class_material[k] at rho = mu / (0.1 murho_cls[k]) clamped to [0, rho_max]
    (murho_cls[k]: mass attenuation of that material at the effective energy,
    cm^2/g).  Returns (mat, rho FP64, hist, thresholds)."""
    hist, b = histogram(vol, lo, hi, nbins)
    t0, t1 = otsu(hist, classes)
    cls = np.where(b < t0, 0, np.where((classes == 2) | (b < t1), 1, 2))
    mu = np.asarray(vol, dtype=np.float64).ravel()
    mat = np.asarray(class_material)[cls].astype(np.uint8)
    mr = np.asarray(murho_cls, dtype=np.float64)[cls]
    rho = np.where(cls == 0, float(np.float32(class_density0)), np.clip(mu / (0.1 * np.where(cls == 0, 1.0, mr)),
                                                                       0.0, rho_max))
    shape = np.shape(vol)
    return mat.reshape(shape), rho.reshape(shape), hist, (t0, t1)


def line_integrals(I, I0):
    """a = -ln(I / I0), both clamped below at 1e-30 (Sec. II-E)."""
    return -np.log(np.maximum(np.asarray(I, np.float64), 1e-30) / np.maximum(np.asarray(I0, np.float64), 1e-30))


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


def correct(a, ip, is_, is_scale=1.0):
    """Eq. (Correction): c = a - ln(Ip / (Ip + s Is)), Ip clamped below at 1e-30 and Is at 0 (s: the pixel-area
    ratio when Is was simulated on coarser pixels, 1 otherwise)."""
    ip = np.maximum(np.asarray(ip, np.float64), 1e-30)
    is_ = np.maximum(np.asarray(is_, np.float64), 0.0) * is_scale
    return np.asarray(a, np.float64) - np.log(ip / (ip + is_))


def bin_volume(mat, rho, murho):
    """Down-sampling of a segmented volume by 2 along each axis for the Monte Carlo step (Sec. II-C.2:
    the number of voxels is down-sampled to cut the ray-tracing time; Sec. II-E).

    mat [nz][ny][nx] material ids, rho the same shape in g/cm^3 (FP64), murho[m] the mass attenuation of
    material m at the correction's effective energy; even dimensions.  Each 2x2x2 block becomes one voxel of
    the material holding the block's largest mass (ties to the lower id), with the density that keeps the
    block's summed attenuation at the effective energy:
        rho_b = sum_v murho[m_v] rho_v / (8 murho[m_b]).
    Returns (mat_b, rho_b) as FP64."""
    nz, ny, nx = mat.shape
    if nx % 2 or ny % 2 or nz % 2:
        raise ValueError("even dimensions needed")
    nm = len(murho)
    blk = lambda t: t.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).transpose(0, 2, 4, 1, 3, 5).reshape(
        nz // 2, ny // 2, nx // 2, 8)
    m8, r8 = blk(mat.astype(np.int64)), blk(np.asarray(rho, dtype=np.float64))
    mass = np.stack([np.where(m8 == m, r8, 0.0).sum(-1) for m in range(nm)], -1)
    mat_b = np.argmax(mass, axis=-1)  # first maximum: the lowest id on ties
    mu = (np.asarray(murho, dtype=np.float64)[m8] * r8).sum(-1)
    rho_b = mu / (8.0 * np.asarray(murho, dtype=np.float64)[mat_b])
    return mat_b.astype(np.uint8), rho_b
