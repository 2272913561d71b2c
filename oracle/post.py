"""ORACLE -- test infrastructure only (see oracle/__init__.py).

Plain numpy restatement of the smoothing and dual interpolation applied to the
simulated scatter, arXiv 2201.13191 Sec. II-C.3 and II-C.4:

* Savitzky-Golay smoothing: at every sample, a least-squares polynomial of the
  given order is fitted to a window of samples and evaluated at the sample
  (Sec. II-C.4 fixes order three).  Near an edge the window is the first or
  last `win` samples (the fit is the same, evaluated off-centre).  The 2-D
  filter applies the 1-D one along rows, then along columns.
* interpolation between simulated projections: linear in angle, periodic in
  2 pi (Sec. II-C.3, "half of these projections ... interpolation");
* spatial up-sampling by cubic interpolation (Sec. II-C.3): Keys' cubic
  convolution kernel with parameter a, pixel centres aligned (source
  coordinate (X + 1/2) n/N - 1/2), indices clamped at the edges.

Each step is written from its definition, one sample at a time, so that it
can be read against the paper; it is slow and meant for small images.
"""

from __future__ import annotations

import numpy as np


def sg_fit_value(samples, positions, order, at):
    """Least-squares polynomial of `order` through (positions, samples), evaluated at `at`."""
    V = np.vander(np.asarray(positions, dtype=np.float64), order + 1, increasing=True)
    coef, *_ = np.linalg.lstsq(V, np.asarray(samples, dtype=np.float64), rcond=None)
    return float(np.polyval(coef[::-1], at))


def sg_smooth_1d(x, win, order):
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    if n < win:
        raise ValueError("line shorter than the window")
    m = win // 2
    out = np.empty(n)
    for i in range(n):
        s = min(max(i - m, 0), n - win)
        # positions measured from the window start keep the fit well conditioned
        pos = np.arange(win, dtype=np.float64)
        out[i] = sg_fit_value(x[s : s + win], pos, order, i - s)
    return out


def sg_smooth_2d(img, win, order):
    img = np.asarray(img, dtype=np.float64)
    rows = np.stack([sg_smooth_1d(r, win, order) for r in img])
    return np.stack([sg_smooth_1d(c, win, order) for c in rows.T]).T


def keys_kernel(x, a):
    x = abs(x)
    if x <= 1.0:
        return (a + 2.0) * x**3 - (a + 3.0) * x**2 + 1.0
    if x < 2.0:
        return a * x**3 - 5.0 * a * x**2 + 8.0 * a * x - 4.0 * a
    return 0.0


def cubic_upsample(img, NV, NU, a=-0.5):
    img = np.asarray(img, dtype=np.float64)
    nv, nu = img.shape
    out = np.empty((NV, NU))
    for Y in range(NV):
        sy = (Y + 0.5) * nv / NV - 0.5
        y0 = int(np.floor(sy))
        for X in range(NU):
            sx = (X + 0.5) * nu / NU - 0.5
            x0 = int(np.floor(sx))
            acc = 0.0
            for ky in range(y0 - 1, y0 + 3):
                wy = keys_kernel(sy - ky, a)
                yi = min(max(ky, 0), nv - 1)
                for kx in range(x0 - 1, x0 + 3):
                    wx = keys_kernel(sx - kx, a)
                    xi = min(max(kx, 0), nu - 1)
                    acc += wy * wx * img[yi, xi]
            out[Y, X] = acc
    return out


def angle_lerp(images, in_angles, out_angle):
    """Linear interpolation in angle between the bracketing simulated angles, periodic in 2 pi."""
    images = np.asarray(images, dtype=np.float64)
    ang = np.asarray(in_angles, dtype=np.float64)
    n = len(ang)
    if n == 1:
        return images[0].copy()
    two_pi = 2.0 * np.pi
    th = (float(out_angle) - ang[0]) % two_pi
    rel = ang - ang[0]
    k = n - 1
    for i in range(n - 1):
        if th < rel[i + 1]:
            k = i
            break
    lo = rel[k]
    hi = rel[k + 1] if k + 1 < n else two_pi
    f = (th - lo) / (hi - lo)
    return (1.0 - f) * images[k] + f * images[(k + 1) % n]


def smooth_upsample(images, in_angles, out_angles, NU, NV, win=9, order=3, a=-0.5, smooth=True):
    imgs = [sg_smooth_2d(im, win, order) if smooth else np.asarray(im, dtype=np.float64) for im in images]
    return np.stack([cubic_upsample(angle_lerp(imgs, in_angles, th), NV, NU, a) for th in out_angles])
