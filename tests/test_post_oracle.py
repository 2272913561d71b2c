"""Pins of the smoothing / interpolation oracle (arXiv 2201.13191 Sec. II-C.3, II-C.4)."""

import os

import numpy as np
import pytest

from oracle import post

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_sg():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "savitzky_golay_w5_cubic.txt")) if not l.startswith("#")]
    return [(float(r[0]), np.array([float(x) for x in r[1:]])) for r in rows]


def test_sg_weights_match_published_table():
    """Centre weights of the cubic fit equal Savitzky & Golay's Table I."""
    for norm, wts in _golden_sg():
        win = len(wts)
        x = np.zeros(3 * win)
        got = []
        for k in range(win):
            x[:] = 0.0
            x[win + k] = 1.0  # impulse at offset k - m from the centre sample
            got.append(post.sg_smooth_1d(x, win, 3)[win + win // 2])
        np.testing.assert_allclose(np.array(got), wts / norm, atol=1e-12)


@pytest.mark.parametrize("win", [5, 9, 11])
def test_sg_reproduces_cubics_including_edges(win):
    rng = np.random.default_rng(win)
    n = 23
    for _ in range(3):
        c = rng.normal(size=4)
        t = np.arange(n, dtype=np.float64)
        line = c[0] + c[1] * t + c[2] * t**2 + c[3] * t**3
        np.testing.assert_allclose(post.sg_smooth_1d(line, win, 3), line, rtol=1e-9, atol=1e-9 * np.abs(line).max())
    yy, xx = np.meshgrid(np.arange(17.0), np.arange(19.0), indexing="ij")
    img = 1 + 0.5 * xx - 0.1 * yy**2 + 0.01 * xx**3 + 0.02 * xx * yy
    np.testing.assert_allclose(post.sg_smooth_2d(img, win, 3), img, rtol=1e-9, atol=1e-9)


def test_sg_white_noise_variance_factor():
    """Interior output variance of white noise = sum of squared weights."""
    norm, wts = _golden_sg()[1]
    rng = np.random.default_rng(0)
    x = rng.normal(size=20000)
    y = post.sg_smooth_1d(x, 7, 3)[10:-10]
    expect = np.sum((wts / norm) ** 2)
    assert abs(y.var() / expect - 1.0) < 0.05


def test_keys_a075_matches_torch_bicubic():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    img = rng.normal(size=(7, 9))
    ref = torch.nn.functional.interpolate(
        torch.tensor(img)[None, None], size=(17, 23), mode="bicubic", align_corners=False
    )[0, 0].numpy()
    np.testing.assert_allclose(post.cubic_upsample(img, 17, 23, a=-0.75), ref, atol=1e-10)


def test_keys_a05_reproduces_quadratics_interior():
    # Keys (a = -1/2) cubic convolution is exact for polynomials up to degree 2
    nv, nu, NV, NU = 12, 14, 36, 42
    y = np.arange(nv, dtype=np.float64)[:, None]
    x = np.arange(nu, dtype=np.float64)[None, :]
    img = 0.3 + 0.2 * x - 0.05 * y + 0.01 * x * x + 0.02 * x * y - 0.03 * y * y
    out = post.cubic_upsample(img, NV, NU, a=-0.5)
    Y = (np.arange(NV) + 0.5) * nv / NV - 0.5
    X = (np.arange(NU) + 0.5) * nu / NU - 0.5
    ref = 0.3 + 0.2 * X[None] - 0.05 * Y[:, None] + 0.01 * X[None] ** 2 + 0.02 * X[None] * Y[:, None] - 0.03 * Y[:, None] ** 2
    sl = (slice(6, NV - 6), slice(6, NU - 6))  # away from the clamped border
    np.testing.assert_allclose(out[sl], ref[sl], atol=1e-10)


def test_angle_lerp_exact_at_nodes_and_periodic():
    rng = np.random.default_rng(2)
    ang = np.sort(rng.uniform(0, 2 * np.pi, size=6))
    imgs = rng.normal(size=(6, 3, 4))
    for k in range(6):
        np.testing.assert_allclose(post.angle_lerp(imgs, ang, ang[k]), imgs[k], atol=1e-12)
        np.testing.assert_allclose(post.angle_lerp(imgs, ang, ang[k] + 2 * np.pi), imgs[k], atol=1e-12)
    # midway across the wrap from the last angle to the first (+ 2 pi)
    mid = 0.5 * (ang[-1] + ang[0] + 2 * np.pi)
    np.testing.assert_allclose(post.angle_lerp(imgs, ang, mid), 0.5 * (imgs[-1] + imgs[0]), atol=1e-12)
    # linear between neighbours
    th = ang[2] + 0.25 * (ang[3] - ang[2])
    np.testing.assert_allclose(post.angle_lerp(imgs, ang, th), 0.75 * imgs[2] + 0.25 * imgs[3], atol=1e-12)
