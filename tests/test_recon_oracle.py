"""Pins of the correction-plumbing oracle (oracle/recon.py): Ram-Lak kernel,
FDK of analytic projections of a uniform cylinder, Otsu thresholds, eq. (Correction)."""

import numpy as np

from oracle import recon

SOD, SDD = 300.0, 600.0


def cylinder_projections(n_proj, nu, nv, pu, pv, R, Hc, mu):
    """Exact line integrals of a uniform cylinder (axis z, radius R, height Hc) for this geometry."""
    angles = 2 * np.pi * np.arange(n_proj) / n_proj
    p = np.zeros((n_proj, nv, nu))
    for k, b in enumerate(angles):
        s = SOD * np.array([np.cos(b), np.sin(b), 0.0])
        c = (SOD - SDD) * np.array([np.cos(b), np.sin(b), 0.0])
        eu = np.array([-np.sin(b), np.cos(b), 0.0])
        iu = (np.arange(nu) - 0.5 * (nu - 1)) * pu
        iv = (np.arange(nv) - 0.5 * (nv - 1)) * pv
        P = c[None, None, :] + iu[None, :, None] * eu[None, None, :] + iv[:, None, None] * np.array([0, 0, 1.0])
        D = P - s
        d = np.linalg.norm(D, axis=-1)
        w = D / d[..., None]
        # |s_xy + t w_xy|^2 = R^2
        A = w[..., 0] ** 2 + w[..., 1] ** 2
        B = 2 * (s[0] * w[..., 0] + s[1] * w[..., 1])
        Cc = s[0] ** 2 + s[1] ** 2 - R * R
        disc = B * B - 4 * A * Cc
        ok = disc > 0
        sq = np.sqrt(np.where(ok, disc, 0.0))
        t1, t2 = (-B - sq) / (2 * A), (-B + sq) / (2 * A)
        # clip to |z| <= Hc/2
        with np.errstate(divide="ignore", invalid="ignore"):
            tz1 = np.where(w[..., 2] != 0, (-Hc / 2 - s[2]) / w[..., 2], -np.inf)
            tz2 = np.where(w[..., 2] != 0, (Hc / 2 - s[2]) / w[..., 2], np.inf)
        lo = np.maximum(t1, np.minimum(tz1, tz2))
        hi = np.minimum(t2, np.maximum(tz1, tz2))
        p[k] = np.where(ok, np.maximum(hi - lo, 0.0), 0.0) * mu
    return angles, p


def test_ramlak_zero_dc():
    h = recon.ramlak(4001, 0.5)
    assert abs(h.sum() * 0.5) < 2e-4  # the ramp has zero DC gain (truncated tail)
    np.testing.assert_allclose(h, h[::-1])


def test_fdk_recovers_uniform_cylinder():
    mu = 0.02
    angles, p = cylinder_projections(90, 64, 48, 2.0, 2.0, 20.0, 80.0, mu)
    vol = recon.fdk(p, angles, 2.0, 2.0, SOD, SDD, (48, 48, 9, 1.0, 1.0, 1.0))
    sl = vol[4]
    x = np.arange(48) - 23.5
    r = np.sqrt(x[None, :] ** 2 + x[:, None] ** 2)
    assert abs(sl[r < 15].mean() / mu - 1.0) < 0.02
    assert np.abs(sl[r > 26]).max() < 0.1 * mu


def test_otsu_bimodal_and_trimodal():
    h = np.zeros(64)
    h[10], h[50] = 100, 100
    a, _ = recon.otsu(h, 2)
    assert 10 < a <= 50
    h3 = np.zeros(64)
    h3[5], h3[30], h3[55] = 100, 80, 60
    a, b = recon.otsu(h3, 3)
    assert 5 < a <= 30 < b <= 55


def test_correction_formula():
    rng = np.random.default_rng(0)
    ip = rng.uniform(0.1, 1.0, 100)
    is_ = rng.uniform(0.0, 0.5, 100)
    i0 = 1.3
    a = -np.log((ip + is_) / i0)
    np.testing.assert_allclose(recon.correct(a, ip, is_), -np.log(ip / i0), atol=1e-12)
    np.testing.assert_allclose(recon.correct(a, ip, np.zeros(100)), a, atol=0)
