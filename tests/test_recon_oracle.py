"""Pins of the correction-plumbing oracle (oracle/recon.py): Ram-Lak kernel,
FDK of analytic projections of a uniform cylinder, Otsu thresholds, eq. (Correction)."""

import numpy as np
import pytest

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


def test_otsu_ties_and_within_class_minimum():
    """Otsu's thresholds maximise the between-class variance, which is the same
    as minimising the total within-class variance (their sum is the fixed total
    variance): checked against that second formula by brute force; two or
    three point masses give a flat optimum, resolved to the smallest
    thresholds."""
    h = np.zeros(64)
    h[10], h[50] = 100, 100
    assert recon.otsu(h, 2) == (11, 64)
    h3 = np.zeros(64)
    h3[5], h3[30], h3[55] = 100, 80, 60
    assert recon.otsu(h3, 3) == (6, 31)
    rng = np.random.default_rng(3)
    c = np.arange(64) + 0.5
    h = np.round(300 * np.exp(-0.5 * ((c - 12) / 4) ** 2) + 200 * np.exp(-0.5 * ((c - 33) / 5) ** 2)
                 + 120 * np.exp(-0.5 * ((c - 52) / 3) ** 2) + rng.integers(0, 4, 64))

    def within(cuts):
        tot = 0.0
        for lo, hi in zip((0,) + cuts, cuts + (64,)):
            w = h[lo:hi]
            if w.sum() > 0:
                m = (w * c[lo:hi]).sum() / w.sum()
                tot += (w * (c[lo:hi] - m) ** 2).sum()
        return tot

    best2 = min(range(1, 64), key=lambda a: (within((a,)), a))
    assert recon.otsu(h, 2) == (best2, 64)
    best3 = min(((a, b) for a in range(1, 64) for b in range(a + 1, 64)), key=lambda t: (within(t), t))
    assert recon.otsu(h, 3) == best3


def test_histogram_and_segmentation_map():
    """256 bins over [lo, hi): a value at a bin's centre lands in that bin,
    values outside the range in the end bins; a three-level volume splits into
    its three classes, class 0 takes the background density and the others
    rho = mu / (0.1 mu/rho) of their material."""
    lo, hi = -0.01, 0.09
    centres = lo + (np.arange(256) + 0.5) * (hi - lo) / 256
    hist, b = recon.histogram(centres, lo, hi)
    np.testing.assert_array_equal(b, np.arange(256))
    assert np.all(hist == 1)
    hist, b = recon.histogram(np.array([-5.0, lo, hi, 7.0]), lo, hi)
    assert list(b) == [0, 0, 255, 255] and hist.sum() == 4
    rng = np.random.default_rng(2)
    lvl = rng.choice(3, size=(6, 7, 8))
    mu = np.array([0.0002, 0.0206, 0.075])[lvl] + rng.normal(0, 0.001, lvl.shape)
    murho = [1.0, 0.206, 0.278]  # class 0's entry is unused
    mat, rho, hist, (t0, t1) = recon.segment(mu, lo, hi, 3, [0, 1, 3], murho, 0.001205)
    np.testing.assert_array_equal(mat, np.array([0, 1, 3], np.uint8)[lvl])
    assert hist.sum() == mu.size and 0 < t0 < t1 < 256
    np.testing.assert_allclose(rho[lvl == 0], np.float32(0.001205), rtol=0)
    for k, m in ((1, 0.206), (2, 0.278)):
        np.testing.assert_allclose(rho[lvl == k], np.clip(mu[lvl == k] / (0.1 * m), 0, 30), rtol=1e-15)
    # two classes: one cut between two of the levels, no level split, air in class 0
    mat2, _, _, (a, bb) = recon.segment(mu, lo, hi, 2, [0, 1, 1], murho, 0.001205)
    assert bb == 256 and np.all(mat2[lvl == 0] == 0) and np.all(mat2[lvl == 2] == 1)
    assert len(np.unique(mat2[lvl == 1])) == 1


def test_line_integrals():
    rng = np.random.default_rng(1)
    I0 = rng.uniform(0.5, 2.0, (4, 5))
    a = rng.uniform(0.0, 6.0, (3, 4, 5))
    np.testing.assert_allclose(recon.line_integrals(I0 * np.exp(-a), I0), a, atol=1e-12)


def test_correction_formula():
    rng = np.random.default_rng(0)
    ip = rng.uniform(0.1, 1.0, 100)
    is_ = rng.uniform(0.0, 0.5, 100)
    i0 = 1.3
    a = -np.log((ip + is_) / i0)
    np.testing.assert_allclose(recon.correct(a, ip, is_), -np.log(ip / i0), atol=1e-12)
    np.testing.assert_allclose(recon.correct(a, ip, np.zeros(100)), a, atol=0)
    # Is simulated on pixels k times larger than the panel's: scaled by the area ratio
    np.testing.assert_allclose(recon.correct(a, ip, 4.0 * is_, is_scale=0.25), -np.log(ip / i0), atol=1e-12)


def test_bin_volume_pins():
    """2x2x2 down-sampling for the Monte Carlo step: a uniform block keeps its material and density; the
    attenuation at the effective energy is conserved block by block; the block's material is the one with
    the largest mass, ties to the lower id."""
    from oracle.recon import bin_volume

    murho = np.array([0.19, 0.206, 0.2, 0.278, 0.29])
    rng = np.random.default_rng(4)
    mat = rng.choice(np.array([0, 1, 3]), size=(6, 8, 4)).astype(np.uint8)
    rho = np.where(mat == 0, 0.0012, np.where(mat == 1, 1.0, 2.7)) * rng.uniform(0.8, 1.2, mat.shape)
    mb, rb = bin_volume(mat, rho, murho)
    assert mb.shape == (3, 4, 2) and rb.shape == (3, 4, 2)
    mu_f = (murho[mat] * rho).reshape(3, 2, 4, 2, 2, 2).sum(axis=(1, 3, 5))
    np.testing.assert_allclose(8.0 * murho[mb] * rb, mu_f, rtol=1e-12)
    # the largest mass per block, by brute force
    for z in range(3):
        for y in range(4):
            for x in range(2):
                m = mat[2 * z:2 * z + 2, 2 * y:2 * y + 2, 2 * x:2 * x + 2].ravel()
                r = rho[2 * z:2 * z + 2, 2 * y:2 * y + 2, 2 * x:2 * x + 2].ravel()
                masses = {k: r[m == k].sum() for k in set(m.tolist())}
                best = max(sorted(masses), key=lambda k: masses[k])
                assert mb[z, y, x] == best
    # uniform blocks are unchanged; ties go to the lower id
    u = np.full((2, 2, 2), 3, np.uint8)
    mb, rb = bin_volume(u, np.full((2, 2, 2), 2.5), murho)
    assert mb[0, 0, 0] == 3 and abs(rb[0, 0, 0] - 2.5) < 1e-15
    t = np.zeros((2, 2, 2), np.uint8)
    t.ravel()[:4] = 1
    t.ravel()[4:] = 2
    mb, _ = bin_volume(t, np.ones((2, 2, 2)), murho)
    assert mb[0, 0, 0] == 1
    with pytest.raises(ValueError):
        bin_volume(np.zeros((3, 2, 2), np.uint8), np.ones((3, 2, 2)), murho)
