"""Forced detection in the oracle (the variance-reduction technique Sec. I of
arXiv 2201.13191 names beside splitting and Russian roulette): every scatter
interaction scores every pixel once instead of n_split randomly drawn pixels.

Pinned against the deterministic single-scatter quadrature of the homogeneous
water box (the same integral the paper's estimator is pinned to, with power
against a 3% bias), against the paper's split estimator on the same run
(equal means), and for what it is for: a lower variance per interaction."""

import numpy as np
import pytest

from mc_inputs import make_workload, mono_spectrum, slab_phantom
from mc_inputs.tables import MAT_WATER
from test_oracle_pins import BOX, BOX_GEO, _single_scatter_quadrature


GEO4 = dict(BOX_GEO, nu=4, nv=4, pu=8.0, pv=8.0)  # the same panel area in 4 x 4 pixels


def _box_oracle(oracle_lib, table_path, forced, geo=BOX_GEO):
    o = oracle_lib.Oracle(table_path)
    o.load_volume(slab_phantom((BOX["n"],) * 3, (BOX["dv"],) * 3, MAT_WATER, 1.0))
    o.set_spectrum(*mono_spectrum(60.0))
    o.set_geometry(**geo)
    o.set_forced(forced)
    return o


def _batches(o, N, B, seed):
    parts = [o.scatter(0.0, N, 1.0, seed, h_begin=b * N // B, h_end=(b + 1) * N // B, orders=True)["orders"][0]
             for b in range(B)]
    return np.array(parts)


def test_forced_detection_single_scatter_quadrature(oracle_lib, table_path, tables):
    """Order-1 image per pixel within 3 sigma of the quadrature on the 8 x 8
    panel; on a 4 x 4 panel of the same area, with more histories, the total
    within 3 standard errors while the total scaled by 3% is rejected."""
    ref = _single_scatter_quadrature(tables, table_path, oracle_lib, 60.0)
    o = _box_oracle(oracle_lib, table_path, 1)
    N, B = 30_000, 10
    parts = _batches(o, N, B, 91)
    est = parts.sum(axis=0)
    sig = np.sqrt(parts.var(axis=0, ddof=1) * B)
    z = np.abs(est - ref) / sig
    assert np.mean(z < 3.0) >= 0.95, z.max()
    ref = _single_scatter_quadrature(tables, table_path, oracle_lib, 60.0, geo=GEO4)
    parts = _batches(_box_oracle(oracle_lib, table_path, 1, GEO4), 400_000, B, 92)
    tot = parts.sum(axis=(1, 2))
    se = np.sqrt(tot.var(ddof=1) * B)
    assert abs(tot.sum() - ref.sum()) < 3.0 * se, (tot.sum(), ref.sum(), se)
    assert abs(1.03 * tot.sum() - ref.sum()) > 3.0 * se


def test_forced_detection_matches_split_estimator_with_less_noise(oracle_lib, table_path, tables):
    """Both estimators have the same mean, and forced detection's per-pixel
    noise is lower (the photon walks are statistically the same but not the
    same draws: forced detection reserves one counter block per pixel)."""
    N, B = 20_000, 10
    pf = _batches(_box_oracle(oracle_lib, table_path, 1), N, B, 5)
    ps = _batches(_box_oracle(oracle_lib, table_path, 0), N, B, 5)
    tf, ts = pf.sum(axis=(1, 2)), ps.sum(axis=(1, 2))
    se = np.sqrt((tf.var(ddof=1) + ts.var(ddof=1)) * B)
    assert abs(tf.sum() - ts.sum()) < 3.0 * se
    # per-pixel noise: forced detection removes the pixel-selection variance
    vf = pf.var(axis=0, ddof=1).sum()
    vs = ps.var(axis=0, ddof=1).sum()
    assert vf < 0.5 * vs, (vf, vs)


def test_forced_detection_with_tiles_and_walks(oracle_lib, table_path, tables):
    """Forced detection scores every pixel once per scatter interaction; one
    tile covering the panel equals no tiles; the option is 0 or 1."""
    wl = make_workload("tiny8", tables)
    o = oracle_lib.Oracle(table_path)
    o.setup(wl)
    o.set_forced(1)
    a = o.scatter(0.4, 4000, wl["step_mm"], 3)
    o.set_tiles(wl["geometry"]["nu"], wl["geometry"]["nv"])
    b = o.scatter(0.4, 4000, wl["step_mm"], 3)
    np.testing.assert_array_equal(a["Is"], b["Is"])
    npix = wl["geometry"]["nu"] * wl["geometry"]["nv"]
    inter = a["stats"]["compton"] + a["stats"]["rayleigh"]
    assert a["stats"]["nee_rays"] == inter * npix
    with pytest.raises(RuntimeError):
        o.set_forced(2)
