"""Tile-stratified point-detector scoring in the oracle (tally locality, eq. Is).

History h aims every pseudo-particle at tile t = (h + o) mod T of the panel
(o uniform on [0, T), one per run and angle), at a pixel drawn uniformly
inside it, and scores with the factor T, so that each pixel receives in
expectation what the unstratified estimator gives it.  Pins: one tile
covering the panel reproduces the unstratified image bit for bit; the order-1
image with ragged tiles equals the deterministic single-scatter quadrature;
the full image agrees with the unstratified one within the noise for a
polyenergetic spectrum with more tiles than histories in its tail bins.
"""

import numpy as np
import pytest

from mc_inputs import kramers_spectrum, make_workload, mono_spectrum, slab_phantom
from mc_inputs.tables import MAT_WATER

from test_oracle_pins import BOX, BOX_GEO, _blocks, _single_scatter_quadrature


def test_one_tile_reduces_to_the_unstratified_estimator(oracle_lib, table_path, tables):
    wl = make_workload("cyl64", tables)
    a = oracle_lib.Oracle(table_path)
    a.setup(wl)
    b = oracle_lib.Oracle(table_path)
    b.setup(wl)
    g = wl["geometry"]
    b.set_tiles(g["nu"], g["nv"] + 7)
    ra = a.scatter(0.3, 20_000, wl["step_mm"], 4)
    rb = b.scatter(0.3, 20_000, wl["step_mm"], 4)
    np.testing.assert_array_equal(ra["Is"], rb["Is"])
    assert ra["stats"] == rb["stats"]


def test_tiled_order1_matches_single_scatter_quadrature(oracle_lib, table_path, tables):
    vol = slab_phantom((BOX["n"],) * 3, (BOX["dv"],) * 3, MAT_WATER, 1.0)
    o = oracle_lib.Oracle(table_path)
    o.load_volume(vol)
    o.set_spectrum(*mono_spectrum(60.0))
    o.set_geometry(**BOX_GEO)
    o.set_tiles(3, 5)  # 8 x 8 panel: 3 x 2 tiles of 3x5, 3x3, 2x5 and 2x3 pixels
    ref = _single_scatter_quadrature(tables, table_path, oracle_lib, 60.0)
    N, B = 240_000, 12
    parts = np.array([o.scatter(0.0, N, 1.0, 91, h_begin=b * N // B, h_end=(b + 1) * N // B, orders=True)["orders"][0]
                      for b in range(B)])
    est = parts.sum(axis=0)
    sig = np.sqrt(parts.var(axis=0, ddof=1) * B)
    assert np.mean(np.abs(est - ref) / sig < 3.0) >= 0.95
    rel = np.linalg.norm(est - ref) / np.linalg.norm(ref)
    assert rel < 3.0 * np.linalg.norm(sig) / np.linalg.norm(ref) + 2e-3, rel


def test_tiled_agrees_with_unstratified_polyenergetic(oracle_lib, table_path, tables):
    wl = make_workload("cyl64", tables)
    wl["energies"], wl["weights"] = kramers_spectrum(tables, kvp=90)
    N, B = 120_000, 12

    def batches(tiles, seed):
        o = oracle_lib.Oracle(table_path)
        o.setup(wl)
        if tiles:
            o.set_tiles(*tiles)
        return np.array([_blocks(o.scatter(0.5, N, wl["step_mm"], seed, h_begin=b * N // B,
                                           h_end=(b + 1) * N // B)["Is"], 16) for b in range(B)])

    pa, pb = batches(None, 5), batches((40, 24), 6)  # 128 x 128 panel: 4 x 6 ragged tiles
    se = lambda x: np.sqrt(x.var(axis=0, ddof=1) * B)
    z = np.abs(pa.sum(0) - pb.sum(0)) / np.sqrt(se(pa) ** 2 + se(pb) ** 2)
    assert np.mean(z < 3.0) >= 0.95 and z.max() < 5.0, (np.mean(z < 3.0), z.max())
    ta, tb = pa.sum(axis=(1, 2)), pb.sum(axis=(1, 2))
    sig = np.sqrt((ta.var(ddof=1) + tb.var(ddof=1)) * B)
    assert abs(tb.sum() - ta.sum()) < 4.0 * sig, (tb.sum() / ta.sum(), sig / ta.sum())


def test_bad_tiles_are_refused(oracle_lib, table_path):
    o = oracle_lib.Oracle(table_path)
    with pytest.raises(RuntimeError):
        o.set_tiles(8, 0)
    with pytest.raises(RuntimeError):
        o.set_tiles(-1, -1)
