"""Tile-stratified tally on the GPU against the oracle.

With the same seed and the same tiles both sides aim each history's
pseudo-particles at the same tile (the per-angle offset comes from the same
Philox block) and the same pixels, so the images agree history for history;
the GPU accumulates each tile in shared memory chunk by chunk.
"""

import numpy as np
import pytest

from mc_inputs import kramers_spectrum, make_workload

from test_gpu_parity import _ctx, _orc, _same_seed_check

pytestmark = pytest.mark.gpu

TILES = (40, 24)  # 128 x 128 panel: 4 x 6 tiles, ragged in both directions


def test_tiled_same_seed_matches_oracle(gpu, oracle_lib, table_path, tables):
    wl = make_workload("cyl64", tables)
    N = 1_000_000
    c = _ctx(gpu, table_path, wl, n_batches=10, tally_mode=4, tile_u=TILES[0], tile_v=TILES[1])
    out = c.project([0.4], N, wl["step_mm"], 9, primary=False, variance=True)
    g = out["scatter"][0].cpu().numpy().astype(np.float64)
    var = out["variance"][0].cpu().numpy().astype(np.float64)
    st = c.last_stats()
    o = _orc(oracle_lib, table_path, wl)
    o.set_tiles(*TILES)
    r = o.scatter(0.4, N, wl["step_mm"], 9)
    _same_seed_check(g, r["Is"], var)
    assert abs(g.sum() / r["Is"].sum() - 1.0) < 2e-3
    for k in ("histories", "compton", "rayleigh", "photo", "nee_rays"):
        assert abs(st[k] / r["stats"][k] - 1.0) < 3e-4, k


def test_tiled_history_ranges_and_angles(gpu, oracle_lib, table_path, tables):
    """Sub-ranges of a polyenergetic run over two angles: each angle has its own
    tile offset, and a range's histories keep the tiles they have in the whole run."""
    wl = make_workload("cyl64", tables)
    wl["energies"], wl["weights"] = kramers_spectrum(tables, kvp=90)
    N = 2_000_000
    c = _ctx(gpu, table_path, wl, tally_mode=4, tile_u=TILES[0], tile_v=TILES[1])
    o = _orc(oracle_lib, table_path, wl)
    o.set_tiles(*TILES)
    for h0, cnt in ((0, 3000), (1_234_567, 2500)):
        g = c.project_histories([0.2, 2.5], N, h0, cnt, wl["step_mm"], 31).cpu().numpy().astype(np.float64)
        for k, ang in enumerate((0.2, 2.5)):
            ref = o.scatter(ang, N, wl["step_mm"], 31, h_begin=h0, h_end=h0 + cnt, angle_index=k)["Is"]
            assert np.abs(g[k] - ref).sum() <= 5e-3 * ref.sum(), (h0, k)


def test_tiled_mode_limits(gpu, table_path, tables):
    wl = make_workload("cyl64", tables)
    c = _ctx(gpu, table_path, wl, n_batches=20, tally_mode=4, tile_u=64, tile_v=64)
    with pytest.raises(gpu.MCError, match="INVALID_ARG"):
        c.project([0.0], 100_000, 0.5, 1, primary=False, variance=True)  # 20 x 64 x 64 > 12288
    with pytest.raises(gpu.MCError, match="INVALID_ARG"):
        _ctx(gpu, table_path, wl, tile_u=0)
    # one tile covering the panel: the same image as the global tally up to summation order
    wl = make_workload("tiny8", tables)
    one = _ctx(gpu, table_path, wl, tally_mode=4, tile_u=8, tile_v=9)
    ref = _ctx(gpu, table_path, wl, tally_mode=1)
    a = one.project([0.3], 200_000, 0.5, 3, primary=False)["scatter"].cpu().numpy()
    b = ref.project([0.3], 200_000, 0.5, 3, primary=False)["scatter"].cpu().numpy()
    np.testing.assert_allclose(a, b, rtol=2e-5, atol=1e-12)
