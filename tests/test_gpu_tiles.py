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


def test_tiled_full_size_ell256_16x16(gpu, oracle_lib, table_path, tables):
    """The bench's tile-stratified side run (ell256: 256^3, 512^2, 1e8 photons, 16x16 tiles): histories from
    the middle of the run, recomputed one by one on both sides, match history for history; a 4000-history
    block agrees to a small fraction of its noise."""
    wl = make_workload("ell256", tables)
    N = wl["n_photons"]
    c = _ctx(gpu, table_path, wl, tally_mode=4, tile_u=16, tile_v=16)
    o = _orc(oracle_lib, table_path, wl)
    o.set_tiles(16, 16)
    h0 = 41_000_000
    same, close, scat = 0, 0, 0
    for h in range(h0, h0 + 200):
        g = c.project_histories([0.0], N, h, 1, wl["step_mm"], wl["seed"])[0].cpu().numpy().astype(np.float64)
        ref = o.scatter(0.0, N, wl["step_mm"], wl["seed"], h_begin=h, h_end=h + 1)["Is"]
        if ref.sum() == 0 and g.sum() == 0:
            continue
        scat += 1
        l1 = np.abs(g - ref).sum() / ref.sum()
        same += l1 < 1e-4
        close += l1 < 1e-2  # a midpoint within rounding of a voxel face may see the neighbouring voxel
    assert scat >= 20, scat
    assert same >= 0.8 * scat and close >= 0.95 * scat, (same, close, scat)
    cnt = 4000
    g = c.project_histories([0.0], N, h0, cnt, wl["step_mm"], wl["seed"])[0].cpu().numpy().astype(np.float64)
    ref = o.scatter(0.0, N, wl["step_mm"], wl["seed"], h_begin=h0, h_end=h0 + cnt)["Is"]
    parts = np.array([o.scatter(0.0, N, wl["step_mm"], wl["seed"] + 1, h_begin=h0 + b * cnt // 10,
                                h_end=h0 + (b + 1) * cnt // 10)["Is"] for b in range(10)])
    var = parts.var(axis=0, ddof=1) * 10
    assert np.linalg.norm(g - ref) <= 0.2 * np.linalg.norm(np.sqrt(var))
