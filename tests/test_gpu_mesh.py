"""Triangle-mesh (CAD) geometry on the GPU against the oracle.

Primary images: the GPU casts every pixel's source ray through a bounding-
volume hierarchy with the same watertight test and half-open edge rule as the
oracle's brute force; per-material path lengths are exact, so the images must
agree to FP32 rounding of the crossing parameters (1e-5 per pixel).

Scatter: the GPU walks each flight's crossings in windows of the nearest few
while the oracle sorts them all; with the same seed both run the same
histories on the same Philox streams, so images, interaction counts and
crossing counts agree history for history up to FP32 branch flips.
"""

import numpy as np
import pytest

from mc_inputs import kramers_spectrum, mono_spectrum
from mc_inputs.meshes import assemble, box_mesh, cylinder_rod_mesh, nested_boxes_mesh, sphere_mesh
from mc_inputs.tables import MAT_AL, MAT_BONE, MAT_PMMA, MAT_WATER

pytestmark = pytest.mark.gpu


def _pair(gpu, oracle_lib, table_path, mesh, spec, geo, **opt):
    c = gpu.Context(0, **opt)
    c.load_tables(table_path)
    c.set_spectrum(*spec)
    c.set_geometry(**geo)
    c.load_mesh(mesh)
    o = oracle_lib.Oracle(table_path)
    o.load_mesh(mesh)
    o.set_spectrum(*spec)
    o.set_geometry(**geo)
    return c, o


def _check(g, ref):
    rel = np.abs(g.astype(np.float64) / ref - 1.0)
    assert rel.max() < 1e-4, rel.max()
    assert np.mean(rel <= 1e-5) >= 0.99, np.mean(rel <= 1e-5)


def test_mesh_primary_cylinder_rod(gpu, oracle_lib, table_path, tables):
    geo = dict(sod=300.0, sdd=600.0, nu=96, nv=80, pu=1.3, pv=1.7)
    c, o = _pair(gpu, oracle_lib, table_path, cylinder_rod_mesh(192), mono_spectrum(60.0), geo)
    angles = np.array([0.0, 0.37, 2.9], np.float32)
    out = c.project(angles, 1, 0.5, 1, scatter=False)["primary"].cpu().numpy()
    for k, a in enumerate(angles):
        _check(out[k], o.mesh_primary(float(a)))


def test_mesh_primary_nested_polyenergetic(gpu, oracle_lib, table_path, tables):
    vo, to = box_mesh((40.0, 35.0, 30.0))
    vs, ts = sphere_mesh(18.0, 3, center=(5.0, -4.0, 2.0))
    vi, ti = box_mesh((4.0, 4.0, 12.0), center=(-20.0, 10.0, 0.0))
    mesh = assemble([(vo, to, MAT_PMMA, 1.19, -1), (vs, ts, MAT_BONE, 1.85, 0), (vi, ti, MAT_AL, 2.7, 0)])
    geo = dict(sod=250.0, sdd=550.0, nu=64, nv=48, pu=2.6, pv=2.9)
    E, w = kramers_spectrum(tables, kvp=120, be_mm=0.5)
    c, o = _pair(gpu, oracle_lib, table_path, mesh, (E, w), geo)
    out = c.project([1.1], 1, 0.5, 1, scatter=False)["primary"][0].cpu().numpy()
    _check(out, o.mesh_primary(1.1))


def test_mesh_mode_errors_and_switch_back(gpu, table_path, tables):
    from mc_inputs import make_workload

    c = gpu.Context(0)
    c.load_tables(table_path)
    bad = cylinder_rod_mesh(32)
    bad = dict(bad, triangles=bad["triangles"].copy())
    bad["triangles"][0, 0] = len(bad["vertices"])
    with pytest.raises(gpu.MCError, match="INVALID_ARG"):
        c.load_mesh(bad)
    wl = make_workload("cyl64", tables)
    c.setup(wl)
    c.load_mesh(cylinder_rod_mesh(32))
    with pytest.raises(gpu.MCError, match="STATE"):
        c.autotune([0.0], 1000, 0.1, 0.8, 5e-3)  # the autotuner tunes the voxel march
    prim = c.project([0.0], 1, 0.5, 1, scatter=False)["primary"]
    assert float(prim.min()) > 0
    assert float(c.project([0.0], 1000, 0.5, 1)["scatter"].sum()) > 0
    v = wl["volume"]
    c.load_volume(v["mat"], v["rho"], v["spacing"])  # back to the voxel geometry
    out = c.project([0.0], 1000, 0.5, 1)
    assert float(out["scatter"].sum()) > 0


GEO_NB = dict(sod=200.0, sdd=400.0, nu=48, nv=40, pu=3.4, pv=3.2)


def _scatter_pair(gpu, oracle_lib, table_path, mesh, spec, geo, angle, N, seed, nee_mode=0, doppler=0):
    c, o = _pair(gpu, oracle_lib, table_path, mesh, spec, geo, n_batches=20, nee_mode=nee_mode, doppler=doppler)
    out = c.project([angle], N, 0.5, seed, primary=False, variance=True)
    g = out["scatter"][0].cpu().numpy().astype(np.float64)
    var = out["variance"][0].cpu().numpy().astype(np.float64)
    o.set_nee_mode(nee_mode)
    o.set_doppler(doppler)
    r = o.scatter(angle, N, 0.5, seed)
    return c, o, g, var, c.last_stats(), r


def _same_seed(g, ref, var, st, rs, frac=0.1):
    sig = np.sqrt(var)
    nz = ref > 0
    assert np.mean(np.abs(g - ref)[nz] <= frac * sig[nz] + 1e-6 * ref[nz]) >= 0.99
    assert np.linalg.norm(g - ref) <= frac * np.linalg.norm(sig)
    assert abs(g.sum() / ref.sum() - 1.0) < 2e-3
    for k in ("compton", "rayleigh", "photo", "nee_rays", "escape"):
        assert abs(st[k] / rs[k] - 1.0) < 3e-4, (k, st[k], rs[k])
    # surface crossings walked by the flights and counted by the point-detector rays
    assert abs(st["flight_steps"] / rs["flight_steps"] - 1.0) < 3e-4
    assert abs(st["nee_steps"] / rs["nee_steps"] - 1.0) < 3e-4


@pytest.mark.parametrize("angle", [0.0, 0.9])
def test_mesh_scatter_same_seed_nested_boxes(gpu, oracle_lib, table_path, tables, angle):
    """Coincident faces (the inner box shares the outer box's top face) and photons that
    start their flights inside either body."""
    c, o, g, var, st, r = _scatter_pair(gpu, oracle_lib, table_path, nested_boxes_mesh(), mono_spectrum(60.0),
                                        GEO_NB, angle, 400_000, 17)
    _same_seed(g, r["Is"], var, st, r["stats"])
    assert st["histories"] == 400_000


def test_mesh_scatter_same_seed_cylinder_rod_polyenergetic(gpu, oracle_lib, table_path, tables):
    E, w = kramers_spectrum(tables, kvp=120, be_mm=0.5)
    geo = dict(sod=300.0, sdd=600.0, nu=64, nv=56, pu=2.0, pv=2.4)
    c, o, g, var, st, r = _scatter_pair(gpu, oracle_lib, table_path, cylinder_rod_mesh(96), (E, w), geo, 0.4,
                                        150_000, 5)
    _same_seed(g, r["Is"], var, st, r["stats"])


def test_mesh_scatter_expected_value_and_doppler(gpu, oracle_lib, variant_table):
    """Expected-value scoring and Doppler broadening (bound tables) through the mesh
    geometry; judged, as on voxels, against the noise of the paper's estimator."""
    from mc_inputs import read_tables

    tp = variant_table("bound")
    mesh, spec = nested_boxes_mesh(), mono_spectrum(40.0)
    c, o, g, _, st, r = _scatter_pair(gpu, oracle_lib, tp, mesh, spec, GEO_NB, 0.3, 300_000, 41, nee_mode=1,
                                      doppler=1)
    paper = _pair(gpu, oracle_lib, tp, mesh, spec, GEO_NB, n_batches=20, doppler=1)[0]
    var = paper.project([0.3], 300_000, 0.5, 42, primary=False, variance=True)["variance"][0]
    _same_seed(g, r["Is"], var.cpu().numpy().astype(np.float64), st, r["stats"])
    assert st["sampler_fail"] == 0
    assert read_tables(tp).I_incoh is not None


def test_mesh_scatter_histories_one_by_one(gpu, oracle_lib, table_path, tables):
    """Histories recomputed one at a time agree history for history."""
    c, o = _pair(gpu, oracle_lib, table_path, nested_boxes_mesh(), mono_spectrum(60.0), GEO_NB)
    N = 10_000_000
    same = scat = 0
    for h in range(3_000_000, 3_000_400):
        g = c.project_histories([1.3], N, h, 1, 0.5, 7)[0].cpu().numpy().astype(np.float64)
        ref = o.scatter(1.3, N, 0.5, 7, h_begin=h, h_end=h + 1)["Is"]
        if ref.sum() == 0 and g.sum() == 0:
            continue
        scat += 1
        same += np.abs(g - ref).sum() / max(ref.sum(), 1e-300) < 1e-4
    assert scat >= 100, scat
    assert same >= 0.97 * scat, (same, scat)


def test_mesh_tally_modes_and_static_entry(gpu, oracle_lib, table_path, tables):
    """On meshes every tally mode is the global one (same image to FP64 order); the
    static-scratch entry point and the autotuner serve voxel volumes only."""
    mesh, spec = nested_boxes_mesh(), mono_spectrum(60.0)
    imgs = []
    for mode in (1, 3, 4):
        c, _ = _pair(gpu, oracle_lib, table_path, mesh, spec, GEO_NB, tally_mode=mode, tile_u=16, tile_v=16)
        imgs.append(c.project([0.2], 50_000, 0.5, 4, primary=False)["scatter"].cpu().numpy())
    for im in imgs[1:]:
        np.testing.assert_allclose(im, imgs[0], rtol=1e-5, atol=1e-12)
    with pytest.raises(gpu.MCError, match="STATE"):
        c.project_scatter_static([0.2], 1000, 0.5, 1)
