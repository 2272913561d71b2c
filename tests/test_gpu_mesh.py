"""Triangle-mesh (CAD) primary images on the GPU against the oracle.

The GPU casts every pixel's source ray through a bounding-volume hierarchy
with the same watertight test and half-open edge rule as the oracle's brute
force; per-material path lengths are exact, so the images must agree to FP32
rounding of the crossing parameters (1e-5 per pixel).
"""

import numpy as np
import pytest

from mc_inputs import kramers_spectrum, mono_spectrum
from mc_inputs.meshes import assemble, box_mesh, cylinder_rod_mesh, sphere_mesh
from mc_inputs.tables import MAT_AL, MAT_BONE, MAT_PMMA, MAT_WATER

pytestmark = pytest.mark.gpu


def _pair(gpu, oracle_lib, table_path, mesh, spec, geo):
    c = gpu.Context(0)
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
        c.project([0.0], 1000, 0.5, 1)  # scatter on meshes is not available
    prim = c.project([0.0], 1, 0.5, 1, scatter=False)["primary"]
    assert float(prim.min()) > 0
    v = wl["volume"]
    c.load_volume(v["mat"], v["rho"], v["spacing"])  # back to the voxel geometry
    out = c.project([0.0], 1000, 0.5, 1)
    assert float(out["scatter"].sum()) > 0
