"""Triangle-mesh (CAD) geometry in the oracle: closed-form pins.

A box is exactly its triangulation, so the primary of a mesh box must equal
the Beer-Lambert closed form to rounding, also for a box nested in another
(the inner material replaces the outer one) and for rays aimed exactly at the
diagonal edges shared by two triangles (the watertight half-open edge rule
counts each crossing once).  A tessellated cylinder converges to the analytic
cylinder as the tessellation is refined.
"""

import numpy as np

from mc_inputs import kramers_spectrum, mono_spectrum
from mc_inputs.meshes import assemble, box_mesh, cylinder_mesh, cylinder_rod_mesh
from mc_inputs.tables import MAT_AL, MAT_BONE, MAT_WATER


def _oracle(oracle_lib, table_path, mesh, spec, geo):
    o = oracle_lib.Oracle(table_path)
    o.load_mesh(mesh)
    o.set_spectrum(*spec)
    o.set_geometry(**geo)
    return o


def _rays(geo, beta):
    s = geo["sod"] * np.array([np.cos(beta), np.sin(beta), 0.0])
    c = (geo["sod"] - geo["sdd"]) * np.array([np.cos(beta), np.sin(beta), 0.0])
    eu, ev = np.array([-np.sin(beta), np.cos(beta), 0.0]), np.array([0.0, 0.0, 1.0])
    for j in range(geo["nv"]):
        for i in range(geo["nu"]):
            P = c + (i + 0.5 - geo["nu"] / 2) * geo["pu"] * eu + (j + 0.5 - geo["nv"] / 2) * geo["pv"] * ev
            d = np.linalg.norm(P - s)
            yield j, i, s, (P - s) / d, d


def _box_chord(s, w, lo, hi):
    ta, tb = 0.0, np.inf
    for k in range(3):
        if w[k] != 0:
            u, v = sorted([(lo[k] - s[k]) / w[k], (hi[k] - s[k]) / w[k]])
            ta, tb = max(ta, u), min(tb, v)
        elif not (lo[k] <= s[k] <= hi[k]):
            return 0.0
    return max(0.0, tb - ta)


def test_box_mesh_primary_closed_form(oracle_lib, table_path, tables):
    v, t = box_mesh((30.0, 25.0, 20.0))
    mesh = assemble([(v, t, MAT_AL, 2.7, -1)])
    E, w = kramers_spectrum(tables)
    geo = dict(sod=200.0, sdd=500.0, nu=11, nv=9, pu=3.0, pv=4.0)
    o = _oracle(oracle_lib, table_path, mesh, (E, w), geo)
    rho = float(np.float32(2.7))
    mu = np.array([tables.mu_rho_at(MAT_AL, e) for e in E.astype(np.float64)]) * 0.1 * rho
    for beta in (0.0, 0.4):
        b32 = float(np.float32(beta))
        Ip = o.mesh_primary(beta)
        for j, i, s, wv, d in _rays(geo, b32):
            L = _box_chord(s, wv, (-30, -25, -20), (30, 25, 20))
            ref = np.sum(w * E * np.exp(-mu * L)) * 12.0 * (500.0 / d) / (4 * np.pi * d * d)
            assert abs(Ip[j, i] / ref - 1.0) < 1e-11, (beta, j, i)


def test_nested_boxes_replace_the_parent_material(oracle_lib, table_path, tables):
    vo, to = box_mesh((30.0, 30.0, 30.0))
    vi, ti = box_mesh((10.0, 8.0, 6.0), center=(3.0, -2.0, 1.0))
    mesh = assemble([(vo, to, MAT_WATER, 1.0, -1), (vi, ti, MAT_BONE, 1.85, 0)])
    geo = dict(sod=200.0, sdd=450.0, nu=13, nv=11, pu=2.5, pv=2.5)
    E, w = mono_spectrum(50.0)
    o = _oracle(oracle_lib, table_path, mesh, (E, w), geo)
    mw = tables.mu_rho_at(MAT_WATER, 50.0) * 0.1 * float(np.float32(1.0))
    mb = tables.mu_rho_at(MAT_BONE, 50.0) * 0.1 * float(np.float32(1.85))
    Ip = o.mesh_primary(0.3)
    for j, i, s, wv, d in _rays(geo, float(np.float32(0.3))):
        Lo = _box_chord(s, wv, (-30, -30, -30), (30, 30, 30))
        Li = _box_chord(s, wv, (-7.0, -10.0, -5.0), (13.0, 6.0, 7.0))
        ref = 50.0 * np.exp(-mw * (Lo - Li) - mb * Li) * 2.5 * 2.5 * (450.0 / d) / (4 * np.pi * d * d)
        assert abs(Ip[j, i] / ref - 1.0) < 1e-11


def test_rays_through_shared_edges_count_once(oracle_lib, table_path, tables):
    """Pixels whose rays pass exactly through the diagonals (and the corners) of
    the box faces, the edges two triangles share."""
    v, t = box_mesh((20.0, 20.0, 20.0))
    mesh = assemble([(v, t, MAT_WATER, 1.0, -1)])
    # source on the x axis, panel pixels on a grid that contains the face diagonals' images
    geo = dict(sod=100.0, sdd=200.0, nu=9, nv=9, pu=10.0, pv=10.0)
    o = _oracle(oracle_lib, table_path, mesh, mono_spectrum(60.0), geo)
    Ip = o.mesh_primary(0.0)
    mu = tables.mu_rho_at(MAT_WATER, 60.0) * 0.1
    for j, i, s, wv, d in _rays(geo, 0.0):
        L = _box_chord(s, wv, (-20, -20, -20), (20, 20, 20))
        ref = 60.0 * np.exp(-mu * L) * 100.0 * (200.0 / d) / (4 * np.pi * d * d)
        assert abs(Ip[j, i] / ref - 1.0) < 1e-11, (j, i, L)


def test_tessellated_cylinder_converges(oracle_lib, table_path, tables):
    geo = dict(sod=300.0, sdd=600.0, nu=32, nv=4, pu=3.5, pv=8.0)
    E, w = mono_spectrum(60.0)
    mu = tables.mu_rho_at(MAT_WATER, 60.0) * 0.1
    errs = []
    for n_seg in (32, 128, 512):
        v, t = cylinder_mesh(25.0, 60.0, n_seg)
        o = _oracle(oracle_lib, table_path, assemble([(v, t, MAT_WATER, 1.0, -1)]), (E, w), geo)
        Ip = o.mesh_primary(0.0)
        e = []
        for j, i, s, wv, d in _rays(geo, 0.0):
            # analytic chord through the infinite-height cylinder x^2 + y^2 <= 25^2 (|z| stays < 30 here)
            a = wv[0] ** 2 + wv[1] ** 2
            b = 2 * (s[0] * wv[0] + s[1] * wv[1])
            cc = s[0] ** 2 + s[1] ** 2 - 625.0
            disc = b * b - 4 * a * cc
            L = np.sqrt(disc) / a if disc > 0 else 0.0
            ref = 60.0 * np.exp(-mu * L) * 3.5 * 8.0 * (600.0 / d) / (4 * np.pi * d * d)
            e.append(abs(Ip[j, i] / ref - 1.0))
        errs.append(max(e))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 2e-4, errs


def test_cylinder_rod_mesh_close_to_the_voxel_phantom(oracle_lib, table_path, tables):
    from mc_inputs import make_workload

    wl = make_workload("cyl64", tables)
    ov = oracle_lib.Oracle(table_path)
    ov.setup(wl)
    om = _oracle(oracle_lib, table_path, cylinder_rod_mesh(256), (wl["energies"], wl["weights"]), wl["geometry"])
    iv, _ = ov.primary(0.0, 0.1)
    im = om.mesh_primary(0.0)
    # voxelisation at 1 mm: the line integrals differ by a few per cent at most, mostly at edges
    la, lb = -np.log(iv / iv.max()), -np.log(im / im.max())
    assert np.median(np.abs(la - lb)) < 0.01 and np.abs(la - lb).max() < 0.35
