"""Detector response eta(E) (Sec. II-D.2) on the GPU, against the oracle.

With the flat-panel response set on both sides, the primary image (eq. Ip,
S(E_n) eta(E_n) per bin) must meet the same per-pixel bar as without it, and
the scatter image of the same histories (eq. Is, eta at the scattered energy
E') must agree with the oracle's to a small fraction of the Monte Carlo noise.
"""

import numpy as np
import pytest

from mc_inputs import flat_panel_response, kramers_spectrum, make_workload

from test_gpu_parity import _check_primary, _ctx, _orc, _same_seed_check, _small_poly_workload

pytestmark = pytest.mark.gpu


def _with_panel(wl, tables):
    wl = dict(wl)
    wl["detector_response"] = flat_panel_response(tables.energies)
    return wl


def test_primary_parity_with_panel_response(gpu, oracle_lib, table_path, tables):
    wl = _with_panel(_small_poly_workload(tables), tables)
    wl["energies"], wl["weights"] = kramers_spectrum(tables, kvp=140, be_mm=0.5)
    c = _ctx(gpu, table_path, wl)
    angles = np.array([0.3, 2.2], np.float32)
    out = c.project(angles, 1000, wl["step_mm"], 1, scatter=False)
    o = _orc(oracle_lib, table_path, wl)
    for k, a in enumerate(angles):
        Ip, bound = o.primary(float(a), wl["step_mm"])
        _check_primary(out["primary"][k].cpu().numpy(), Ip, bound, f"panel response angle {a}")


def test_scatter_same_seed_with_panel_response(gpu, oracle_lib, table_path, tables):
    wl = _with_panel(_small_poly_workload(tables), tables)
    N = 400_000
    c = _ctx(gpu, table_path, wl, n_batches=20)
    out = c.project([0.5], N, wl["step_mm"], 13, primary=False, variance=True)
    g = out["scatter"][0].cpu().numpy().astype(np.float64)
    var = out["variance"][0].cpu().numpy().astype(np.float64)
    ref = _orc(oracle_lib, table_path, wl).scatter(0.5, N, wl["step_mm"], 13)["Is"]
    _same_seed_check(g, ref, var)
    assert abs(g.sum() / ref.sum() - 1.0) < 2e-3
    # and the response changed the image: the energy-integrating one is far away
    plain = _ctx(gpu, table_path, dict(wl, detector_response=None))
    p = plain.project([0.5], N, wl["step_mm"], 13, primary=False)["scatter"][0].cpu().numpy()
    assert np.linalg.norm(p - g) > 0.2 * np.linalg.norm(g)


def test_identity_response_matches_default(gpu, table_path, tables):
    wl = make_workload("cyl64", tables)
    a = _ctx(gpu, table_path, wl)
    b = _ctx(gpu, table_path, dict(wl, detector_response=tables.energies))
    ra = a.project([0.2], 200_000, wl["step_mm"], 3)
    rb = b.project([0.2], 200_000, wl["step_mm"], 3)
    for k in ("primary", "scatter"):
        x, y = ra[k].cpu().numpy(), rb[k].cpu().numpy()
        assert np.allclose(x, y, rtol=2e-6, atol=1e-6 * np.abs(x).max()), k


def test_response_errors(gpu, table_path, tables):
    c = gpu.Context(0)
    with pytest.raises(gpu.MCError, match="STATE"):
        c.set_detector_response(np.ones(tables.n_E))
    c.load_tables(table_path)
    with pytest.raises(gpu.MCError, match="INVALID_ARG"):
        c.set_detector_response(np.ones(tables.n_E + 1))
    bad = np.ones(tables.n_E)
    bad[0] = np.nan
    with pytest.raises(gpu.MCError, match="INVALID_ARG"):
        c.set_detector_response(bad)
    c.set_detector_response(None)
