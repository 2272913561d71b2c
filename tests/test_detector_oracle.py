"""Detector response eta(E) (Sec. II-D.2) in the oracle and the input model.

The oracle replaces eta(E) = E by a response table interpolated between the
table's energy nodes, in the primary sum of eq. (Ip), in the point-detector
score of eq. (Is) (at the scattered energy E') and in its analog tally.  The
pins: a table holding eta(E) = E reproduces the default; the primary of a
homogeneous box equals its closed form with the panel response; the order-1
scatter image equals the deterministic single-scatter quadrature with the
same response; and the two unbiased scatter estimators (point detector and
analog hits) still agree with it.
"""

import numpy as np
import pytest

from mc_inputs import flat_panel_response, kramers_spectrum, make_workload, mono_spectrum, slab_phantom
from mc_inputs.tables import MAT_AL, MAT_WATER, kn_energy_transfer_fraction

from test_oracle_pins import BOX, BOX_GEO, _blocks, _oracle_with, _single_scatter_quadrature


def test_kn_energy_transfer_fraction_textbook_values():
    """Mean fraction of the photon energy given to a free electron by a
    Klein-Nishina scatter: 0.0187, 0.138, 0.440, 0.683 at 0.01, 0.1, 1 and 10 MeV
    (the standard tabulation, e.g. Attix, Introduction to Radiological Physics,
    Compton-effect table)."""
    f = kn_energy_transfer_fraction([10.0, 100.0, 1000.0, 10000.0])
    assert np.allclose(f, [0.0187, 0.138, 0.440, 0.683], rtol=6e-3, atol=0)


def test_flat_panel_response_limits():
    E = np.arange(10.0, 151.0)
    eta = flat_panel_response(E)
    assert np.all(eta > 0) and np.all(eta < E)
    # a thin screen deposits linearly in its thickness; a thick bare screen keeps
    # only the interaction share mu_en/mu (no cover, everything interacts)
    t1 = flat_panel_response(E, gos_cm=1e-8, carbon_cm=0.0, al_cm=0.0)
    t2 = flat_panel_response(E, gos_cm=2e-8, carbon_cm=0.0, al_cm=0.0)
    assert np.allclose(t2 / t1, 2.0, rtol=1e-4)
    thick = flat_panel_response(E, gos_cm=100.0, carbon_cm=0.0, al_cm=0.0)
    thin = flat_panel_response(E, gos_cm=1e-10, carbon_cm=0.0, al_cm=0.0)
    # thin / (1e-10 cm * 7.32) = E mu_en ; thick = E mu_en / mu  ->  ratio = mu = mass attenuation
    from mc_inputs.detector import GOS
    from mc_inputs.tables import composition_attenuation

    pe, inc, coh = composition_attenuation(GOS, E)
    assert np.allclose(thin / (1e-10 * 7.32) / thick, pe + inc + coh, rtol=2e-6)


def test_identity_response_reproduces_default(oracle_lib, table_path, tables):
    wl = make_workload("cyl64", tables)
    a = oracle_lib.Oracle(table_path)
    a.setup(wl)
    b = oracle_lib.Oracle(table_path)
    b.setup(wl)
    b.set_detector_response(tables.energies)
    pa, _ = a.primary(0.3, 0.5)
    pb, _ = b.primary(0.3, 0.5)
    assert np.allclose(pa, pb, rtol=1e-12, atol=0)
    sa = a.scatter(0.3, 100_000, 0.5, 9, h_begin=0, h_end=2000, analog=True)
    sb = b.scatter(0.3, 100_000, 0.5, 9, h_begin=0, h_end=2000, analog=True)
    for k in ("Is", "analog", "analog0"):
        assert np.allclose(sa[k], sb[k], rtol=1e-12, atol=1e-300), k
    b.set_detector_response(None)
    assert np.array_equal(b.primary(0.3, 0.5)[0], pa)


def test_response_table_errors(oracle_lib, table_path, tables):
    o = oracle_lib.Oracle(table_path)
    with pytest.raises(RuntimeError):
        o.set_detector_response(np.ones(tables.n_E - 1))
    bad = np.ones(tables.n_E)
    bad[3] = -1.0
    with pytest.raises(RuntimeError):
        o.set_detector_response(bad)


def test_primary_closed_form_with_panel_response(oracle_lib, table_path, tables):
    vol = slab_phantom((32, 32, 32), (2.0, 2.0, 2.0), MAT_AL, 2.7)
    E, w = kramers_spectrum(tables, be_mm=0.5)
    geo = dict(sod=200.0, sdd=500.0, nu=9, nv=7, pu=3.0, pv=4.0)
    o = _oracle_with(oracle_lib, table_path, vol, (E, w), geo)
    eta_nodes = flat_panel_response(tables.energies)
    o.set_detector_response(eta_nodes)
    Ip, _ = o.primary(0.0, 0.3)
    s = np.array([200.0, 0.0, 0.0])
    c = np.array([-300.0, 0.0, 0.0])
    eu, ev = np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0])
    rho = float(np.float16(2.7))
    Ed = E.astype(np.float64)
    eta = flat_panel_response(Ed)  # the bins sit on nodes: the interpolation is exact there
    mu = np.array([tables.mu_rho_at(MAT_AL, e) for e in Ed]) * 0.1 * rho
    for j in range(7):
        for i in range(9):
            P = c + (i - 4) * 3.0 * eu + (j - 3) * 4.0 * ev
            d = np.linalg.norm(P - s)
            wv = (P - s) / d
            ta, tb = 0.0, d
            for k in range(3):
                if wv[k] != 0:
                    u, v = sorted([(-32 - s[k]) / wv[k], (32 - s[k]) / wv[k]])
                    ta, tb = max(ta, u), min(tb, v)
            ref = np.sum(w * eta * np.exp(-mu * (tb - ta))) * 12.0 * (500.0 / d) / (4 * np.pi * d * d)
            assert abs(Ip[j, i] / ref - 1.0) < 1e-11


def test_single_scatter_quadrature_with_panel_response(oracle_lib, table_path, tables):
    nodes = tables.energies
    eta_nodes = flat_panel_response(nodes)
    vol = slab_phantom((BOX["n"],) * 3, (BOX["dv"],) * 3, MAT_WATER, 1.0)
    o = oracle_lib.Oracle(table_path)
    o.load_volume(vol)
    o.set_spectrum(*mono_spectrum(60.0))
    o.set_geometry(**BOX_GEO)
    o.set_detector_response(eta_nodes)
    ref = _single_scatter_quadrature(tables, table_path, oracle_lib, 60.0,
                                     eta=lambda e: np.interp(e, nodes, eta_nodes))
    N, B = 200_000, 10
    parts = np.array([o.scatter(0.0, N, 1.0, 79, h_begin=b * N // B, h_end=(b + 1) * N // B, orders=True)["orders"][0]
                      for b in range(B)])
    est = parts.sum(axis=0)
    sig = np.sqrt(parts.var(axis=0, ddof=1) * B)
    assert np.mean(np.abs(est - ref) / sig < 3.0) >= 0.95
    rel = np.linalg.norm(est - ref) / np.linalg.norm(ref)
    assert rel < 3.0 * np.linalg.norm(sig) / np.linalg.norm(ref) + 2e-3, rel
    # the response matters: the energy-integrating image differs by far more than the noise
    plain = _single_scatter_quadrature(tables, table_path, oracle_lib, 60.0)
    assert np.linalg.norm(plain - ref) / np.linalg.norm(ref) > 10 * rel


def test_nee_matches_analog_with_panel_response(oracle_lib, table_path, tables):
    wl = make_workload("cyl64", tables)
    o = oracle_lib.Oracle(table_path)
    o.setup(wl)
    o.set_detector_response(flat_panel_response(tables.energies))
    N, B = 200_000, 10
    nee, ana = [], []
    for b in range(B):
        r = o.scatter(0.0, N, 0.5, 4, h_begin=b * N // B, h_end=(b + 1) * N // B, analog=True)
        nee.append(_blocks(r["Is"], 32))
        ana.append(_blocks(r["analog"], 32))
    nee, ana = np.array(nee), np.array(ana)
    se = lambda x: np.sqrt(x.var(axis=0, ddof=1) * B)
    z = np.abs(nee.sum(0) - ana.sum(0)) / np.sqrt(se(nee) ** 2 + se(ana) ** 2)
    assert np.mean(z < 3.0) >= 0.9 and z.max() < 5.0, z
