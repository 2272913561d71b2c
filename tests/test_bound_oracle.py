"""Bound-electron incoherent scattering (the S(q,Z) of Sec. II-A, eq.
pmueforIncoherent) in the tables and the oracle.

The tables' normalisation integral is checked against adaptive quadrature and
its limits; the oracle's sampler (Kahn, then acceptance on S_mol/S_max) against
the density KN x S_mol by chi-square, with power against the free-electron
density; the point-detector pdf integrates to one; the order-1 image equals
the single-scatter quadrature with the bound pdf; point-detector and analog
estimators agree.
"""

import numpy as np
import pytest
from scipy import integrate

from mc_inputs import build_tables, make_workload, mono_spectrum, slab_phantom
from mc_inputs.tables import C_F, HC_KEVA, MAT_AL, MAT_WATER, MEC2_KEV, incoherent_integral, kn_shape_integral

from test_oracle_pins import BOX, BOX_GEO, _blocks, _chi2_equiprobable, _kn_density, _single_scatter_quadrature


@pytest.fixture(scope="module")
def bound(data_dir):
    from mc_inputs import default_table_path, read_tables

    p = default_table_path("bound", data_dir)
    return p, read_tables(p)


@pytest.mark.parametrize("Z", [1, 8, 13, 20])
def test_incoherent_integral_matches_adaptive_quadrature(Z):
    b = C_F * Z ** (-2.0 / 3.0)
    for E in (1.0, 10.0, 60.0, 150.0):
        K = (E / HC_KEVA) ** 2

        def f(mu):
            r = 1.0 / (1.0 + E / MEC2_KEV * (1.0 - mu))
            return r * r * (r + 1.0 / r - 1.0 + mu * mu) * Z * (1.0 - (1.0 + b * K * (1.0 - mu) / 2.0) ** -4)

        q, _ = integrate.quad(f, -1.0, 1.0, points=[1 - 1e-3, 1 - 1e-5], limit=500, epsabs=0, epsrel=1e-13)
        assert abs(incoherent_integral(Z, b, E)[0] / q - 1.0) < 1e-11


def test_incoherent_integral_limits():
    Z, b = 8.0, C_F * 8 ** (-2.0 / 3.0)
    # tightly bound at low energy (S -> 0 over the whole sphere), free at high energy
    assert incoherent_integral(Z, b, 0.05)[0] / (Z * kn_shape_integral(0.05)[0]) < 1e-3
    assert abs(incoherent_integral(Z, b, 5000.0)[0] / (Z * kn_shape_integral(5000.0)[0]) - 1.0) < 1e-4


def test_bound_tables_round_trip(bound, tables):
    p, T = bound
    assert T.I_incoh is not None and tables.I_incoh is None
    ref = build_tables(variant="bound")
    assert np.array_equal(T.I_incoh, ref.I_incoh) and np.array_equal(T.mu_incoh, ref.mu_incoh)
    # mu_incoh = pi r0^2 N_A I_incoh, and below the free-electron value
    assert np.allclose(T.mu_incoh, np.pi * T.consts["r0"] ** 2 * T.consts["N_A"] * T.I_incoh, rtol=1e-14)
    assert np.all(T.mu_incoh <= tables.mu_incoh * (1 + 1e-12))


def _smol(comps, u):
    return sum(w * Z * (1.0 - (1.0 + b * u) ** -4) for Z, w, b in comps)


@pytest.mark.parametrize("mat", [MAT_WATER, MAT_AL])
@pytest.mark.parametrize("E", [15.0, 40.0, 100.0])
def test_bound_incoherent_sampler_chi2(oracle_lib, bound, mat, E):
    p, T = bound
    o = oracle_lib.Oracle(p)
    s = o.sample_incoherent(mat, E, 600_000, seed=311 + int(E) + 5 * mat)
    K = (E / HC_KEVA) ** 2
    pdf = lambda m: _kn_density(E, m) * _smol(T.comps[mat], 0.5 * K * (1.0 - m))
    chi2, pv = _chi2_equiprobable(s, pdf, -1.0, 1.0, ngrid=2_000_001)
    assert pv > 1e-4, (mat, E, chi2)


def test_bound_sampler_detects_free_electron_density(oracle_lib, bound):
    p, _ = bound
    s = oracle_lib.Oracle(p).sample_incoherent(MAT_WATER, 15.0, 600_000, seed=5)
    _, pv = _chi2_equiprobable(s, lambda m: _kn_density(15.0, m), -1.0, 1.0)
    assert pv < 1e-6


@pytest.mark.parametrize("E", [10.0, 30.0, 80.0, 140.0])
def test_bound_nee_pdf_normalised(oracle_lib, bound, E):
    p, _ = bound
    o = oracle_lib.Oracle(p)
    for m in (MAT_WATER, MAT_AL):
        f = lambda lam: o.nee_pdf(1, m, E, lam)[0]
        q, _ = integrate.quad(f, -1.0, 1.0, points=[1 - 1e-3, 1 - 1e-5], limit=400, epsrel=1e-11)
        assert abs(q - 1.0) < 1e-9, (m, E, q)


def test_bound_single_scatter_quadrature(oracle_lib, bound):
    p, T = bound
    vol = slab_phantom((BOX["n"],) * 3, (BOX["dv"],) * 3, MAT_WATER, 1.0)
    o = oracle_lib.Oracle(p)
    o.load_volume(vol)
    o.set_spectrum(*mono_spectrum(30.0))
    o.set_geometry(**BOX_GEO)
    ref = _single_scatter_quadrature(T, p, oracle_lib, 30.0, T)
    N, B = 200_000, 10
    parts = np.array([o.scatter(0.0, N, 1.0, 83, h_begin=b * N // B, h_end=(b + 1) * N // B, orders=True)["orders"][0]
                      for b in range(B)])
    est = parts.sum(axis=0)
    sig = np.sqrt(parts.var(axis=0, ddof=1) * B)
    assert np.mean(np.abs(est - ref) / sig < 3.0) >= 0.95
    rel = np.linalg.norm(est - ref) / np.linalg.norm(ref)
    assert rel < 3.0 * np.linalg.norm(sig) / np.linalg.norm(ref) + 2e-3, rel


def test_bound_nee_matches_analog(oracle_lib, bound):
    p, T = bound
    wl = make_workload("cyl64", T)
    o = oracle_lib.Oracle(p)
    o.setup(wl)
    N, B = 200_000, 10
    nee, ana = [], []
    for b in range(B):
        r = o.scatter(0.0, N, 0.5, 12, h_begin=b * N // B, h_end=(b + 1) * N // B, analog=True)
        nee.append(_blocks(r["Is"], 32))
        ana.append(_blocks(r["analog"], 32))
    nee, ana = np.array(nee), np.array(ana)
    se = lambda x: np.sqrt(x.var(axis=0, ddof=1) * B)
    z = np.abs(nee.sum(0) - ana.sum(0)) / np.sqrt(se(nee) ** 2 + se(ana) ** 2)
    assert np.mean(z < 3.0) >= 0.9 and z.max() < 5.0, z
