"""Doppler broadening of incoherent scattering in the oracle (impulse
approximation with the orbital model behind the form factor; Sec. II-A names
bound-electron effects through S(q,Z), broadening completes them).

Pins: at a fixed angle the sampled E'/E follows the density obtained by
changing variables in the Compton profiles, sum_i w_i S_i(x) J_i(p_z(tau))
|dp_z/dtau| (chi-square, independent of the sampler's root solving), with
power against the unbroadened line; point-detector and analog estimators agree
with broadening on; energy is conserved history by history.
"""

import numpy as np
import pytest

from mc_inputs import make_workload, mono_spectrum
from mc_inputs.tables import HC_KEVA, MAT_AL, MAT_WATER, MEC2_KEV

from test_oracle_pins import _blocks, _chi2_equiprobable

ALPHA = 1.0 / 137.035999084
A0 = 0.529177210903


@pytest.fixture(scope="module")
def bound(data_dir):
    from mc_inputs import default_table_path, read_tables

    p = default_table_path("bound", data_dir)
    return p, read_tables(p)


def _tau_density(comps, E, c):
    """Unnormalised density of tau = E'/E on a grid, from the profiles by change of variables."""
    kappa = E / MEC2_KEV
    a = 1.0 + kappa * (1.0 - c)
    u = 0.5 * (E / HC_KEVA) ** 2 * (1.0 - c)

    def pdf(tau):
        tau = np.asarray(tau, dtype=np.float64)
        root = np.sqrt(1.0 + tau * tau - 2.0 * tau * c)
        P = (a * tau - 1.0) / root                       # p_z / (m_e c)
        dP = (a * root - (a * tau - 1.0) * (tau - c) / root) / (root * root)
        f = np.zeros_like(tau)
        for Z, w, b in comps:
            zeta = 2.0 * np.pi * A0 / np.sqrt(b)
            pz = P / ALPHA                                # atomic units
            J = 8.0 / (3.0 * np.pi * zeta) * (1.0 + (pz / zeta) ** 2) ** -3
            S = w * Z * (1.0 - (1.0 + b * u) ** -4)
            f += S * J * np.abs(dP) / ALPHA
        return f

    return pdf, 1.0 / a


@pytest.mark.parametrize("mat", [MAT_WATER, MAT_AL])
@pytest.mark.parametrize("E,c", [(30.0, 0.0), (60.0, -0.5), (100.0, 0.6)])
def test_doppler_energy_distribution(oracle_lib, bound, mat, E, c):
    p, T = bound
    o = oracle_lib.Oracle(p)
    tau = o.sample_doppler(mat, E, c, 400_000, seed=71 + int(E) + 3 * mat)
    pdf, tc = _tau_density(T.comps[mat], E, c)
    assert tau.min() > 0 and tau.max() <= 1.0
    lo, hi = max(1e-6, tau.min() * 0.999), 1.0
    chi2, pv = _chi2_equiprobable(tau, pdf, lo, hi, ngrid=2_000_001)
    assert pv > 1e-4, (mat, E, c, chi2)
    # the line is broadened around the Compton energy, not shifted far from it
    assert abs(np.median(tau) / tc - 1.0) < 0.01
    assert np.std(tau) > 1e-3 * tc


def test_doppler_detects_the_unbroadened_line(oracle_lib, bound):
    p, T = bound
    tau = oracle_lib.Oracle(p).sample_doppler(MAT_WATER, 60.0, 0.0, 200_000, seed=3)
    tc = 1.0 / (1.0 + 60.0 / MEC2_KEV)
    # a narrow line of the same mean is rejected: the sample really is broadened
    assert np.mean(np.abs(tau - tc) > 0.002 * tc) > 0.3


def test_doppler_needs_bound_tables(oracle_lib, table_path):
    o = oracle_lib.Oracle(table_path)
    with pytest.raises(RuntimeError):
        o.set_doppler(1)


def test_doppler_nee_matches_analog_and_conserves_energy(oracle_lib, bound):
    p, T = bound
    wl = make_workload("cyl64", T)
    wl["energies"], wl["weights"] = mono_spectrum(40.0)
    o = oracle_lib.Oracle(p)
    o.setup(wl)
    o.set_doppler(1)
    N, B = 200_000, 10
    nee, ana = [], []
    worst = 0.0
    for b in range(B):
        r = o.scatter(0.0, N, 0.5, 21, h_begin=b * N // B, h_end=(b + 1) * N // B, analog=True)
        nee.append(_blocks(r["Is"], 32))
        ana.append(_blocks(r["analog"], 32))
        worst = max(worst, r["stats"]["max_energy_error"])
        assert r["stats"]["sampler_fail"] == 0
    assert worst < 1e-12
    nee, ana = np.array(nee), np.array(ana)
    se = lambda x: np.sqrt(x.var(axis=0, ddof=1) * B)
    z = np.abs(nee.sum(0) - ana.sum(0)) / np.sqrt(se(nee) ** 2 + se(ana) ** 2)
    assert np.mean(z < 3.0) >= 0.9 and z.max() < 5.0, z
