"""Expected-value point-detector scoring in the oracle (variance reduction, Sec. II-C.1).

At every interaction the expected-value mode scores (mu_incoh/mu) x the Compton
term at E' plus (mu_coh/mu) x the Rayleigh term at E, instead of the term of
the type the photon then draws: the expectation of the paper's score over the
type draw.  Pins: its order-1 image equals the deterministic single-scatter
quadrature, its full image agrees with the paper's estimator and with analog
detector hits, and its variance per history is lower.
"""

import numpy as np

from mc_inputs import make_workload, mono_spectrum, slab_phantom
from mc_inputs.tables import MAT_WATER

from test_oracle_pins import BOX, BOX_GEO, _blocks, _single_scatter_quadrature


def test_ev_order1_matches_single_scatter_quadrature(oracle_lib, table_path, tables):
    vol = slab_phantom((BOX["n"],) * 3, (BOX["dv"],) * 3, MAT_WATER, 1.0)
    o = oracle_lib.Oracle(table_path)
    o.load_volume(vol)
    o.set_spectrum(*mono_spectrum(60.0))
    o.set_geometry(**BOX_GEO)
    o.set_nee_mode(1)
    ref = _single_scatter_quadrature(tables, table_path, oracle_lib, 60.0)
    N, B = 200_000, 10
    parts = np.array([o.scatter(0.0, N, 1.0, 81, h_begin=b * N // B, h_end=(b + 1) * N // B, orders=True)["orders"][0]
                      for b in range(B)])
    est = parts.sum(axis=0)
    sig = np.sqrt(parts.var(axis=0, ddof=1) * B)
    assert np.mean(np.abs(est - ref) / sig < 3.0) >= 0.95
    rel = np.linalg.norm(est - ref) / np.linalg.norm(ref)
    assert rel < 3.0 * np.linalg.norm(sig) / np.linalg.norm(ref) + 2e-3, rel


def _batches(o, N, B, seed, step):
    return np.array([_blocks(o.scatter(0.0, N, step, seed, h_begin=b * N // B, h_end=(b + 1) * N // B)["Is"], 16)
                     for b in range(B)])


def test_ev_agrees_with_sampled_type_and_has_lower_variance(oracle_lib, table_path, tables):
    wl = make_workload("cyl64", tables)
    N, B = 200_000, 12
    a = oracle_lib.Oracle(table_path)
    a.setup(wl)
    b = oracle_lib.Oracle(table_path)
    b.setup(wl)
    b.set_nee_mode(1)
    pa = _batches(a, N, B, 5, wl["step_mm"])
    pb = _batches(b, N, B, 6, wl["step_mm"])
    se = lambda x: np.sqrt(x.var(axis=0, ddof=1) * B)
    z = np.abs(pa.sum(0) - pb.sum(0)) / np.sqrt(se(pa) ** 2 + se(pb) ** 2)
    assert np.mean(z < 3.0) >= 0.9 and z.max() < 5.0, z.max()
    # variance per history: the expected value removes the type-draw noise
    va, vb = (se(pa) ** 2).sum(), (se(pb) ** 2).sum()
    assert vb < 0.9 * va, (vb, va)


def test_ev_matches_analog(oracle_lib, table_path, tables):
    wl = make_workload("cyl64", tables)
    o = oracle_lib.Oracle(table_path)
    o.setup(wl)
    o.set_nee_mode(1)
    N, B = 200_000, 10
    nee, ana = [], []
    for b in range(B):
        r = o.scatter(0.0, N, 0.5, 8, h_begin=b * N // B, h_end=(b + 1) * N // B, analog=True)
        nee.append(_blocks(r["Is"], 32))
        ana.append(_blocks(r["analog"], 32))
    nee, ana = np.array(nee), np.array(ana)
    se = lambda x: np.sqrt(x.var(axis=0, ddof=1) * B)
    z = np.abs(nee.sum(0) - ana.sum(0)) / np.sqrt(se(nee) ** 2 + se(ana) ** 2)
    assert np.mean(z < 3.0) >= 0.9 and z.max() < 5.0, z


def test_ev_mode_keeps_the_photon_histories(oracle_lib, table_path, tables):
    """The photon's own walk (interaction counts, energy bookkeeping) is the
    same in both modes: only the scoring differs."""
    wl = make_workload("cyl64", tables)
    a = oracle_lib.Oracle(table_path)
    a.setup(wl)
    b = oracle_lib.Oracle(table_path)
    b.setup(wl)
    b.set_nee_mode(1)
    ra = a.scatter(0.0, 50_000, 0.5, 3)
    rb = b.scatter(0.0, 50_000, 0.5, 3)
    for k in ("histories", "photo", "compton", "rayleigh", "escape", "flight_steps", "e_deposit", "e_escape"):
        assert ra["stats"][k] == rb["stats"][k], k
    assert rb["stats"]["nee_rays"] > ra["stats"]["nee_rays"]  # absorption sites are scored too
