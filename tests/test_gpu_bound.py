"""Bound-electron incoherent scattering (S(q,Z), Sec. II-A) on the GPU against the oracle.

With the 'bound' tables both sides sample incoherent angles by Kahn's method
plus acceptance on S_mol and score KN x S_mol / I_incoh: same-seed scatter
images must agree history for history up to a small fraction of the noise,
and the primary (which sees the smaller incoherent attenuation) must meet the
usual per-pixel bar.
"""

import numpy as np
import pytest

from mc_inputs import make_workload, mono_spectrum, read_tables

from test_gpu_parity import _check_primary, _ctx, _orc, _same_seed_check

pytestmark = pytest.mark.gpu


def _low_energy_cylinder(T):
    wl = make_workload("cyl64", T)
    wl["energies"], wl["weights"] = mono_spectrum(30.0)  # where S(x, Z) matters
    return wl


def test_bound_same_seed_matches_oracle(gpu, oracle_lib, variant_table):
    tp = variant_table("bound")
    T = read_tables(tp)
    wl = _low_energy_cylinder(T)
    N = 1_000_000
    c = _ctx(gpu, tp, wl, n_batches=20)
    out = c.project([0.3], N, wl["step_mm"], 17, primary=False, variance=True)
    g = out["scatter"][0].cpu().numpy().astype(np.float64)
    var = out["variance"][0].cpu().numpy().astype(np.float64)
    st = c.last_stats()
    r = _orc(oracle_lib, tp, wl).scatter(0.3, N, wl["step_mm"], 17)
    _same_seed_check(g, r["Is"], var)
    assert abs(g.sum() / r["Is"].sum() - 1.0) < 2e-3
    for k in ("compton", "rayleigh", "photo", "nee_rays"):
        assert abs(st[k] / r["stats"][k] - 1.0) < 3e-4, k
    assert st["sampler_fail"] == 0


def test_bound_primary_parity(gpu, oracle_lib, variant_table):
    tp = variant_table("bound")
    wl = _low_energy_cylinder(read_tables(tp))
    c = _ctx(gpu, tp, wl)
    out = c.project([0.9], 1000, wl["step_mm"], 1, scatter=False)
    Ip, bound = _orc(oracle_lib, tp, wl).primary(0.9, wl["step_mm"])
    _check_primary(out["primary"][0].cpu().numpy(), Ip, bound, "bound tables", min_strict=0.99)


def test_bound_changes_the_scatter(gpu, table_path, tables, variant_table):
    """At 30 keV the scattering function removes forward incoherent scatter: the
    total scatter on the panel drops (by about 9% for this cylinder), far beyond
    the noise of either image."""
    tp = variant_table("bound")
    N = 4_000_000

    def run(path, T):
        c = _ctx(gpu, path, _low_energy_cylinder(T), n_batches=20)
        o = c.project([0.0], N, 0.5, 3, primary=False, variance=True)
        return float(o["scatter"][0].double().sum()), float(o["variance"][0].double().sum())

    sb, vb = run(tp, read_tables(tp))
    sf, vf = run(table_path, tables)
    assert sf - sb > 4.0 * np.sqrt(vb + vf), (sb, sf, vb, vf)
