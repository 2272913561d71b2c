"""Doppler broadening (impulse approximation) on the GPU against the oracle.

Same seed: the photons' broadened energies come from their own streams and the
point-detector energies from each pseudo-particle's side stream on both sides,
so the images must agree history for history up to a small fraction of the
noise; broadening needs the bound tables.
"""

import numpy as np
import pytest

from mc_inputs import make_workload, mono_spectrum, read_tables

from test_gpu_parity import _ctx, _orc, _same_seed_check

pytestmark = pytest.mark.gpu


def _wl(T, E=40.0):
    wl = make_workload("cyl64", T)
    wl["energies"], wl["weights"] = mono_spectrum(E)
    return wl


@pytest.mark.parametrize("nee_mode", [0, 1])
def test_doppler_same_seed_matches_oracle(gpu, oracle_lib, variant_table, nee_mode):
    tp = variant_table("bound")
    wl = _wl(read_tables(tp))
    N = 1_000_000
    c = _ctx(gpu, tp, wl, n_batches=20, doppler=1, nee_mode=nee_mode)
    out = c.project([0.7], N, wl["step_mm"], 23, primary=False, variance=True)
    g = out["scatter"][0].cpu().numpy().astype(np.float64)
    var = out["variance"][0].cpu().numpy().astype(np.float64)
    st = c.last_stats()
    o = _orc(oracle_lib, tp, wl)
    o.set_doppler(1)
    o.set_nee_mode(nee_mode)
    r = o.scatter(0.7, N, wl["step_mm"], 23)
    if nee_mode == 1:
        # judged against the noise of the paper's estimator (the expected value's own sigma is
        # smaller while an FP32 branch flip costs the same; see test_gpu_ev)
        paper = _ctx(gpu, tp, wl, n_batches=20, doppler=1)
        var = paper.project([0.7], N, wl["step_mm"], 24, primary=False, variance=True)["variance"][0]
        var = var.cpu().numpy().astype(np.float64)
    _same_seed_check(g, r["Is"], var)
    assert abs(g.sum() / r["Is"].sum() - 1.0) < 2e-3
    for k in ("compton", "rayleigh", "photo", "nee_rays"):
        assert abs(st[k] / r["stats"][k] - 1.0) < 3e-4, k
    assert st["sampler_fail"] == 0


def test_doppler_needs_bound_tables(gpu, table_path, tables):
    c = _ctx(gpu, table_path, _wl(tables), doppler=1)
    with pytest.raises(gpu.MCError, match="STATE"):
        c.project([0.0], 1000, 0.5, 1)
