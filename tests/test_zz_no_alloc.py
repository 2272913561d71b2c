"""The scatter entry point that allocates nothing (mc_project_scatter_static).

Callers that cannot allocate device memory while running (a fixed memory
pool reserved at start-up, real-time loops that cannot afford cudaMalloc's
implicit synchronisation) call this entry point after loading their inputs.
It keeps its scratch in a fixed array inside the library; these tests check,
through the C ABI, that two calls in a row give the same images as
mc_project with the same seeds (up to the order of the FP64 tally sums) and
that requests beyond the array's size are refused.
"""

import numpy as np
import pytest

from mc_inputs import make_workload

pytestmark = pytest.mark.gpu


def _ctx(gpu, table_path, wl):
    c = gpu.Context(0)
    c.load_tables(table_path)
    c.setup(wl)
    return c


def test_static_entry_matches_mc_project_twice(gpu, table_path, tables):
    torch = pytest.importorskip("torch")
    wl = make_workload("cyl64", tables)
    c = _ctx(gpu, table_path, wl)
    angles = np.array([0.3, 1.7], np.float32)
    out = torch.empty((2, c.nv, c.nu), dtype=torch.float32, device="cuda")
    for seed in (5, 6):  # two calls in a row on the shared array
        ref = c.project(angles, 200_000, wl["step_mm"], seed, primary=False)["scatter"].cpu().numpy()
        ref_stats = c.last_stats()
        out.fill_(-1.0)
        got = c.project_scatter_static(angles, 200_000, wl["step_mm"], seed, out=out)
        st = c.last_stats()
        np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=1e-5, atol=1e-12)
        for k in ("histories", "flight_steps", "nee_steps", "compton", "rayleigh", "photo"):
            assert st[k] == ref_stats[k], k


def test_static_entry_polyenergetic(gpu, table_path, tables):
    wl = make_workload("ell256", tables)
    c = _ctx(gpu, table_path, wl)
    ref = c.project([0.0], 2_000_000, wl["step_mm"], 3, primary=False)["scatter"].cpu().numpy()
    got = c.project_scatter_static([0.0], 2_000_000, wl["step_mm"], 3).cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-12)


def test_static_entry_rejects_oversize(gpu, table_path, tables):
    wl = make_workload("cyl64", tables)
    c = _ctx(gpu, table_path, wl)
    with pytest.raises(gpu.MCError, match="INVALID_ARG"):
        c.project_scatter_static(np.zeros(5000, np.float32), 100, wl["step_mm"], 1)  # > 4096 angles
    with pytest.raises(gpu.MCError, match="INVALID_ARG"):
        c.project_scatter_static(np.zeros(257, np.float32), 100, wl["step_mm"], 1)  # 257 x 128^2 > 4194304
    fresh = gpu.Context(0)
    with pytest.raises(gpu.MCError, match="STATE"):
        fresh.project_scatter_static([0.0], 100, 0.5, 1)
