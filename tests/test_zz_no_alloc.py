"""The scatter entry point that allocates nothing (mc_project_scatter_static).

Callers that cannot allocate device memory while running (a fixed memory
pool reserved at start-up, real-time loops that cannot afford cudaMalloc's
implicit synchronisation) call this entry point after loading their inputs.
It keeps its scratch in a fixed array inside the library; these tests check,
through the C ABI, that two calls in a row give the same images as
mc_project with the same seeds (up to the order of the FP64 tally sums), that
a call with a caller-supplied output changes neither the device's free memory
nor the caching allocator's reservation, and that requests beyond the array's
size (angles, tally pixels, staged tables) are refused.
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


def test_static_entry_allocates_nothing(gpu, table_path, tables):
    """After a first call in this context, a call with a caller-supplied
    output leaves the device's free memory and torch's reservation unchanged."""
    torch = pytest.importorskip("torch")
    wl = make_workload("cyl64", tables)
    c = _ctx(gpu, table_path, wl)
    out = torch.empty((1, c.nv, c.nu), dtype=torch.float32, device="cuda")
    c.project_scatter_static([0.2], 50_000, wl["step_mm"], 1, out=out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    res0 = torch.cuda.memory_reserved()
    c.project_scatter_static([0.9], 50_000, wl["step_mm"], 2, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_reserved() == res0
    assert free1 == free0, (free0, free1)


def test_static_entry_rejects_oversize_tables(gpu, tmp_path):
    """Eight materials on 1 keV nodes up to 300 keV: a 250 keV spectrum stages
    251 nodes, 8 x 251 x 50 + 800 > 65536 bytes, which the static table area
    refuses while mc_project accepts the same request."""
    from mc_inputs import mono_spectrum
    from mc_inputs.tables import MATERIALS, build_tables, write_tables

    mats = MATERIALS + [(f"{n}_copy", r, f) for n, r, f in MATERIALS[1:4]]
    assert len(mats) == 8
    tp = str(tmp_path / "tables8.bin")
    write_tables(build_tables(n_E=300, materials=mats), tp)
    c = gpu.Context(0)
    c.load_tables(tp)
    mat = np.zeros((8, 8, 8), np.uint8)
    mat[2:6, 2:6, 2:6] = 7
    rho = np.where(mat == 7, 2.7, 0.001205).astype(np.float16)
    c.load_volume(mat, rho, (2.0, 2.0, 2.0))
    c.set_geometry(300.0, 600.0, 16, 16, 4.0, 4.0)
    E, w = mono_spectrum(250.0)
    c.set_spectrum(E, w)
    c.project([0.0], 10_000, 1.0, 1, primary=False)
    with pytest.raises(gpu.MCError, match="INVALID_ARG"):
        c.project_scatter_static([0.0], 10_000, 1.0, 1)
    E, w = mono_spectrum(60.0)  # 61 nodes fit
    c.set_spectrum(E, w)
    c.project_scatter_static([0.0], 10_000, 1.0, 1)


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
