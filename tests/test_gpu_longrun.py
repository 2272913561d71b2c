"""Chunked long run on the GPU: the sum of chunk images from mc_project_histories,
checkpointed and resumed, equals the one-call projection up to the order of the
FP64 additions (rounded to the FP32 outputs)."""

import numpy as np
import pytest

from mc_inputs import make_workload

from paper_2201_13191_gb300.longrun import run_chunks
from test_gpu_parity import _ctx

pytestmark = pytest.mark.gpu


def test_gpu_chunks_resume_to_the_one_call_image(gpu, table_path, tables, tmp_path):
    wl = make_workload("cyl64", tables)
    N, chunk = 1_000_000, 300_000
    c = _ctx(gpu, table_path, wl)
    runner = lambda h0, cnt: c.project_histories([0.6], N, h0, cnt, wl["step_mm"], 21)[0].double().cpu().numpy()
    ck = str(tmp_path / "ck.npz")
    part, n1 = run_chunks(runner, N, chunk, meta={"seed": 21}, checkpoint=ck, stop_after=2)
    assert part is None and n1 == 2
    total, n2 = run_chunks(runner, N, chunk, meta={"seed": 21}, checkpoint=ck)
    assert n2 == 4
    one = c.project([0.6], N, wl["step_mm"], 21, primary=False)["scatter"][0].double().cpu().numpy()
    np.testing.assert_allclose(total, one, rtol=2e-6, atol=1e-9 * np.abs(one).max())
