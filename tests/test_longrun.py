"""Chunked long runs: checkpoint/resume and recovery from a dead worker (CPU, oracle).

Histories are keyed by index, so any partition of the run into history ranges
sums to the same image; with the deterministic oracle as the range runner an
interrupted-and-resumed run, and a run whose worker died, give the
uninterrupted total bit for bit.
"""

import os

import numpy as np
import pytest

from paper_2201_13191_gb300.longrun import chunk_ranges, run_chunks, run_workers

N, CHUNK, STEP, SEED = 9_000, 2_000, 0.5, 13


def _make_runner():
    from mc_inputs import default_table_path, make_workload, read_tables

    import oracle

    tp = default_table_path("full", os.environ["MC_TEST_DATA"])
    wl = make_workload("tiny8", read_tables(tp))
    o = oracle.Oracle(tp)
    o.setup(wl)
    return lambda h0, cnt: o.scatter(0.3, N, STEP, SEED, h_begin=h0, h_end=h0 + cnt)["Is"]


@pytest.fixture()
def runner_env(table_path, oracle_lib, monkeypatch):
    monkeypatch.setenv("MC_TEST_DATA", os.path.dirname(table_path))
    return _make_runner()


def test_chunk_ranges():
    assert chunk_ranges(9_000, 2_000) == [(0, 2000), (2000, 2000), (4000, 2000), (6000, 2000), (8000, 1000)]
    assert chunk_ranges(0, 5) == []
    with pytest.raises(ValueError):
        chunk_ranges(10, 0)


def test_resume_is_bit_identical(runner_env, tmp_path):
    ref, n = run_chunks(runner_env, N, CHUNK, meta={"seed": SEED})
    assert n == 5
    # the chunk sum is the one-range image up to FP64 rounding
    whole = runner_env(0, N)
    assert np.allclose(ref, whole, rtol=1e-12, atol=1e-12 * np.abs(whole).max())
    ck = str(tmp_path / "run.npz")
    part, n1 = run_chunks(runner_env, N, CHUNK, meta={"seed": SEED}, checkpoint=ck, stop_after=2)
    assert part is None and n1 == 2
    # interrupted again without progress, then resumed to the end
    total, n2 = run_chunks(runner_env, N, CHUNK, meta={"seed": SEED}, checkpoint=ck)
    assert n2 == 5
    np.testing.assert_array_equal(total, ref)
    with pytest.raises(ValueError):
        run_chunks(runner_env, N, CHUNK, meta={"seed": SEED + 1}, checkpoint=ck)


def test_dead_worker_is_recovered(runner_env, tmp_path):
    ref, _ = run_chunks(runner_env, N, CHUNK)
    total, failed = run_workers(_make_runner, N, CHUNK, str(tmp_path / "work"), world=2, die_after={1: 1})
    assert failed == [1]
    np.testing.assert_array_equal(total, ref)
