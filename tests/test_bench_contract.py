"""The reference arm of bench.py runs on the host cores (CPU only) and prints one JSON
line with the keys the benchmark contract names."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line(tmp_path):
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "histories/s"
    assert line["config"]["workload"] == "ell256"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_reference_arm_reports_march_steps():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--workload", "cyl64"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    cb = json.loads(r.stdout.strip().splitlines()[-1])["cpu_baseline"]
    # every history marches at least a flight step, and the oracle counts them exactly
    assert cb["steps_per_s"] > cb["value"]


def test_recorded_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    """The per-step traffic is read from a profile line only while its hash is that of the current transport
    sources and flags, and only for its own workload; the branch-efficiency field is optional."""
    sys.path.insert(0, ROOT)
    import bench

    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "transport_source_hash", lambda: "abc123")
    (prof / "k_transport_w1.md").write_text(
        "text\ntraffic-per-step: kernel=abc123 workload=w1 dram_bytes=0.5 l2_bytes=6.0 simt_lanes=16\n")
    (prof / "k_transport_w2_extra.md").write_text(
        "traffic-per-step: kernel=stale00 workload=w2 dram_bytes=1 l2_bytes=2\n"
        "traffic-per-step: kernel=abc123 workload=w2 dram_bytes=3 l2_bytes=4\n")
    assert bench.recorded_traffic("w1") == (0.5, 6.0, 16.0)
    d, l2, simt = bench.recorded_traffic("w2")
    assert (d, l2) == (3.0, 4.0) and simt != simt  # no simt field: NaN
    assert bench.recorded_traffic("w3") is None
    (prof / "k_transport_w1.md").write_text("traffic-per-step: kernel=other workload=w1 dram_bytes=0.5 l2_bytes=6\n")
    assert bench.recorded_traffic("w1") is None


def test_spread_blocks_cover_the_history_range():
    sys.path.insert(0, ROOT)
    import bench

    N, blk = 1_000_000, 512
    for phase in (0.0, 0.25, 0.99):
        starts = bench.spread_blocks(N, 64, blk, phase)
        assert len(starts) == 64 and starts == sorted(starts)
        assert all(0 <= b <= N - blk for b in starts)
        # evenly spread: every sixteenth of the range holds four block starts
        counts = [sum(1 for b in starts if k * N // 16 <= b < (k + 1) * N // 16) for k in range(16)]
        assert min(counts) >= 3 and max(counts) <= 5, counts
