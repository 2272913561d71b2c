"""Multi-rank path on CPU (gloo, world size 2).

Each rank scores its contiguous range of histories (here with the oracle, the
same history-range interface the GPU path exposes through
mc_project_histories); the FP64 sum of the partial images equals the image of
the whole range on one process, up to the order of the FP64 additions; the
job time is the maximum over ranks.
"""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2201_13191_gb300.shard import angle_range, history_range


def test_ranges_partition():
    for n in (0, 1, 7, 1000, 10**9 + 7):
        for world in (1, 2, 3, 8):
            spans = [history_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0
            for (b0, c0), (b1, _) in zip(spans, spans[1:]):
                assert b0 + c0 == b1
            assert sum(c for _, c in spans) == n
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    assert angle_range(360, 3, 8) == (135, 45)
    with pytest.raises(ValueError):
        history_range(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, table_path, n, out_dir):
    import torch
    import torch.distributed as dist

    from mc_inputs import make_workload, read_tables
    from paper_2201_13191_gb300.shard import history_range, max_time, reduce_images

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = make_workload("cyl64", read_tables(table_path))
    o = oracle.Oracle(table_path)
    o.setup(wl)
    h0, cnt = history_range(n, rank, world)
    img = o.scatter(0.0, n, wl["step_mm"], 5, h_begin=h0, h_end=h0 + cnt)["Is"]
    tot = reduce_images(torch.from_numpy(img))
    t = max_time(0.25 + rank)
    if rank == 0:
        np.save(os.path.join(out_dir, "sum.npy"), tot.numpy())
        np.save(os.path.join(out_dir, "tmax.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_history_sharding_reduces_to_the_single_process_image(table_path, tables, oracle_lib, tmp_path):
    n = 6000
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, table_path, n, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    wl = make_workload_cyl(tables)
    o = oracle_lib.Oracle(table_path)
    o.setup(wl)
    ref = o.scatter(0.0, n, wl["step_mm"], 5)["Is"]
    got = np.load(tmp_path / "sum.npy")
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    assert float(np.load(tmp_path / "tmax.npy")[0]) == 1.25


def make_workload_cyl(tables):
    from mc_inputs import make_workload

    return make_workload("cyl64", tables)


def _angle_worker(rank, world, port, table_path, n_ang, n, out_dir):
    import torch
    import torch.distributed as dist

    from mc_inputs import make_workload, read_tables
    from paper_2201_13191_gb300.shard import angle_range, reduce_images

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = make_workload("tiny8", read_tables(table_path))
    o = oracle.Oracle(table_path)
    o.setup(wl)
    angles = 2 * np.pi * np.arange(n_ang) / n_ang
    a0, cnt = angle_range(n_ang, rank, world)
    imgs = np.zeros((n_ang, o.nv, o.nu))
    for k in range(a0, a0 + cnt):  # the angle index keys the random streams, as on one process
        imgs[k] = o.scatter(float(angles[k]), n, 2.0, 9, angle_index=k)["Is"]
    tot = reduce_images(torch.from_numpy(imgs))
    if rank == 0:
        np.save(os.path.join(out_dir, "angles.npy"), tot.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_angle_sharding_reassembles_the_projection_set(table_path, tables, oracle_lib, tmp_path):
    """The paper's scheme (projections split over GPUs, Sec. II-B): three ranks take contiguous angle
    ranges of a 7-angle set; the reduced stack equals the single-process stack exactly (disjoint angles)."""
    n_ang, n = 7, 2000
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_angle_worker, args=(r, 3, port, table_path, n_ang, n, str(tmp_path)))
             for r in range(3)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    from mc_inputs import make_workload

    wl = make_workload("tiny8", tables)
    o = oracle_lib.Oracle(table_path)
    o.setup(wl)
    angles = 2 * np.pi * np.arange(n_ang) / n_ang
    ref = np.stack([o.scatter(float(angles[k]), n, 2.0, 9, angle_index=k)["Is"] for k in range(n_ang)])
    np.testing.assert_array_equal(np.load(tmp_path / "angles.npy"), ref)
