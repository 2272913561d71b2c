"""Long projections in resumable chunks: checkpoint/resume and failure recovery.

A history's random numbers are keyed by its index (Philox4x32-10 counter), so
a projection of N photons is the sum of the images of any partition of
0 .. N-1 into history ranges, and a range can be re-run anywhere with the same
result.  These helpers cut a long run into contiguous chunks and keep every
finished chunk's image:

- ``run_chunks``: one process; with a checkpoint file it writes the FP64 sum of
  the finished chunks and their list after each chunk (atomically: temporary
  file, then rename), and a later call with the same parameters resumes from it.
- ``run_workers``: several processes (one per GPU, or CPU workers); every
  chunk's image goes to its own file in a work directory, workers take chunks
  round-robin, and the coordinator re-runs in-process the chunks of any worker
  that died (non-zero exit) before summing all chunks in chunk order.

The sum is taken in chunk order in FP64 in both, so with a deterministic range
runner (one that adds its histories in a fixed order, as a CPU implementation
does) a run that was interrupted and resumed, or whose worker died, gives the
same total bit for bit as an uninterrupted one.  The
GPU's own tally adds in FP64 in a data-dependent order, so its chunk images
agree to FP64 rounding.  Host logic only: nothing here computes the method.
"""

from __future__ import annotations

import hashlib
import json
import os

import numpy as np


def chunk_ranges(n_photons, chunk):
    """[(h_begin, h_count)] covering 0 .. n_photons-1 in chunks of `chunk` (the last may be shorter)."""
    n_photons, chunk = int(n_photons), int(chunk)
    if n_photons < 0 or chunk < 1:
        raise ValueError("need n_photons >= 0 and chunk >= 1")
    return [(h, min(chunk, n_photons - h)) for h in range(0, n_photons, chunk)]


def _meta_key(meta):
    return hashlib.sha256(json.dumps(meta, sort_keys=True).encode()).hexdigest()


def _save_atomic(path, **arrays):
    tmp = path + ".tmp.npz"
    np.savez(tmp, **arrays)
    os.replace(tmp, path)


def run_chunks(runner, n_photons, chunk, meta=None, checkpoint=None, stop_after=None):
    """Sum runner(h_begin, h_count) (an FP64 array, the same shape every call) over
    the chunks of 0 .. n_photons-1.

    meta: JSON-serialisable description of the run (angles, seed, step, ...);
    a checkpoint only resumes a run with the same meta, n_photons and chunk.
    checkpoint: path of the checkpoint file (None: no checkpoint).
    stop_after: return after this many newly finished chunks (None: run to the end).
    Returns (total or None if chunks remain, number of finished chunks)."""
    ranges = chunk_ranges(n_photons, chunk)
    key = _meta_key({"meta": meta, "n_photons": int(n_photons), "chunk": int(chunk)})
    total, done = None, np.zeros(len(ranges), dtype=bool)
    if checkpoint and os.path.exists(checkpoint):
        with np.load(checkpoint) as z:
            if str(z["key"]) != key:
                raise ValueError("checkpoint belongs to another run")
            done = z["done"].copy()
            total = z["total"].copy() if bool(z["has_total"]) else None
    fresh = 0
    for i, (h0, cnt) in enumerate(ranges):
        if done[i]:
            continue
        if stop_after is not None and fresh >= stop_after:
            return None, int(done.sum())
        img = np.asarray(runner(h0, cnt), dtype=np.float64)
        total = img.copy() if total is None else total + img
        done[i] = True
        fresh += 1
        if checkpoint:
            _save_atomic(checkpoint, key=np.array(key), done=done, has_total=np.array(True), total=total)
    return total, int(done.sum())


def _chunk_file(workdir, i):
    return os.path.join(workdir, f"chunk_{i:08d}.npy")


def _write_chunk(workdir, i, img):
    path = _chunk_file(workdir, i)
    tmp = path + ".tmp.npy"
    np.save(tmp, np.asarray(img, dtype=np.float64))
    os.replace(tmp, path)


def worker_loop(make_runner, n_photons, chunk, rank, world, workdir, die_after=None):
    """Worker body: take chunks rank, rank + world, ... not yet on disk, write each image.
    make_runner() builds this process's runner (e.g. a GPU context); die_after
    exits the process abruptly after that many chunks (failure injection in tests)."""
    runner = make_runner()
    n = 0
    for i, (h0, cnt) in enumerate(chunk_ranges(n_photons, chunk)):
        if i % world != rank or os.path.exists(_chunk_file(workdir, i)):
            continue
        if die_after is not None and n >= die_after:
            os._exit(3)
        _write_chunk(workdir, i, runner(h0, cnt))
        n += 1


def run_workers(make_runner, n_photons, chunk, workdir, world, die_after=None, timeout=600.0):
    """Run the chunks on `world` spawned processes, recover the chunks of workers
    that failed by running them here, and return (total, failed ranks).

    make_runner must be picklable (a module-level function); die_after: {rank: n}
    failure injection."""
    import multiprocessing as mp

    os.makedirs(workdir, exist_ok=True)
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=worker_loop,
                         args=(make_runner, n_photons, chunk, r, world, workdir, (die_after or {}).get(r)))
             for r in range(world)]
    for p in procs:
        p.start()
    failed = []
    for r, p in enumerate(procs):
        p.join(timeout)
        if p.is_alive():
            p.terminate()
            p.join()
        if p.exitcode != 0:
            failed.append(r)
    ranges = chunk_ranges(n_photons, chunk)
    missing = [i for i in range(len(ranges)) if not os.path.exists(_chunk_file(workdir, i))]
    if missing:
        runner = make_runner()
        for i in missing:
            _write_chunk(workdir, i, runner(*ranges[i]))
    total = None
    for i in range(len(ranges)):
        img = np.load(_chunk_file(workdir, i))
        total = img.copy() if total is None else total + img
    return total, failed
