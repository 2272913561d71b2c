"""Writes cyl64_scatter_1e9.npz: the oracle's scatter image (eq. Is) of the
64^3 cylinder/rod phantom (60 keV, SOD/SDD 300/600 mm, 128^2 x 1 mm panel,
step 0.5 mm, 10 pseudo-particles per interaction) at beta = 0 from 1e9 photon
histories, seed 32, in 50 batches of consecutive history ranges, so that a
test can compare a GPU image of the same depth pixel by pixel.

Calls only oracle/ and mc_inputs/ (the seeded inputs).  Stored: the image,
the variance of that image estimated from the batches, and a fingerprint of
the oracle's transport (the image of histories 0..1999) that the test
recomputes, so a changed oracle cannot silently keep a stale reference.

    python tests/golden/make_cyl64_scatter_reference.py [processes]
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

N = 1_000_000_000
BATCHES = 50
SEED = 32
OUT = os.path.join(HERE, "cyl64_scatter_1e9.npz")


def _oracle():
    import tempfile

    import oracle
    from mc_inputs import default_table_path, make_workload, read_tables

    tp = default_table_path("full", os.path.join(tempfile.gettempdir(), "mc_golden_tables"))
    wl = make_workload("cyl64", read_tables(tp))
    o = oracle.Oracle(tp)
    o.setup(wl)
    return o, wl


def fingerprint():
    o, wl = _oracle()
    return o.scatter(0.0, N, wl["step_mm"], SEED, h_begin=0, h_end=2000)["Is"]


def batch(b):
    o, wl = _oracle()
    return o.scatter(0.0, N, wl["step_mm"], SEED, h_begin=b * N // BATCHES, h_end=(b + 1) * N // BATCHES)["Is"]


def main():
    import multiprocessing as mp

    procs = int(sys.argv[1]) if len(sys.argv) > 1 else max(1, (os.cpu_count() or 2) - 2)
    t0 = time.time()
    with mp.get_context("spawn").Pool(procs) as pool:
        parts = np.array(pool.map(batch, range(BATCHES), chunksize=1))
    img = parts.sum(0)
    var = parts.var(axis=0, ddof=1) * BATCHES
    np.savez_compressed(OUT, image=img, variance=var, fingerprint=fingerprint(), photons=N, batches=BATCHES,
                        seed=SEED)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s; relative noise {np.sqrt(var.sum()) / np.linalg.norm(img):.4f}")


if __name__ == "__main__":
    main()
