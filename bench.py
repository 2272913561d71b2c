#!/usr/bin/env python3
"""Throughput of the GB300 Monte Carlo scatter forward projection.

One step = one mc_project call over the whole path: the primary image
(eq. Ip) and n_photons scatter histories scored on the panel (eq. Is) for one
projection of the 256^3 / 512^2 / 1e8-photon polyenergetic workload (ell256:
seeded ellipsoids of water, PMMA, aluminium and bone in air, 120 kVp Kramers
spectrum with 2 mm Al, SOD/SDD 400/800 mm, 0.4 mm pixels, 0.25 mm step).
Metric: photon histories/s, whole job.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU runs are replicas (one independent projection per rank, no
collective on the data path): value = histories of all ranks / max time.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "photon histories/s on 1 GB300; s/projection at <=2% scatter L2 error vs plain MC"
UNIT = "histories/s"
WORKLOAD = "ell256"
FLOPS_PER_STEP = 10  # algorithmic FP32 operations per fixed-step march step


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--photons", type=float, default=None, help="override photons per step")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle sample budget")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--voxel-layout", type=int, default=0, help="0 default, 1 linear, 2 4^3 bricks")
    p.add_argument("--workload", default=WORKLOAD, help="ell256 (default) or ell512 (batched angles)")
    p.add_argument("--angles", type=int, default=1, help="projection angles per step (one launch)")
    p.add_argument("--per-angle", action="store_true", help="one mc_project call per angle instead of one batch")
    p.add_argument("--graph", action="store_true", help="replay a captured CUDA graph")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-tiled-alt", action="store_true",
                   help="skip the extra (untimed-for-value) run of the tile-stratified tally")
    p.add_argument("--detector", default="energy", choices=["energy", "panel"],
                   help="detector response: energy integrating (eta = E) or the flat-panel Gd2O2S model")
    p.add_argument("--autotune", action="store_true",
                   help="pick step (within --tune-step-min..max at --tune-tol primary error) and launch shape first")
    p.add_argument("--tune-step-min", type=float, default=0.1)
    p.add_argument("--tune-step-max", type=float, default=0.4)
    p.add_argument("--tune-tol", type=float, default=0.005)
    p.add_argument("--denoise-eval", action="store_true",
                   help="seconds per projection at <= 2%% scatter error: plain MC vs smoothing vs learned denoiser")
    p.add_argument("--conv-bench", action="store_true",
                   help="tensor-core throughput of the denoiser's convolutions and its inference latency")
    p.add_argument("--correct-eval", action="store_true", help="iterative scatter correction on a large flat panel")
    p.add_argument("--vr-eval", action="store_true",
                   help="point-detector scoring variants (expected value, forced detection) by figure of merit")
    p.add_argument("--vr-panel", type=int, default=32, help="coarse panel pixels a side for forced detection")
    p.add_argument("--vr-photons", type=float, default=2e6, help="photons per projection on the coarse panel")
    p.add_argument("--mesh-bench", action="store_true", help="primary images of the triangle-mesh phantom")
    p.add_argument("--tally-eval", action="store_true", help="figure of merit of the tally modes")
    p.add_argument("--primary-bench", action="store_true", help="primary images of the correction workload")
    p.add_argument("--fdk-bench", action="store_true", help="FDK of 256 projections of the correction workload")
    p.add_argument("--upsample-bench", action="store_true", help="smoothing + interpolation to 1024 x 2048^2")
    p.add_argument("--primary-speckle", type=float, default=0.0, help="fraction of voxels given another material")
    p.add_argument("--mesh-segments", type=int, default=1024)
    p.add_argument("--nee-mode", type=int, default=0, help="0 sampled-type scoring (the paper's), 1 expected value")
    p.add_argument("--n-split", type=int, default=10, help="pseudo-particles per scatter interaction")
    p.add_argument("--tally", choices=["auto", "global", "shared", "warp", "tiled"], default="auto",
                   help="how point-detector scores reach the image (tiled: tile-stratified, --tile pixels)")
    p.add_argument("--tile", type=int, nargs=2, default=[64, 64], metavar=("U", "V"))
    p.add_argument("--cor-detector", type=int, default=2048)
    p.add_argument("--cor-pixel", type=float, default=0.1)
    p.add_argument("--cor-proj", type=int, default=1024)
    p.add_argument("--cor-volume", type=int, default=512)
    p.add_argument("--cor-voxel", type=float, default=0.2)
    p.add_argument("--cor-seed", type=int, default=4242)
    p.add_argument("--cor-phantom", default="cylinder", choices=["cylinder", "ellipsoids"],
                   help="water cylinder with inserts (cupping) or the ellipsoid generator")
    p.add_argument("--cor-step", type=float, default=0.2)
    p.add_argument("--cor-meas-grid", type=int, default=256)
    p.add_argument("--cor-meas-angles", type=int, default=32)
    p.add_argument("--cor-meas-photons", type=float, default=1e8)
    p.add_argument("--cor-total-photons", type=float, default=1e10)
    p.add_argument("--cor-sim-grid", type=int, default=256)
    p.add_argument("--cor-mc-bin", type=int, choices=[0, 2], default=0,
                   help="2: Monte Carlo on the segmented volume down-sampled by 2 per axis (the paper's speed-up)")
    p.add_argument("--cor-sim-angles", type=int, default=180)
    p.add_argument("--cor-sim-photons", type=float, default=1e6)
    p.add_argument("--cor-iters", type=int, default=3)
    p.add_argument("--conv-size", type=int, default=256)
    p.add_argument("--conv-batch", type=int, default=8)
    p.add_argument("--train-phantoms", type=int, default=200)
    p.add_argument("--train-angles", type=int, default=10)
    p.add_argument("--train-inputs", type=float, nargs="+", default=[1e6])
    p.add_argument("--target-photons", type=float, default=1e9)
    p.add_argument("--train-steps", type=int, default=3000)
    p.add_argument("--save-weights", default=None, help="write the trained denoiser here (--denoise-eval)")
    p.add_argument("--ref-photons", type=float, default=1e10)
    p.add_argument("--eval-angles", type=int, default=360)
    p.add_argument("--no-c4", action="store_true", help="skip the denoised-scatter figures of the default run")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.first = 0

    def mark(self):
        """Summarise only the samples taken from now on (the sampler is started
        ahead of the timed region, so that its start-up stays outside it)."""
        self.first = len(self.lines)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines[self.first:]:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def device_id(torch, dev):
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        return str(dev)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def host_cpu():
    """Host core count and model name (for the CPU-baseline record)."""
    name = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    name = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not name:
        try:
            name = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            name = next((l.split(":", 1)[1].strip() for l in name.splitlines() if l.startswith("Model name")), "")
        except Exception:
            name = ""
    import platform

    return os.cpu_count() or 1, (name or platform.machine())


def _oracles(tp, wl, threads):
    import oracle

    orcs = [oracle.Oracle(tp) for _ in range(threads)]
    for o in orcs:
        o.setup(wl)
    return orcs


def _oracle_blocks(orcs, wl, n_photons, blocks, block):
    """Histories [b, b + block) for every start b in `blocks`, dealt round-robin
    to the oracles and run on all of them at once (the oracle's C calls release
    the GIL, so threads run in parallel)."""
    from concurrent.futures import ThreadPoolExecutor

    def run(i):
        steps = 0
        for b in blocks[i :: len(orcs)]:
            st = orcs[i].scatter(0.0, n_photons, wl["step_mm"], wl["seed"], int(b), int(min(b + block, n_photons)))
            steps += st["stats"]["flight_steps"] + st["stats"]["nee_steps"]
        return steps

    if len(orcs) == 1:
        return run(0)
    with ThreadPoolExecutor(len(orcs)) as ex:
        return sum(ex.map(run, range(len(orcs))))


def spread_blocks(n_photons, n_blocks, block, phase=0.0):
    """Starts of n_blocks history blocks spread evenly over [0, n_photons).

    Histories are stratified over the spectrum's energy bins in index order
    (the lowest bins first), so a sample must span the whole range: block k
    starts at (k + phase) n_photons / n_blocks (phase in [0, 1))."""
    n_blocks = max(1, int(n_blocks))
    span = n_photons / n_blocks
    starts = [int((k + phase) * span) for k in range(n_blocks)]
    return [min(b, max(0, n_photons - block)) for b in starts]


def oracle_rate(tp, wl, n_photons, budget_s, threads=1):
    """Oracle histories/s on a bounded sample of the workload: the primary image
    once (single thread), then blocks of histories spread evenly over the whole
    history range (so every energy bin is sampled in proportion), run on
    `threads` threads, extrapolated to one projection."""
    orcs = _oracles(tp, wl, threads)
    t0 = time.perf_counter()
    orcs[0].primary(0.0, wl["step_mm"])
    t_primary = time.perf_counter() - t0
    # single-thread calibration on a spread sample
    block = 64
    cal = spread_blocks(n_photons, 16, block, 0.5)
    t0 = time.perf_counter()
    _oracle_blocks(orcs[:1], wl, n_photons, cal, block)
    t1 = (time.perf_counter() - t0) / (len(cal) * block)
    rate1 = n_photons / (t_primary + n_photons * t1)
    left = max(2.0, budget_s - t_primary - len(cal) * block * t1)
    n_hist = int(max(threads * 256, min(5e6, left / t1 * threads)))
    block = 512
    starts = spread_blocks(n_photons, max(threads, n_hist // block), block, 0.25)
    t0 = time.perf_counter()
    steps = _oracle_blocks(orcs, wl, n_photons, starts, block)
    dt = time.perf_counter() - t0
    done = sum(min(b + block, n_photons) - b for b in starts)
    rate = n_photons / (t_primary + n_photons * dt / done)
    steps_per_s = steps / dt  # march steps per second of the sampled histories, all threads
    sample = (f"oracle, {threads} thread(s): primary image once, single thread ({t_primary:.2f} s) + {done} histories "
              f"in {len(starts)} blocks of {block} spread evenly over the {int(n_photons)}-photon run ({dt:.1f} s "
              "wall), extrapolated to one full projection")
    return rate, sample, rate1, steps_per_s


def make_inputs(tables_dir, photons, workload=WORKLOAD):
    from mc_inputs import default_table_path, make_workload, read_tables

    tp = default_table_path("full", tables_dir)
    wl = make_workload(workload, read_tables(tp))
    if photons:
        wl["n_photons"] = int(photons)
    return tp, wl


def bench_config(args, wl, n_ang=1, detector=None):
    """The workload description both arms print (same keys, same values)."""
    vol = wl["volume"]
    g = wl["geometry"]
    nz, ny, nx = vol["mat"].shape
    return {"workload": args.workload,
            "volume": f"{nx}x{ny}x{nz} voxels at {vol['spacing'][0]} mm, uint8 material + fp16 density",
            "detector": f"{g['nu']}x{g['nv']} pixels at {g['pu']} mm",
            "photons_per_projection": int(wl["n_photons"]), "angles_per_step": n_ang, "step_mm": wl["step_mm"],
            "n_split": args.n_split, "spectrum": f"{len(wl['weights'])} bins", "response": detector or args.detector,
            "nee_mode": args.nee_mode, "l2_flush": True,
            "parallelism": "replicas" if int(os.environ.get("WORLD_SIZE", 1)) > 1 else "single",
            "launch": "per-angle" if args.per_angle else "batched", "graph": bool(args.graph),
            "voxel_layout": args.voxel_layout,
            "tally": args.tally + (f" {args.tile[0]}x{args.tile[1]}" if args.tally == "tiled" else "")}


def run_reference(args):
    """The oracle as it stands, on all host cores (one oracle per thread); each
    step is a bounded sample of the projection: blocks of histories spread
    evenly over the whole history range, at a new phase every step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    tdir = tempfile.mkdtemp(prefix="mcbench")
    tp, wl = make_inputs(tdir, args.photons, args.workload)
    cores, cpu_name = host_cpu()
    orcs = _oracles(tp, wl, cores)
    N = wl["n_photons"]
    block = 256
    # size each step to ~ (budget / (K + W)) seconds
    per_step = max(2.0, min(20.0, 150.0 / (args.steps + args.warmup)))
    cal = spread_blocks(N, cores * 4, block, 0.5)
    t0 = time.perf_counter()
    _oracle_blocks(orcs, wl, N, cal, block)  # calibration with every thread busy
    t_h = (time.perf_counter() - t0) / (len(cal) * block)  # wall seconds per history, all threads
    n_blocks = max(cores, int(per_step / max(t_h, 1e-9) / block))
    golden = 0.6180339887498949

    def one_step(k):
        starts = spread_blocks(N, n_blocks, block, (k * golden) % 1.0)
        steps = _oracle_blocks(orcs, wl, N, starts, block)
        return sum(min(b + block, N) - b for b in starts), steps

    for k in range(args.warmup):
        one_step(k)
    done, marched = 0, 0
    t0 = time.perf_counter()
    for k in range(args.steps):
        d, m = one_step(args.warmup + k)
        done += d
        marched += m
    el = time.perf_counter() - t0
    value = done / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args, wl),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_name,
                         "steps_per_s": marched / el,
                         "sample": f"per step {n_blocks} blocks of {block} scatter histories spread evenly over the "
                                   f"{N}-photon run (new phase each step), {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


TRANSPORT_SOURCES = ("paper_2201_13191_gb300/csrc/k_transport.cu", "paper_2201_13191_gb300/csrc/mc_device.cuh")


def transport_source_hash():
    """First 16 hex digits of the SHA-256 of the transport kernel's sources and its compiler flags."""
    import hashlib

    from paper_2201_13191_gb300.build import FLAGS, SOURCE_FLAGS

    h = hashlib.sha256()
    for f in TRANSPORT_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(FLAGS + SOURCE_FLAGS.get("k_transport.cu", [])).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload):
    """Per-march-step DRAM and L2 bytes of k_transport from the ncu summaries
    profiles/k_transport_<workload>*.md (a line 'traffic-per-step: kernel=<hash> workload=<name>
    dram_bytes=<x> l2_bytes=<y> [simt_lanes=<z>]'), or None when the summary was taken on other
    sources than the current kernel's."""
    import glob

    lines = []
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", f"k_transport_{workload}*.md"))):
        lines += open(path).read().splitlines()
    want = transport_source_hash()
    for line in lines:
        if line.startswith("traffic-per-step:"):
            kv = dict(x.split("=", 1) for x in line.split()[1:])
            if kv.get("kernel") == want and kv.get("workload") == workload:
                return float(kv["dram_bytes"]), float(kv["l2_bytes"]), float(kv.get("simt_lanes", "nan"))
    return None


def probe_library():
    """libmcprobe.so (include/mc_probe.h): the measurement kernels, built beside the product library."""
    import ctypes as C

    from paper_2201_13191_gb300.build import build_probe

    L = C.CDLL(build_probe())
    vp, i, u64 = C.c_void_p, C.c_int, C.c_uint64
    L.mc_probe_stream.argtypes = [vp, u64, i, i, i, vp, vp]
    L.mc_probe_gather.argtypes = [vp, u64, i, i, i, vp, vp]
    L.mc_probe_mma.argtypes = [i, i, i, vp, vp]
    return L


def _event_time(torch, stream, fn, reps=5, warm=2):
    for _ in range(warm):
        fn()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return float(np.median(ts))


def packed_words(shape, voxel_layout, props):
    """Words of the library's packed volume: a one-voxel border, x fastest, or
    4x4x4 bricks (the default switches to bricks beyond 3/4 of L2)."""
    nz, ny, nx = shape
    px, py, pz = nx + 2, ny + 2, nz + 2
    lin = px * py * pz
    brick = -(-px // 4) * -(-py // 4) * -(-pz // 4) * 64
    l2 = int(getattr(props, "L2_cache_size", 126 * 1024 * 1024))
    if voxel_layout == 1 or (voxel_layout == 0 and lin * 4 <= 0.75 * l2):
        return lin
    return brick


def memory_roofline(torch, props, shape, layout_words, steps_per_s, stream):
    """Voxel-gather roofline of the transport at the memory level the packed
    volume lives in.  Algorithmic bytes: 3 per march step (1-byte material +
    2-byte FP16 density); the kernel reads them as one 4-byte word.  Peak:
    coalesced streaming reads (mc_probe_stream) over a buffer the size of the
    packed volume, measured live: from L2 when the buffer fits, from HBM when
    it does not.  Secondary figure: random 4-byte gathers (mc_probe_gather)
    over the same buffer, each touching its own 32-byte sector."""
    import ctypes as C

    P = probe_library()
    n_bytes = (layout_words * 4 + 15) // 16 * 16
    l2 = int(getattr(props, "L2_cache_size", 126 * 1024 * 1024))
    level = "l2" if n_bytes <= 0.75 * l2 else "hbm"
    buf = torch.ones(n_bytes // 4, dtype=torch.int32, device="cuda")
    sms = props.multi_processor_count
    grid, block = sms * 8, 256
    sink = torch.empty(grid * block, dtype=torch.int32, device="cuda")
    sh = C.c_void_p(stream.cuda_stream)
    passes = 20 if level == "l2" else 4

    def stream_read():
        if P.mc_probe_stream(C.c_void_p(buf.data_ptr()), n_bytes, passes, grid, block, C.c_void_p(sink.data_ptr()),
                             sh):
            raise RuntimeError("mc_probe_stream failed")

    rounds = 256

    def gather():
        if P.mc_probe_gather(C.c_void_p(buf.data_ptr()), n_bytes // 4, rounds, grid, block,
                             C.c_void_p(sink.data_ptr()), sh):
            raise RuntimeError("mc_probe_gather failed")

    stream_bps = passes * n_bytes / _event_time(torch, stream, stream_read)
    gathers_ps = 8 * rounds * grid * block / _event_time(torch, stream, gather)
    del buf, sink
    algo = 3.0 * steps_per_s
    return {"level": level, "unit": "GB/s", "achieved": algo / 1e9, "peak": stream_bps / 1e9,
            "frac": algo / stream_bps, "bytes_per_step": 3, "word_bytes_per_step": 4,
            "word_GBps": 4.0 * steps_per_s / 1e9,
            "peak_basis": f"mc_probe_stream: coalesced 16-byte reads over {n_bytes / 1e6:.1f} MB (the packed "
                          f"volume's size), {passes} passes, {grid}x{block} threads; L2 {l2 / 1e6:.0f} MB",
            "random_gather": {"gathers_per_s": gathers_ps, "sector_GBps": 32.0 * gathers_ps / 1e9,
                              "steps_per_random_gather": steps_per_s / gathers_ps}}


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_2201_13191_gb300 as mcx

    mcx.build()
    tdir = tempfile.mkdtemp(prefix=f"mcbench{rank}")
    tp, wl = make_inputs(tdir, args.photons, args.workload)
    N = wl["n_photons"]
    n_ang = max(1, args.angles)
    angles = (2.0 * np.pi * np.arange(n_ang) / n_ang).astype(np.float32)
    seed = wl["seed"] + 1000 * rank
    tally = {"auto": 0, "global": 1, "shared": 2, "warp": 3, "tiled": 4}[args.tally]
    ctx = mcx.Context(local, voxel_layout=args.voxel_layout, use_graph=int(args.graph), nee_mode=args.nee_mode,
                      tally_mode=tally, tile_u=args.tile[0], tile_v=args.tile[1], n_split=args.n_split)
    ctx.load_tables(tp)
    ctx.setup(wl)
    if args.detector == "panel":
        from mc_inputs import read_tables, table_response

        ctx.set_detector_response(table_response(read_tables(tp)))
    stream = torch.cuda.current_stream()
    tuned = None
    if args.autotune:
        t0 = time.perf_counter()
        probe = angles[:: max(1, n_ang // 8)][:8]
        tuned = ctx.autotune(probe, 2_000_000, args.tune_step_min, args.tune_step_max, args.tune_tol, stream=stream)
        tuned["seconds"] = time.perf_counter() - t0
        tuned["probe_angles"] = int(len(probe))
        wl["step_mm"] = float(tuned["step_mm"])
    out = {"primary": ctx.empty_images(n_ang), "scatter": ctx.empty_images(n_ang)}
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    flush.zero_()  # the first touch of a fresh allocation maps its pages (~0.25 s): keep it out of the timed region

    split = {}

    def step(k):
        """One step: the projection(s) of all angles, batched or one call per angle."""
        if not args.per_angle:
            ctx.project(angles, N, wl["step_mm"], seed + k, out=out, stream=stream)
            st = ctx.last_stats()
            split.update(flight_steps=st["flight_steps"], nee_steps=st["nee_steps"], nee_rays=st["nee_rays"],
                         interactions=st["compton"] + st["rayleigh"] + st["photo"])
            return st["transport_ms"], st["flight_steps"] + st["nee_steps"], 3
        ms, steps = 0.0, 0.0
        for i in range(n_ang):
            o = {"primary": out["primary"][i : i + 1], "scatter": out["scatter"][i : i + 1]}
            ctx.project(angles[i : i + 1], N, wl["step_mm"], seed + k * n_ang + i, out=o, stream=stream)
            st = ctx.last_stats()
            ms += st["transport_ms"]
            steps += st["flight_steps"] + st["nee_steps"]
        return ms, steps, 3 * n_ang

    clocks = Clocks(device_id(torch, local))
    clocks.start()
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    clocks.mark()
    t_kernel, steps_per, launches = [], [], 0
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(args.steps):
        flush.zero_()  # evict the volume from L2 between steps
        ms, stp, nl = step(args.warmup + k)
        t_kernel.append(ms)
        steps_per.append(stp)
        launches += nl
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    el_ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    if world > 1:
        from paper_2201_13191_gb300.shard import max_time

        el_ms = max_time(el_ms, device="cuda")
    value = world * N * n_ang * args.steps / (el_ms / 1e3)

    # end to end through the C ABI with host buffers: volume upload from pinned
    # host memory, projection, read-back of both images
    vol = wl["volume"]
    e2e_value = None
    h2d = vol["mat"].nbytes + vol["rho"].nbytes + 4 * n_ang + len(wl["weights"]) * 12
    d2h = 2 * ctx.nu * ctx.nv * 4 * n_ang
    if not args.no_e2e:
        h_mat = torch.from_numpy(vol["mat"]).pin_memory()
        h_rho = torch.from_numpy(vol["rho"].view(np.int16)).pin_memory()
        h_out = torch.empty((2, n_ang, ctx.nv, ctx.nu), dtype=torch.float32).pin_memory()
        e2e_steps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            ctx.load_volume(h_mat, h_rho, vol["spacing"], stream=stream)
            ctx.project(angles, N, wl["step_mm"], seed + 100 + k, out=out, stream=stream)
            h_out[0].copy_(out["primary"], non_blocking=True)
            h_out[1].copy_(out["scatter"], non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        if world > 1:
            from paper_2201_13191_gb300.shard import max_time

            e2e_s = max_time(e2e_s, device="cuda")
        e2e_value = world * N * n_ang * e2e_steps / e2e_s

    # the same projection with the tile-stratified tally (16x16 tiles: shared-memory
    # tile images flushed into the FP64 image per chunk), outside the timed region:
    # its kernel rate beside the headline's plain global tally
    tiled_alt = None
    if args.tally in ("auto", "global") and not args.per_angle and n_ang == 1 and not args.no_tiled_alt:
        ctx.set_options(tally_mode=4, tile_u=16, tile_v=16)
        for k in range(2):
            ctx.project(angles, N, wl["step_mm"], seed + 200 + k, out=out, stream=stream)
        tk = []
        for k in range(3):
            flush.zero_()
            ctx.project(angles, N, wl["step_mm"], seed + 300 + k, out=out, stream=stream)
            tk.append(ctx.last_stats()["transport_ms"])
        torch.cuda.synchronize()
        ctx.set_options(tally_mode=tally, tile_u=args.tile[0], tile_v=args.tile[1])
        tiled_alt = {"tally": "tiled 16x16", "histories_per_s": N * n_ang / (float(np.mean(tk)) / 1e3),
                     "transport_ms": float(np.mean(tk)), "reps": len(tk),
                     "note": "transport kernel time (CUDA events), L2 flushed between reps; its noise per history "
                             "and figure of merit against the global tally: profiles/tally_modes_ell256.md"}

    # roofline of the dominant kernel (transport): FP32 issue
    props = torch.cuda.get_device_properties(local)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = props.multi_processor_count * 128 * sm_max * 1e6 / 1e12
    mean_ms = float(np.mean(t_kernel))
    achieved = FLOPS_PER_STEP * float(np.mean(steps_per)) / (mean_ms / 1e3) / 1e12
    rec = recorded_traffic(args.workload)
    traffic = None if rec is None else rec[0] * float(np.mean(steps_per))
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / peak_tflops, "traffic": traffic,
            "traffic_basis": None if rec is None else
            f"ncu dram__bytes_read.sum + dram__bytes_write.sum of a 2e6-photon launch of the same kernel, "
            f"{rec[0]:.4f} B per march step, scaled by the march steps of this launch; L2 bytes per step "
            f"{rec[1]:.2f} (profiles/k_transport_{args.workload}*.md)",
            "kernel": "k_transport", "steps_per_launch": float(np.mean(steps_per)),
            "kernel_ms": mean_ms, "steps_per_s": float(np.mean(steps_per)) / (mean_ms / 1e3),
            "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x {sm_max:.0f} MHz (max clock)",
            "step_split": split}
    roof["memory"] = memory_roofline(torch, props, vol["mat"].shape,
                                     packed_words(vol["mat"].shape, args.voxel_layout, props), roof["steps_per_s"],
                                     stream)
    if rec is not None:
        # bytes the kernel moves from L2 per march step (ncu), against the algorithmic 3
        roof["memory"]["l2_bytes_per_step"] = rec[1]
        roof["memory"]["l2_traffic_over_algorithmic"] = rec[1] / 3.0
        if np.isfinite(rec[2]):
            # branch efficiency: active lanes per warp instruction (ncu thread / warp instructions) of 32
            roof["branch_efficiency"] = rec[2] / 32.0

    # the second half of the metric: seconds per projection at <= 2% scatter
    # error for plain MC, Savitzky-Golay smoothing and the learned denoiser
    # (weights trained by bench.py --denoise-eval), on the held-out phantom
    c4 = None
    if rank == 0 and not args.no_c4 and os.path.exists(C4_WEIGHTS):
        t0 = time.perf_counter()
        ctx4, _ = c4_context(mcx)
        ctx4.denoise_load(C4_WEIGHTS, 1)
        c4 = c4_curves(ctx4, [0.1, 1.7], 2e9, [1e5, 3e5, 1e6, 3e6, 1e7, 3e7, 1e8, 3e8, 1e9, 2e9])
        c4["seconds"] = time.perf_counter() - t0
        c4["workload"] = (f"cylinder/rod phantom seed {C4_HELD_OUT} (held out), {C4_N}^3 x {C4_DV} mm, "
                          f"{C4_PX}^2 x {128.0 / C4_PX} mm panel, 60 keV, step {C4_STEP} mm, 2 angles")
        ctx4.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores, cpu_name = host_cpu()
        rate, sample, rate1, sps = oracle_rate(tp, wl, N, args.cpu_seconds, threads=cores)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "value_1_thread": rate1, "steps_per_s": sps, "cpu": cpu_name}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded ellipsoid phantom, Kramers spectrum)",
            "config": dict(bench_config(args, wl, n_ang), **({"autotune": tuned} if tuned else {})),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": None if e2e_value is None else {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                                                   "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
            "s_per_projection": el_ms / 1e3 / args.steps / n_ang,
            "s_per_projection_at_2pct": None if c4 is None else c4["s_per_projection_at_2pct"],
            "s_per_projection_at_2pct_batched": None if c4 is None else c4["s_per_projection_at_2pct_batched"],
            "denoised_scatter": c4,
            "tally_tiled_alt": tiled_alt,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# The learned-denoiser workload: the cylinder/rod phantom family at 256^3 x 0.25 mm (64 mm field of view,
# feature sizes in mm), 60 keV, SOD/SDD 300/600 mm, 256^2 x 0.5 mm scatter images, step 0.5 mm.
C4_N, C4_DV, C4_PX, C4_STEP = 256, 0.25, 256, 0.5
C4_WEIGHTS = os.path.join(ROOT, "paper_2201_13191_gb300", "weights", "unet_c4_256.bin")
C4_HELD_OUT = 50_000  # phantom seed never used for training


def c4_context(mcx):
    from mc_inputs import default_table_path, mono_spectrum

    tp = default_table_path("full", tempfile.mkdtemp(prefix="mcc4"))
    ctx = mcx.Context(0)
    ctx.load_tables(tp)
    E, w = mono_spectrum(60.0)
    ctx.set_spectrum(E, w)
    ctx.set_geometry(300.0, 600.0, C4_PX, C4_PX, 128.0 / C4_PX, 128.0 / C4_PX)
    return ctx, tp


def c4_phantom(seed):
    from mc_inputs import cylinder_variant_phantom

    return cylinder_variant_phantom(seed, n=C4_N, dv=C4_DV, physical=True)


def c4_scatter(ctx, n_photons, angle, seed):
    out = ctx.project([angle], int(n_photons), C4_STEP, seed, primary=False)["scatter"][0]
    return out, ctx.last_stats()["transport_ms"]


def c4_reference(ctx, n_photons, angle, seed):
    """Plain-MC reference image and the squared norm of its own noise (sum of
    its 20-batch variance), so that an error measured against it can be
    corrected for the reference's noise: E|x - ref|^2 = |x - truth|^2 + sum var."""
    ctx.set_options(n_batches=20)
    out = ctx.project([angle], int(n_photons), C4_STEP, seed, primary=False, variance=True)
    ctx.set_options(n_batches=1)
    return out["scatter"][0].double(), float(out["variance"][0].double().sum())


def c4_error(img, ref, noise2):
    """Relative L2 error against the truth estimated from a noisy reference."""
    import torch

    d2 = float(torch.sum((img.double() - ref) ** 2)) - noise2
    return float(np.sqrt(max(d2, 0.0) / max(float(torch.sum(ref * ref)) - noise2, 1e-300)))


def c4_curves(ctx, angles, ref_photons, grid, seed0=9_000):
    """Error (relative L2 against a ref_photons plain-MC reference, corrected
    for the reference's own noise, mean over the angles) and time per
    projection (transport kernel + post-processing, CUDA events) of plain MC,
    Savitzky-Golay smoothing (window 9, cubic; the paper's Sec. II-C.4, through
    mc_smooth_upsample) and the learned denoiser (mc_denoise_infer, weights
    already in ctx), for each photon count of grid; then the photons and
    seconds per projection where each error curve crosses 2% (log-log
    interpolation between grid points)."""
    import torch

    import paper_2201_13191_gb300 as mcx

    v = c4_phantom(C4_HELD_OUT)
    ctx.load_volume(v["mat"], v["rho"], v["spacing"])
    refs = [c4_reference(ctx, ref_photons, a, seed0 + i) for i, a in enumerate(angles)]
    sg = mcx.Context(0)
    curves = {"plain": [], "smoothed": [], "denoised": []}
    times = {"plain": [], "smoothed": [], "denoised": []}
    for n in grid:
        errs = {k: [] for k in curves}
        t_mc, t_post = [], {"smoothed": [], "denoised": []}
        for i, a in enumerate(angles):
            img, ms = c4_scatter(ctx, n, a, 5_000 + 17 * i + int(np.log10(n) * 100))
            t_mc.append(ms)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            smooth = sg.smooth_upsample(img[None], [0.0], [0.0], C4_PX, C4_PX)[0]
            ev1.record()
            torch.cuda.synchronize()
            t_post["smoothed"].append(ev0.elapsed_time(ev1))
            ev0.record()
            den = ctx.denoise_infer(img[None])[0]
            ev1.record()
            torch.cuda.synchronize()
            t_post["denoised"].append(ev0.elapsed_time(ev1))
            r, nz2 = refs[i]
            errs["plain"].append(c4_error(img, r, nz2))
            errs["smoothed"].append(c4_error(smooth, r, nz2))
            errs["denoised"].append(c4_error(den, r, nz2))
        for k in curves:
            curves[k].append(float(np.mean(errs[k])))
            times[k].append(float(np.mean(t_mc)) + (float(np.mean(t_post[k])) if k in t_post else 0.0))

    def at_target(k, target=0.02):
        e = curves[k]
        for j in range(len(grid)):
            if e[j] <= target:
                if j == 0:
                    return grid[0], times[k][0]
                f = (np.log(e[j - 1]) - np.log(target)) / (np.log(e[j - 1]) - np.log(e[j]))
                n = float(np.exp(np.log(grid[j - 1]) + f * (np.log(grid[j]) - np.log(grid[j - 1]))))
                t = float(np.exp(np.log(times[k][j - 1]) + f * (np.log(times[k][j]) - np.log(times[k][j - 1]))))
                return n, t
        return None, None

    res = {k: at_target(k) for k in curves}
    ref_noise = [float(np.sqrt(nz2 / max(float(torch.sum(r * r)), 1e-300))) for r, nz2 in refs]
    # the batched form at the photons each method needs for 2%: many angles of the phantom
    # in one launch, then their post-processing in one call (plain MC is left single:
    # one projection of its ~1e9 photons already fills the GPU)
    batched = {}
    for k, n_ang in (("denoised", 360), ("smoothed", 8)):
        if res[k][0] is not None:
            batched[k] = {"s": c4_batched(ctx, sg, k, res[k][0], n_ang), "angles": n_ang,
                          "photons": float(res[k][0])}
            if res["plain"][1] is not None:
                batched[k]["speedup_vs_plain"] = res["plain"][1] / 1e3 / batched[k]["s"]
    return {
        "reference_photons": float(ref_photons), "reference_noise_rel_l2": ref_noise,
        "photons_at_2pct": {k: res[k][0] for k in res},
        "s_per_projection_at_2pct": {k: (None if res[k][1] is None else res[k][1] / 1e3) for k in res},
        "speedup_vs_plain": {k: (None if res[k][1] is None or res["plain"][1] is None else res["plain"][1] / res[k][1])
                             for k in ("smoothed", "denoised")},
        "error_curves": {"photons": grid, **curves},
        "ms_per_projection": {"photons": grid, **times},
        "s_per_projection_at_2pct_batched": batched,
    }


def c4_batched(ctx, sg, method, n_photons, n_ang, seed=7_000):
    """Seconds per projection of the batched form of a method: n_ang angles of
    the loaded phantom in one launch (all angles batched), then the method's
    post-processing of all of them in one call (Savitzky-Golay through
    mc_smooth_upsample, or the denoiser over the whole batch); CUDA events
    around both, after one warm-up run."""
    import torch

    angs = (2.0 * np.pi * np.arange(n_ang) / n_ang).astype(np.float32)
    out = {"scatter": ctx.empty_images(n_ang)}

    def run(sd):
        ctx.project(angs, int(n_photons), C4_STEP, sd, primary=False, out=out)
        if method == "smoothed":
            sg.smooth_upsample(out["scatter"], angs, angs, C4_PX, C4_PX)
        elif method == "denoised":
            ctx.denoise_infer(out["scatter"])

    run(seed)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    run(seed + 1)
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / 1e3 / n_ang


def run_denoise_eval(args):
    """Photons and seconds per projection needed to reach <= 2% relative L2
    scatter error against a high-photon reference, for plain Monte Carlo, the
    paper's Savitzky-Golay smoothing (Sec. II-C.4) and the learned denoiser
    trained here on pairs this Monte Carlo produces: 256^2 x 0.5 mm scatter
    images of 256^3 x 0.25 mm cylinder/rod phantoms (60 keV, SOD/SDD 300/600,
    step 0.5 mm), inputs at --train-inputs photons, targets at
    --target-photons.  --save-weights writes the trained network."""
    import threading

    import torch

    import paper_2201_13191_gb300 as mcx

    mcx.build()
    ctx, _ = c4_context(mcx)
    rng = np.random.default_rng(0)
    low_levels = [float(x) for x in args.train_inputs]
    t0 = time.perf_counter()
    xs, ys = [], []
    # phantoms are built on the host one ahead of the GPU
    nxt = {}

    def build(k):
        nxt[k] = c4_phantom(k)

    th = threading.Thread(target=build, args=(0,))
    th.start()
    for k in range(args.train_phantoms):
        th.join()
        v = nxt.pop(k)
        if k + 1 < args.train_phantoms:
            th = threading.Thread(target=build, args=(k + 1,))
            th.start()
        ctx.load_volume(v["mat"], v["rho"], v["spacing"])
        for j in range(args.train_angles):
            ang = float(rng.uniform(0, 2 * np.pi))
            hi, _ = c4_scatter(ctx, args.target_photons, ang, 1_000_000 + 7919 * k + j)
            for q, nl in enumerate(low_levels):
                lo, _ = c4_scatter(ctx, nl, ang, 2_000_000 + 104729 * k + 31 * j + q)
                xs.append(lo.clone())
                ys.append(hi)
    X = torch.stack(xs)
    Y = torch.stack(ys)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    ctx.denoise_init(C4_PX, C4_PX, 16, seed=1)
    t0 = time.perf_counter()
    losses = []
    order = torch.randperm(len(X), generator=torch.Generator().manual_seed(0))
    pos = 0
    for it in range(args.train_steps):
        lr = 1e-3 * 0.5 * (1 + np.cos(np.pi * it / args.train_steps)) + 2e-5
        if pos + 16 > len(X):
            order = torch.randperm(len(X), generator=torch.Generator().manual_seed(it))
            pos = 0
        idx = order[pos : pos + 16]
        pos += 16
        losses.append(ctx.denoise_train_step(X[idx], Y[idx], lr))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    if args.save_weights:
        ctx.denoise_save(args.save_weights)
    angles = [2 * np.pi * a / args.eval_angles + 0.1 for a in range(args.eval_angles)]
    grid = [1e5, 2e5, 5e5, 1e6, 2e6, 5e6, 1e7, 2e7, 5e7, 1e8, 2e8, 5e8, 1e9]
    t0 = time.perf_counter()
    res = c4_curves(ctx, angles, args.ref_photons, grid)
    line = {
        "metric": "s/projection at <=2% relative L2 scatter error vs a high-photon reference",
        "unit": "s/projection", "higher_is_better": False,
        "config": {"workload": f"cylinder/rod family, {C4_N}^3 x {C4_DV} mm, {C4_PX}^2 x {128.0 / C4_PX} mm panel, "
                               f"60 keV, step {C4_STEP} mm",
                   "train_phantoms": args.train_phantoms, "train_angles": args.train_angles,
                   "train_pairs": int(len(X)), "train_inputs_photons": low_levels,
                   "train_target_photons": args.target_photons, "train_steps": args.train_steps,
                   "reference_photons": args.ref_photons, "eval_angles": args.eval_angles,
                   "held_out_phantom_seed": C4_HELD_OUT,
                   "denoiser": "residual U-Net, 4 levels, 32 base channels, BF16"},
        **res,
        "train_loss_first_last": [float(np.mean(losses[:20])), float(np.mean(losses[-20:]))],
        "seconds": {"data": t_data, "train": t_train, "eval": time.perf_counter() - t0},
    }
    print(json.dumps(line), flush=True)


UNET_CONVS = [(16, 32, 0), (32, 32, 0), (32, 64, 1), (64, 64, 1), (64, 128, 2), (128, 128, 2), (128, 256, 3),
              (256, 256, 3), (384, 128, 2), (128, 128, 2), (192, 64, 1), (64, 64, 1), (96, 32, 0), (32, 32, 0),
              (32, 16, 0)]  # (C_in, C_out, level) of the denoiser's 15 convolutions


def run_conv_bench(args):
    """Tensor-core throughput of the denoiser's 3x3 convolutions: every layer
    shape of the U-Net, forward (mc_nn_conv3x3) and weight gradient
    (mc_nn_conv3x3_wgrad), on a batch of images, plus the inference latency of
    the whole network (mc_denoise_infer).  Roofline: dense BF16 tensor peak."""
    import ctypes as C

    import torch

    import paper_2201_13191_gb300 as mcx
    from paper_2201_13191_gb300.binding import library

    mcx.build()
    L = library()
    H = W = args.conv_size
    B = args.conv_batch
    stream = torch.cuda.current_stream()
    sh = C.c_void_p(stream.cuda_stream)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    peaks = measured_peaks()
    peak = float(peaks.get("bf16_tflops", 1891.8))
    reps = 10

    def timed(fn):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    def ptr(t):
        return C.c_void_p(t.data_ptr())

    layers, fl_f, ms_f, fl_w, ms_w = [], 0.0, 0.0, 0.0, 0.0
    g = torch.Generator(device="cuda").manual_seed(0)
    for i, (ci, co, lv) in enumerate(UNET_CONVS):
        h, w = H >> lv, W >> lv
        x = torch.randn((B, h, w, ci), device="cuda", generator=g).to(torch.bfloat16)
        wt = (0.05 * torch.randn((co, 9, ci), device="cuda", generator=g)).to(torch.bfloat16)
        bias = torch.zeros(co, device="cuda")
        y = torch.empty((B, h, w, co), dtype=torch.bfloat16, device="cuda")
        dy = torch.randn((B, h, w, co), device="cuda", generator=g).to(torch.bfloat16)
        dw = torch.zeros((co, 9, ci), device="cuda")
        npx = B * h * w
        ktiles = (9 * ci + 127) // 128
        splits = max(1, min(npx // 256, 4 * 152 // ktiles + 1))

        def fwd():
            if L.mc_nn_conv3x3(ptr(x), ptr(wt), ptr(bias), ptr(y), B, h, w, ci, co, 1, 0, ptr(err), sh):
                raise RuntimeError("mc_nn_conv3x3 failed")

        def wgrad():
            if L.mc_nn_conv3x3_wgrad(ptr(x), ptr(dy), ptr(dw), B, h, w, ci, co, splits, ptr(err), sh):
                raise RuntimeError("mc_nn_conv3x3_wgrad failed")

        flop = 2.0 * 9 * ci * co * npx
        tf, tw = timed(fwd), timed(wgrad)
        layers.append({"layer": i, "cin": ci, "cout": co, "hw": f"{h}x{w}", "fwd_ms": tf, "fwd_tflops": flop / tf / 1e9,
                       "wgrad_ms": tw, "wgrad_tflops": flop / tw / 1e9, "wgrad_splits": splits})
        fl_f += flop
        ms_f += tf
        fl_w += flop
        ms_w += tw
    torch.cuda.synchronize()
    if int(err.item()):
        raise RuntimeError("a tensor-core wait gave up")
    # sustained rate of the MMA shape each layer issues (M = 128, N = C_out tile, K = 16), measured live
    PL = probe_library()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    shape_peak = {}
    for nt in (16, 32, 64, 128, 256):
        rounds = 4096
        ms = timed(lambda: PL.mc_probe_mma(nt, sms, rounds, ptr(err), sh))
        shape_peak[nt] = sms * rounds * 4 * 2.0 * 128 * nt * 16 / ms / 1e9
    torch.cuda.synchronize()
    if int(err.item()):
        raise RuntimeError("a tensor-core wait gave up")

    def tile_n(co):
        n = 16
        while n < co and n < 256:
            n *= 2
        return n

    shape_time = sum(2.0 * 9 * ci * co * B * (H >> lv) * (W >> lv) / shape_peak[tile_n(co)] / 1e9
                     for ci, co, lv in UNET_CONVS)
    ctx = mcx.Context(0)
    ctx.denoise_init(H, W, B, seed=1)
    imgs = torch.rand((B, H, W), device="cuda", generator=g) + 0.5
    out = torch.empty_like(imgs)
    t_batch = timed(lambda: ctx.denoise_infer(imgs, out=out, stream=stream))
    t_one = timed(lambda: ctx.denoise_infer(imgs[:1], out=out[:1], stream=stream))
    net_flop = sum(2.0 * 9 * ci * co * (H >> lv) * (W >> lv) for ci, co, lv in UNET_CONVS)
    best = max(layers, key=lambda r: r["fwd_tflops"])
    line = {
        "metric": "denoiser 3x3 convolution throughput (tcgen05 kind::f16, BF16 operands, FP32 accumulation)",
        "value": fl_f / ms_f / 1e9, "unit": "TFLOP/s", "higher_is_better": True, "dtype": "bf16",
        "config": {"workload": f"U-Net layer shapes at {H}x{W}, batch {B}", "reps": reps},
        "roofline": {"bound": "tensor", "achieved": fl_f / ms_f / 1e9, "peak": peak, "unit": "TFLOP/s",
                     "frac": fl_f / ms_f / 1e9 / peak, "traffic": None,
                     "kernel": "k_conv3x3_fwd over the 15 layer shapes (FLOP-weighted)",
                     "peak_basis": "MEASURED_PEAKS bf16_tflops (cuBLAS burst)",
                     "best_layer": {"layer": best["layer"], "tflops": best["fwd_tflops"],
                                    "frac": best["fwd_tflops"] / peak},
                     "mma_shape_peak_tflops": shape_peak,
                     "shape_limited_peak": fl_f / shape_time / 1e9,
                     "frac_of_shape_limited_peak": (fl_f / ms_f) / (fl_f / shape_time),
                     "shape_note": "tcgen05.mma M=128 x N x K=16 issue rate measured live per N (mc_probe_mma); the "
                                   "layers' C_out tile sets N, so the FLOP-weighted attainable peak is lower than the "
                                   "dense GEMM figure"},
        "wgrad": {"achieved": fl_w / ms_w / 1e9, "frac": fl_w / ms_w / 1e9 / peak},
        "layers": layers,
        "inference": {"batch": B, "batch_ms": t_batch, "one_image_ms": t_one,
                      "net_gflop_per_image": net_flop / 1e9,
                      "batch_tflops": B * net_flop / t_batch / 1e9, "one_image_tflops": net_flop / t_one / 1e9},
    }
    print(json.dumps(line), flush=True)


def run_correct_eval(args):
    """Iterative scatter correction (Sec. II-E, eq. Correction) on a
    high-resolution flat panel: per-iteration time and the cupping error of the
    corrected reconstruction against the scatter-free one.

    Measurements: exact primary (eq. Ip) on the full panel at every angle plus
    Monte Carlo scatter simulated at a subset of angles on a coarse grid,
    smoothed and interpolated to all angles and the full panel (the paper's own
    interpolation step), with Poisson noise of the stated photon budget."""
    import torch

    import paper_2201_13191_gb300 as mcx
    from mc_inputs import cylinder_variant_phantom, default_table_path, ellipsoid_phantom, mono_spectrum

    mcx.build()
    tp = default_table_path("full", tempfile.mkdtemp(prefix="mccor"))
    NU = NV = args.cor_detector
    P = args.cor_pixel
    n_proj = args.cor_proj
    nvx, dv = args.cor_volume, args.cor_voxel
    SOD, SDD = 300.0, 600.0
    step = args.cor_step
    angles = (2.0 * np.pi * np.arange(n_proj) / n_proj).astype(np.float32)
    if args.cor_phantom == "cylinder":
        vol = cylinder_variant_phantom(args.cor_seed, n=nvx, dv=dv)
    else:
        vol = ellipsoid_phantom(n=nvx, dv=dv, seed=args.cor_seed)
    E, w = mono_spectrum(60.0)
    ctx = mcx.Context(0)
    ctx.load_tables(tp)
    ctx.set_spectrum(E, w)
    ctx.set_geometry(SOD, SDD, NU, NV, P, P)
    dev = torch.device("cuda")
    t_meas = time.perf_counter()
    # flat field: the primary of an empty volume
    empty = np.zeros_like(vol["rho"])
    ctx.load_volume(vol["mat"], empty, vol["spacing"])
    I0 = ctx.project([0.0], 1, step, 1, scatter=False)["primary"][0].clone()
    ctx.load_volume(vol["mat"], vol["rho"], vol["spacing"])
    ip = torch.empty((n_proj, NV, NU), dtype=torch.float32, device=dev)
    chunk = 64
    for k in range(0, n_proj, chunk):
        ctx.project(angles[k : k + chunk], 1, step, 1, scatter=False, out={"primary": ip[k : k + chunk]})
    g = args.cor_meas_grid
    meas_angles = angles[:: n_proj // args.cor_meas_angles]
    ctx.set_geometry(SOD, SDD, g, g, P * NU / g, P * NV / g)
    is_meas = ctx.project(meas_angles, int(args.cor_meas_photons), step, 77, primary=False)["scatter"]
    ctx.set_geometry(SOD, SDD, NU, NV, P, P)
    # measured intensity with Poisson noise: N0 photons per unattenuated pixel
    N0 = args.cor_total_photons / (NU * NV)
    raw = torch.empty_like(ip)
    gen = torch.Generator(device=dev).manual_seed(5)
    for k in range(0, n_proj, chunk):
        sl = slice(k, k + chunk)
        # per-pixel values scale with the pixel area: (coarse pixel -> panel pixel)
        isk = ctx.smooth_upsample(is_meas, meas_angles, angles[sl], NU, NV) * ((g / NU) * (g / NV))
        lam = N0 * (ip[sl] + isk) / I0
        raw[sl] = torch.poisson(lam, generator=gen).clamp_min_(0.5) / N0 * I0
        del isk, lam
    torch.cuda.synchronize()
    t_meas = time.perf_counter() - t_meas
    grid = (nvx, nvx, nvx, dv, dv, dv)
    # scatter-free and uncorrected reconstructions (line integrals computed in place)
    sub = slice(0, n_proj, max(1, n_proj // 64))
    a_ref_sub = -torch.log(ip[sub] / I0)
    for k in range(0, n_proj, chunk):
        ip[k : k + chunk] = -torch.log(ip[k : k + chunk] / I0)
    v_ref = ctx.fdk(ip, angles, NU, NV, grid)
    for k in range(0, n_proj, chunk):
        ip[k : k + chunk] = -torch.log(raw[k : k + chunk] / I0)
    a_raw_sub = ip[sub].clone()
    v_raw = ctx.fdk(ip, angles, NU, NV, grid)
    del ip
    torch.cuda.empty_cache()
    stride = max(1, int(round(n_proj / args.cor_sim_angles)))
    prm = mcx.CorrectParams(nx=nvx, ny=nvx, nz=nvx, dx=dv, dy=dv, dz=dv, sim_nu=args.cor_sim_grid,
                            sim_nv=args.cor_sim_grid, sim_angle_stride=stride, photons=int(args.cor_sim_photons),
                            step_mm=step, seed=11, classes=3, class_material=(0, 1, 3), class_density0=0.001205,
                            e_eff_keV=60.0, mu_lo=-0.01, mu_hi=0.12, primary_full_res=1, mc_bin=args.cor_mc_bin)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out, v_cor, secs = ctx.correct_iter(raw, I0, angles, NU, NV, args.cor_iters, prm)
    torch.cuda.synchronize()
    t_total = time.perf_counter() - t0
    obj = torch.from_numpy(vol["mat"] != 0).to(dev)
    soft = torch.from_numpy((vol["mat"] == 1) | (vol["mat"] == 2)).to(dev)

    def verr(v, mask):
        """Relative L2 of 8x8x8-block means over blocks lying wholly inside the mask: the low-frequency
        (cupping, shading) error, with the voxel noise averaged out."""
        k = 8
        m = mask[: nvx // k * k, : nvx // k * k, : nvx // k * k].float()
        pool = lambda t: torch.nn.functional.avg_pool3d(t[None, None], k)[0, 0]
        inside = pool(m) > 0.999
        a, b = pool(v[: nvx // k * k, : nvx // k * k, : nvx // k * k]), pool(
            v_ref[: nvx // k * k, : nvx // k * k, : nvx // k * k])
        return float(torch.linalg.norm((a - b)[inside]) / torch.linalg.norm(b[inside]))

    def aerr(a):
        return float(torch.linalg.norm(a - a_ref_sub) / torch.linalg.norm(a_ref_sub))

    def cupping(v):
        """Radial profile of the central slice over water voxels: (ring - centre) / ring, in per cent,
        with the centre r < 0.2 R and the ring 0.7 R < r < 0.9 R (R the water extent)."""
        zc = nvx // 2
        sl = v[zc]
        water = torch.from_numpy(vol["mat"][zc] == 1).to(dev)
        yy, xx = torch.meshgrid(torch.arange(nvx, device=dev), torch.arange(nvx, device=dev), indexing="ij")
        r = torch.sqrt((xx - (nvx - 1) / 2.0) ** 2 + (yy - (nvx - 1) / 2.0) ** 2)
        R = float(r[water].max()) if bool(water.any()) else 1.0
        centre = water & (r < 0.2 * R)
        ring = water & (r > 0.7 * R) & (r < 0.9 * R)
        if not bool(centre.any()) or not bool(ring.any()):
            return None
        mc, mr = float(sl[centre].mean()), float(sl[ring].mean())
        return 100.0 * (mr - mc) / mr

    line = {
        "metric": "iterative scatter correction: seconds per iteration and cupping error vs the scatter-free "
                  "reconstruction",
        "unit": "s/iteration", "higher_is_better": False, "dtype": "f32",
        "value": float(np.mean(secs)) if secs else None,
        "config": {"workload": f"{n_proj} projections of {NU}x{NV} at {P} mm, {nvx}^3 x {dv} mm {args.cor_phantom} "
                               f"phantom (seed {args.cor_seed}), 60 keV, SOD/SDD {SOD:.0f}/{SDD:.0f}",
                   "measurements": f"exact primary + Monte Carlo scatter at {len(meas_angles)} angles x "
                                   f"{args.cor_meas_photons:.0e} photons on {g}^2, smoothed and interpolated; Poisson "
                                   f"noise with {args.cor_total_photons:.0e} photons per projection",
                   "mc_volume": f"{nvx // 2}^3 x {2 * dv} mm (down-sampled)" if args.cor_mc_bin == 2 else f"{nvx}^3",
                   "iteration": f"FDK to {nvx}^3, Otsu 3 classes, primary on the full panel, scatter at "
                                f"{len(range(0, n_proj, stride))} angles x {args.cor_sim_photons:.0e} photons on "
                                f"{args.cor_sim_grid}^2, Savitzky-Golay, angular lerp + cubic up-sampling, eq. Correction",
                   "iterations": args.cor_iters, "step_mm": step},
        "seconds_per_iteration": secs, "seconds_total": t_total, "seconds_measurements": t_meas,
        "cupping_error": {"uncorrected": verr(v_raw, obj), "corrected": verr(v_cor, obj),
                          "uncorrected_soft_tissue": verr(v_raw, soft), "corrected_soft_tissue": verr(v_cor, soft),
                          "definition": "relative L2 of 8^3-block means of mu against the scatter-free "
                                        "reconstruction, over blocks wholly inside the object"},
        "line_integral_rel_l2": {"uncorrected": aerr(a_raw_sub), "corrected": aerr(out[sub])},
        "cupping_percent": {"scatter_free": cupping(v_ref), "uncorrected": cupping(v_raw), "corrected": cupping(v_cor),
                            "definition": "central slice, water voxels: 100 (ring - centre) / ring, centre r < 0.2 R, "
                                          "ring 0.7 R < r < 0.9 R"},
    }
    print(json.dumps(line), flush=True)


def run_vr_eval(args):
    """Variance reduction of the point-detector scoring on the bench workload:
    transport time, relative L2 noise of the scatter image (batch estimate) and
    the figure of merit 1 / (noise^2 x time) of the paper's sampled-type scoring
    and of expected-value scoring; then, on a coarse panel of the same extent
    (--vr-panel pixels a side, the size of the correction's simulation grids),
    the same two and forced detection (every pixel scored once per interaction)
    alone and with expected-value scoring."""
    import torch

    import paper_2201_13191_gb300 as mcx

    mcx.build()
    tp, wl = make_inputs(tempfile.mkdtemp(prefix="mcvr"), args.photons or 1e7, args.workload)

    def measure(wl, N, **opt):
        ctx = mcx.Context(0, n_batches=20, **opt)
        ctx.load_tables(tp)
        ctx.setup(wl)
        ms, noise = [], []
        for k in range(args.warmup + args.steps):
            out = ctx.project([0.0], N, wl["step_mm"], 100 + k, primary=False, variance=True)
            st = ctx.last_stats()
            if k >= args.warmup:
                img = out["scatter"][0].double()
                var = out["variance"][0].double()
                ms.append(st["transport_ms"])
                noise.append(float(torch.sqrt(var.sum()) / torch.linalg.norm(img)))
        t = float(np.mean(ms)) / 1e3
        n2 = float(np.mean(np.square(noise)))
        ctx.close()
        return {"transport_s": t, "histories_per_s": N / t, "rel_l2_noise": float(np.sqrt(n2)),
                "figure_of_merit": 1.0 / (n2 * t)}

    N = wl["n_photons"]
    res = {mode: measure(wl, N, nee_mode=mode) for mode in (0, 1)}
    g = wl["geometry"]
    P = args.vr_panel
    coarse = dict(wl, geometry=dict(g, nu=P, nv=P, pu=g["pu"] * g["nu"] / P, pv=g["pv"] * g["nv"] / P))
    Nc = int(args.vr_photons)
    modes = {"paper": dict(nee_mode=0), "expected_value": dict(nee_mode=1),
             "forced_detection": dict(forced_detection=1), "forced_detection_expected_value":
             dict(forced_detection=1, nee_mode=1)}
    cres = {name: measure(coarse, Nc, **opt) for name, opt in modes.items()}
    for name in cres:
        cres[name]["fom_gain"] = cres[name]["figure_of_merit"] / cres["paper"]["figure_of_merit"]
    line = {
        "metric": "figure of merit 1/(relative L2 noise^2 x transport time) of the scatter image",
        "unit": "1/s", "higher_is_better": True,
        "config": {"workload": args.workload, "photons": N, "batches": 20, "steps": args.steps,
                   "coarse_panel": f"{P}x{P} over the same extent", "coarse_photons": Nc},
        "paper_scoring": res[0], "expected_value_scoring": res[1],
        "fom_gain": res[1]["figure_of_merit"] / res[0]["figure_of_merit"],
        "coarse_panel": cres,
    }
    print(json.dumps(line), flush=True)


def run_tally_eval(args):
    """Tally modes on the bench workload: transport time, relative L2 noise of the
    scatter image and figure of merit 1 / (noise^2 x time) of the global tally and
    of tile-stratified tallies of several tile sizes.  The noise is taken two ways:
    from the batch variance (10 batches) and from the spread of the images of
    independent seeds; also the distance of each mean image from the global one in
    units of the combined noise (the tile-stratified estimator is unbiased)."""
    import torch

    import paper_2201_13191_gb300 as mcx

    mcx.build()
    tp, wl = make_inputs(tempfile.mkdtemp(prefix="mctally"), args.photons or 1e8, args.workload)
    N = wl["n_photons"]
    modes = [("global", 1, 64)] + [(f"tiled {t}x{t}", 4, t) for t in (8, 16, 24, 32)]
    res, imgs = {}, {}
    for name, mode, t in modes:
        ctx = mcx.Context(0, n_batches=10, tally_mode=mode, tile_u=t, tile_v=t)
        ctx.load_tables(tp)
        ctx.setup(wl)
        ms, noise, runs = [], [], []
        for k in range(args.warmup + args.steps):
            out = ctx.project([0.0], N, wl["step_mm"], 100 + k, primary=False, variance=True)
            st = ctx.last_stats()
            if k >= args.warmup:
                img = out["scatter"][0].double()
                var = out["variance"][0].double()
                ms.append(st["transport_ms"])
                noise.append(float(torch.sqrt(var.sum()) / torch.linalg.norm(img)))
                runs.append(img)
        t_s = float(np.mean(ms)) / 1e3
        n2 = float(np.mean(np.square(noise)))
        R = torch.stack(runs)
        mean = R.mean(0)
        run_var = R.var(0, unbiased=True)  # per run
        n2_runs = float(run_var.sum() / (mean * mean).sum())
        imgs[name] = (mean, run_var / len(runs))
        res[name] = {"transport_s": t_s, "histories_per_s": N / t_s, "rel_l2_noise_batches": float(np.sqrt(n2)),
                     "rel_l2_noise_runs": float(np.sqrt(n2_runs)), "figure_of_merit": 1.0 / (n2_runs * t_s)}
    g_img, g_var = imgs["global"]
    for name in res:
        if name == "global":
            continue
        m, v = imgs[name]
        res[name]["mean_diff_over_noise"] = float(torch.linalg.norm(m - g_img) / torch.sqrt((v + g_var).sum()))
        res[name]["fom_gain"] = res[name]["figure_of_merit"] / res["global"]["figure_of_merit"]
    line = {"metric": "figure of merit 1/(relative L2 noise^2 x transport time) by tally mode", "unit": "1/s",
            "higher_is_better": True,
            "config": {"workload": args.workload, "photons": N, "batches": 10, "steps": args.steps},
            "modes": res}
    print(json.dumps(line), flush=True)


def run_primary_bench(args):
    """Deterministic primary images (eq. Ip) of the correction workload: 512^3 x 0.2 mm
    cylinder phantom (brick layout, HBM-resident), 2048^2 x 0.1 mm panel, step 0.2 mm,
    64 angles per call: rays/s and march steps/s."""
    import torch

    import paper_2201_13191_gb300 as mcx
    from mc_inputs import cylinder_variant_phantom, default_table_path, mono_spectrum

    mcx.build()
    tp = default_table_path("full", tempfile.mkdtemp(prefix="mcprim"))
    nvx, dv, NU, P, step = args.cor_volume, args.cor_voxel, args.cor_detector, args.cor_pixel, args.cor_step
    vol = cylinder_variant_phantom(args.cor_seed, n=nvx, dv=dv)
    if args.primary_speckle > 0:
        # a segmented reconstruction's misclassified voxels: a fraction of them take another material
        rng = np.random.default_rng(3)
        flip = rng.random(vol["mat"].shape) < args.primary_speckle
        vol = dict(vol, mat=vol["mat"].copy())
        vol["mat"][flip] = rng.choice(np.array([0, 1, 3], np.uint8), size=int(flip.sum()))
    ctx = mcx.Context(0)
    ctx.load_tables(tp)
    ctx.set_spectrum(*mono_spectrum(60.0))
    ctx.set_geometry(300.0, 600.0, NU, NU, P, P)
    ctx.load_volume(vol["mat"], vol["rho"], vol["spacing"])
    n_ang = 64
    angles = (2.0 * np.pi * np.arange(n_ang) / n_ang).astype(np.float32)
    out = {"primary": ctx.empty_images(n_ang)}
    st = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        ctx.project(angles, 1, step, 1, scatter=False, out=out, stream=st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        ctx.project(angles, 1, step, 1, scatter=False, out=out, stream=st)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    rays = NU * NU * n_ang
    # march steps: each ray's chord through the volume box over the step, summed on the host
    s_pos = 300.0 * np.stack([np.cos(angles), np.sin(angles), np.zeros(n_ang)], 1)
    c_pos = -300.0 * np.stack([np.cos(angles), np.sin(angles), np.zeros(n_ang)], 1)
    u = (np.arange(0, NU, 8) + 0.5 - NU / 2) * P
    half = nvx * dv / 2
    steps = 0.0
    for a in range(n_ang):
        eu = np.array([-np.sin(angles[a]), np.cos(angles[a]), 0.0])
        Pp = c_pos[a] + u[:, None, None] * eu + u[None, :, None] * np.array([0.0, 0.0, 1.0])
        w = Pp - s_pos[a]
        w /= np.linalg.norm(w, axis=-1, keepdims=True)
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = (-half - s_pos[a]) / w
            t2 = (half - s_pos[a]) / w
        ta = np.nanmax(np.minimum(t1, t2), -1)
        tb = np.nanmin(np.maximum(t1, t2), -1)
        L = np.clip(tb - ta, 0, None)
        steps += float(np.sum(np.where(L > 0, np.maximum(1, np.ceil(L / step)), 0))) * 64  # 8x8 subsampled
    line = {"metric": "primary rays/s (eq. Ip, exact column masses)", "value": rays / (ms / 1e3), "unit": "rays/s",
            "higher_is_better": True, "dtype": "f32",
            "config": {"workload": f"{nvx}^3 x {dv} mm cylinder phantom, {NU}^2 x {P} mm panel, step {step} mm, "
                                   f"{n_ang} angles per call", "speckle": args.primary_speckle, "steps": args.steps},
            "ms_per_call": ms, "ms_per_projection": ms / n_ang, "march_steps_per_s": steps / (ms / 1e3)}
    print(json.dumps(line), flush=True)


def run_fdk_bench(args):
    """FDK reconstruction (ramp filter + voxel-driven backprojection) of 256 projections
    of 2048^2 x 0.1 mm into 512^3 x 0.2 mm: milliseconds and voxel-projection updates/s."""
    import torch

    import paper_2201_13191_gb300 as mcx

    mcx.build()
    NU, P, nvx, dv, n_proj = args.cor_detector, args.cor_pixel, args.cor_volume, args.cor_voxel, 256
    ctx = mcx.Context(0)
    ctx.set_geometry(300.0, 600.0, NU, NU, P, P)
    angles = (2.0 * np.pi * np.arange(n_proj) / n_proj).astype(np.float32)
    g = torch.Generator(device="cuda").manual_seed(1)
    p = torch.rand((n_proj, NU, NU), device="cuda", generator=g)
    grid = (nvx, nvx, nvx, dv, dv, dv)
    for _ in range(max(1, args.warmup)):
        ctx.fdk(p, angles, NU, NU, grid)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ctx.fdk(p, angles, NU, NU, grid)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    upd = float(nvx) ** 3 * n_proj
    line = {"metric": "FDK voxel-projection updates/s", "value": upd / (ms / 1e3), "unit": "updates/s",
            "higher_is_better": True, "dtype": "f32",
            "config": {"workload": f"{n_proj} projections of {NU}^2 x {P} mm -> {nvx}^3 x {dv} mm", "steps": args.steps},
            "ms_per_fdk": ms}
    print(json.dumps(line), flush=True)


def run_upsample_bench(args):
    """Smoothing and dual interpolation of the correction workload (Sec. II-C.3, II-C.4):
    171 scatter images of 256^2 (every 6th of 1024 angles) -> 1024 angles of 2048^2:
    milliseconds and output bytes/s against the measured HBM copy peak."""
    import torch

    import paper_2201_13191_gb300 as mcx

    mcx.build()
    n_out, NU, n_in, g = args.cor_proj, args.cor_detector, 171, args.cor_sim_grid
    ctx = mcx.Context(0)
    ctx.set_geometry(300.0, 600.0, NU, NU, 0.1, 0.1)
    in_angles = (2.0 * np.pi * np.arange(n_in) / n_in).astype(np.float32)
    out_angles = (2.0 * np.pi * np.arange(n_out) / n_out).astype(np.float32)
    gen = torch.Generator(device="cuda").manual_seed(2)
    img = torch.rand((n_in, g, g), device="cuda", generator=gen)
    out = torch.empty((n_out, NU, NU), device="cuda")
    for _ in range(max(1, args.warmup)):
        ctx.smooth_upsample(img, in_angles, out_angles, NU, NU, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ctx.smooth_upsample(img, in_angles, out_angles, NU, NU, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    written = 4.0 * n_out * NU * NU
    peak = float(measured_peaks().get("hbm_gbs", 6801.0))
    line = {"metric": "scatter smoothing + angular lerp + cubic up-sampling, output GB/s", "unit": "GB/s",
            "value": written / (ms / 1e3) / 1e9, "higher_is_better": True, "dtype": "f32",
            "config": {"workload": f"{n_in} images of {g}^2 -> {n_out} x {NU}^2", "steps": args.steps},
            "ms": ms, "roofline": {"bound": "hbm", "peak": peak, "frac": written / (ms / 1e3) / 1e9 / peak,
                                   "unit": "GB/s"}}
    print(json.dumps(line), flush=True)


def run_mesh_bench(args):
    """Primary images of the triangle-mesh (CAD) cylinder-rod phantom by ray casting
    (eq. Ip with exact path lengths): rays per second through the hierarchy."""
    import torch

    import paper_2201_13191_gb300 as mcx
    from mc_inputs import default_table_path, kramers_spectrum, read_tables
    from mc_inputs.meshes import cylinder_rod_mesh

    mcx.build()
    tp = default_table_path("full", tempfile.mkdtemp(prefix="mcmesh"))
    T = read_tables(tp)
    mesh = cylinder_rod_mesh(args.mesh_segments)
    ctx = mcx.Context(0)
    ctx.load_tables(tp)
    ctx.set_spectrum(*kramers_spectrum(T))
    ctx.set_geometry(300.0, 600.0, 512, 512, 0.25, 0.25)
    ctx.load_mesh(mesh)
    n_ang = args.angles if args.angles > 1 else 36
    angles = (2.0 * np.pi * np.arange(n_ang) / n_ang).astype(np.float32)
    out = {"primary": ctx.empty_images(n_ang)}
    st = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        ctx.project(angles, 1, 0.25, 1, scatter=False, out=out, stream=st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        ctx.project(angles, 1, 0.25, 1, scatter=False, out=out, stream=st)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    rays = 512 * 512 * n_ang
    # Monte Carlo scatter through the same surfaces: one projection per step
    N = int(args.photons) if args.photons else 10_000_000
    sc = {"scatter": ctx.empty_images(1)}
    for _ in range(max(3, args.warmup)):
        ctx.project(angles[:1], N, 0.25, 1, primary=False, out=sc, stream=st)
    e0.record(st)
    for k in range(args.steps):
        ctx.project(angles[:1], N, 0.25, 2 + k, primary=False, out=sc, stream=st)
    e1.record(st)
    torch.cuda.synchronize()
    ms_sc = e0.elapsed_time(e1) / args.steps
    stt = ctx.last_stats()
    ray_casts = stt["nee_rays"] + stt["compton"] + stt["rayleigh"] + stt["photo"] + stt["escape"]
    line = {"metric": "mesh primary rays/s (CAD surface model, BVH ray casting)", "value": rays / (ms / 1e3),
            "unit": "rays/s", "higher_is_better": True, "dtype": "f32",
            "config": {"workload": f"cylinder-rod surfaces, {len(mesh['triangles'])} triangles, 512^2 x 0.25 mm, "
                                   f"{n_ang} angles, 111-bin spectrum", "steps": args.steps},
            "ms_per_step": ms, "ms_per_projection": ms / n_ang,
            "scatter": {"photons_per_projection": N, "ms_per_projection": ms_sc,
                        "histories_per_s": N / (ms_sc / 1e3),
                        "flight_and_detector_rays_per_s": ray_casts / (ms_sc / 1e3),
                        "surface_crossings_per_history": (stt["flight_steps"] + stt["nee_steps"]) / N,
                        "n_split": 10}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.denoise_eval:
        run_denoise_eval(args)
    elif args.conv_bench:
        run_conv_bench(args)
    elif args.correct_eval:
        run_correct_eval(args)
    elif args.vr_eval:
        run_vr_eval(args)
    elif args.mesh_bench:
        run_mesh_bench(args)
    elif args.tally_eval:
        run_tally_eval(args)
    elif args.primary_bench:
        run_primary_bench(args)
    elif args.fdk_bench:
        run_fdk_bench(args)
    elif args.upsample_bench:
        run_upsample_bench(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
