"""Build the CUDA libraries in-tree for sm_103a (GB300).

libmc.so is the product (include/mc.h); libmcprobe.so holds the benchmark's
measurement kernels (include/mc_probe.h), kept out of the product.  Each
translation unit is compiled in parallel with nvcc and linked into its shared
library with the CUDA runtime linked statically.  No PyTorch types cross the
library boundary; the Python bindings load them with ctypes.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libmc.so")
PROBE_OUT = os.path.join(HERE, "libmcprobe.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["mc_api.cu", "k_transport.cu", "k_primary.cu", "k_post.cu", "k_static.cu", "k_conv.cu", "k_nn.cu",
           "denoiser.cu", "k_recon.cu", "k_mesh.cu"]
PROBE_SOURCES = ["probe/k_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]
# Per translation unit: the transport takes division and square root in their
# fast forms (within 2 ulp; denormals flushed): its per-ray set-up divides
# several times (chord clipping, step length, pdf factors), and the IEEE forms
# cost 7% of the kernel.  The primary image keeps IEEE division (its 1e-5 bar).
SOURCE_FLAGS = {"k_transport.cu": ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"]}


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(out, sources, header):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if not os.path.isdir(os.path.join(CSRC, f))]
    deps += [os.path.join(CSRC, f) for f in sources]
    deps.append(os.path.join(os.path.dirname(HERE), "include", header))
    return any(os.path.exists(f) and os.path.getmtime(f) > t for f in deps)


def build(force=False, verbose=False, extra=()):
    """libmc.so, the product library."""
    return _build(OUT, SOURCES, "mc.h", force, verbose, extra)


def build_probe(force=False, verbose=False, extra=()):
    """libmcprobe.so, the benchmark's measurement kernels."""
    return _build(PROBE_OUT, PROBE_SOURCES, "mc_probe.h", force, verbose, extra)


def _build(out, sources, header, force, verbose, extra):
    if not force and not _stale(out, sources, header):
        return out
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace("/", "_").replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *SOURCE_FLAGS.get(src, []), *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(sources)) as ex:
        objs = list(ex.map(compile_one, sources))
    tmp = out + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    kw = dict(force="--force" in sys.argv, verbose=True, extra=("-Xptxas", "-v") if "--ptxas" in sys.argv else ())
    build(**kw)
    build_probe(**kw)
