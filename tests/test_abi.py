"""The C-ABI library builds, loads, and exports every entry point include/mc.h declares.

No compute calls: these run without a GPU.
"""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header="mc.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2201_13191_gb300 as mcx

    mcx.build()
    return mcx.library()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mc_create", "mc_load_volume", "mc_set_spectrum", "mc_set_geometry", "mc_project",
              "mc_smooth_upsample", "mc_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_probe_library_is_separate_and_exports_its_header():
    """The measurement kernels live in libmcprobe.so, not in the product library."""
    import ctypes as C

    from paper_2201_13191_gb300.build import build_probe

    probe = C.CDLL(build_probe())
    names = _declared("mc_probe.h")
    assert names == ["mc_probe_gather", "mc_probe_mma", "mc_probe_stream"]
    for n in names:
        assert hasattr(probe, n), n
        assert n not in _declared("mc.h")


def test_binding_names_match_header():
    from paper_2201_13191_gb300.binding import EXPORTED

    assert sorted(EXPORTED) == _declared()


def test_default_options(lib):
    import ctypes as C

    from paper_2201_13191_gb300.binding import Options

    o = Options()
    lib.mc_default_options(C.byref(o))
    assert o.n_split == 10 and o.sg_window == 9 and o.sg_order == 3 and abs(o.cubic_a + 0.5) < 1e-7
    assert o.max_scatter_order == 64 and o.n_batches == 1


def test_product_path_has_no_oracle_dependency():
    pkg = os.path.join(ROOT, "paper_2201_13191_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "oracle" not in txt.lower(), f
