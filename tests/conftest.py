import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libmc.so")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def data_dir(tmp_path_factory):
    d = os.environ.get("MC_DATA_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        return d
    return str(tmp_path_factory.mktemp("mcdata"))


@pytest.fixture(scope="session")
def table_path(data_dir):
    from mc_inputs import default_table_path

    return default_table_path("full", data_dir)


@pytest.fixture(scope="session")
def tables(table_path):
    from mc_inputs import read_tables

    return read_tables(table_path)


@pytest.fixture(scope="session")
def variant_table(data_dir):
    from mc_inputs import default_table_path

    return lambda v: default_table_path(v, data_dir)


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_13191_gb300 as mcx

    mcx.build()
    return mcx


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
