import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    return oracle.load()


def rel_err_instances(batch, C_test, C_ref):
    """Per-instance ||C - C_ref||_F / (||A||_F ||B||_F) over a packed batch.

    The beta*C term is left out of the denominator (the tolerance is stated
    against the product A B)."""
    out = np.empty(batch.count)
    for i in range(batch.count):
        m, n, k, lda, ldb, ldc, ao, bo, co = (int(x) for x in batch.table[i])
        a = batch.instance(i, "A")
        b = batch.instance(i, "B")
        ct = C_test[co:co + ldc * n].reshape((n, ldc)).T[:m, :]
        cr = C_ref[co:co + ldc * n].reshape((n, ldc)).T[:m, :]
        den = np.linalg.norm(a) * np.linalg.norm(b)
        num = np.linalg.norm(ct - cr)
        out[i] = num / den if den > 0 else num
    return out


@pytest.fixture(scope="session")
def bglib():
    """The built C-ABI library (compiled here with nvcc when missing or stale)."""
    from paper_2203_09353_gb300 import build
    build.build()
    import paper_2203_09353_gb300 as bg
    return bg.load_library()


@pytest.fixture(scope="session")
def gpu(bglib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return torch.device("cuda:0")
