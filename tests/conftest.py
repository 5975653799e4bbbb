import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libbsm")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def bsm_lib():
    from paper_1705_10218_gb300 import build as _b

    _b.build()
    import paper_1705_10218_gb300 as P

    P.lib()
    return P


@pytest.fixture(scope="session")
def gpu_ctx(bsm_lib):
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for tests marked gpu")
    ctx = bsm_lib.Context(0)
    yield ctx
    ctx.close()
