import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300); run with -m gpu")
    config.addinivalue_line("markers", "slow: long-running")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def lib_path():
    from paper_2005_01182_gb300 import build
    return build.build()


@pytest.fixture(scope="session")
def ctx(lib_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_01182_gb300 import otassign as ot
    c = ot.Context()
    yield c
    c.close()
