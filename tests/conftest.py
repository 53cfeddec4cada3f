import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def cfg():
    from paper_2206_11535_gb300 import gen
    return gen.load_config()


@pytest.fixture(scope="session")
def ocfg(cfg):
    from oracle import oracle as O
    return O.make_config(cfg)
