import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU oracle runs")


@pytest.fixture(scope="session")
def models():
    """Oracle models of the standard workloads, built once per session."""
    from oracle import atom
    from paper_2010_08482_gb300 import workloads as w
    cache = {}

    def get(name):
        if name not in cache:
            cache[name] = atom.Model(w.WORKLOADS[name][0]())
        return cache[name]
    return get
