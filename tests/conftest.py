import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU validation")


def oracle_config_from(wl, **over):
    from oracle import config_from
    return config_from(wl, **over)


def make_oracle(wl, init=True, **over):
    """Oracle for a workload (optionally overriding configuration fields), initial state set."""
    from oracle import from_workload
    return from_workload(wl, init, **over)


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    return oracle.build_oracle()
