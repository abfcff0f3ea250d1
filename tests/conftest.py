import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")


@pytest.fixture(scope="session")
def tiny_pair():
    from synth import workload_pair
    return workload_pair("tiny_96x72", 0)


TINY_PARAMS = dict(gf_radius=2, disp_max=15.0, n_levels=1, cell=(5,), k_prop=(1,), k_rand=(7,), seed=11)
