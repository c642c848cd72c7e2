import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def h2_mech():
    from paper_1607_03884_gb300 import synth
    return synth.make_mechanism("h2")


@pytest.fixture(scope="session")
def ch4_mech():
    from paper_1607_03884_gb300 import synth
    return synth.make_mechanism("ch4")


def load_closed_forms():
    """tests/golden/radau_iia_closed_forms.txt as a dict of floats / lists."""
    s6 = np.sqrt(6.0)
    out = {}
    path = os.path.join(ROOT, "tests", "golden", "radau_iia_closed_forms.txt")
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split("=", 1)
        out[k.strip()] = eval(v, {"s6": s6})
    return out
