import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

K0 = 2.0 * np.pi


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: oracle checks that take tens of seconds")


@pytest.fixture(scope="session")
def loop_model():
    """Oracle macromodel of the default loop element in its 0.45 x 0.45 x 0.1 box."""
    from paper_1712_02443_gb300.workloads import loop_element
    from oracle.macromodel import build_element
    et = loop_element()
    return build_element(et.scatterer.xyz, et.scatterer.tri, et.equiv.xyz, et.equiv.tri, K0)


@pytest.fixture(scope="session")
def c1_layout():
    from paper_1712_02443_gb300.workloads import loop_array
    return loop_array(2, 2)


@pytest.fixture(scope="session")
def meander_model():
    """Oracle macromodel of the reduced multiscale element (loop + meander, 6x6x1 box)."""
    from paper_1712_02443_gb300 import workloads as wl
    from oracle.macromodel import build_element
    et = wl.multiscale_element(meander=wl.MEANDER_REDUCED, box_div=wl.MEANDER_REDUCED_BOX)
    return build_element(et.scatterer.xyz, et.scatterer.tri, et.equiv.xyz, et.equiv.tri, K0)


@pytest.fixture(scope="session")
def c1_dense(loop_model, c1_layout):
    from oracle.macromodel import dense_exterior_operator
    return dense_exterior_operator([loop_model], c1_layout.type_of, c1_layout.offsets, K0)
