import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the library's kernels)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def tiny_case():
    from oracle import basis as B, potential as P
    from paper_2210_12252_gb300 import inputs
    w = inputs.tiny()
    g = w.geom
    b = B.Basis(g.R, g.tau, g.alpha, g.Nr, g.Nth1, g.Nth2, g.ncyc, g.oversample)
    V = P.gaussian_wells(b, w.atoms)
    return w, b, V
