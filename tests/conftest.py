import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def tiny_problem():
    from paper_2604_11920_b300 import synth
    return synth.tiny()


@pytest.fixture(scope="session")
def tiny_system(tiny_problem):
    """Oracle-side G, G^T and d for the 16x16x8 checkerboard system."""
    import oracle
    p = tiny_problem
    G = oracle.build_G_problem(p)
    GT = oracle.transpose(G)
    d = oracle.rhs_for(p, G)
    return p, G, GT, d
