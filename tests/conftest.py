import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")


def make_problem(n, b, a, seed=0, energy=0.3, eta=1e-3, gamma=0.5):
    """Seeded (A, B) of the synthetic recipe: A from the oracle's assembly of a
    Hermitian H, B anti-Hermitian."""
    from paper_2601_04904_gb300 import inputs
    from oracle import rgf

    h = inputs.hamiltonian(n, b, a, seed=inputs.BASE_SEED + seed)
    bb = inputs.lesser_rhs(n, b, a, seed=inputs.BASE_SEED + 7 + seed)
    return h, rgf.assemble_a(h, energy, eta, gamma), bb


@pytest.fixture
def rng():
    return np.random.default_rng(12345)
