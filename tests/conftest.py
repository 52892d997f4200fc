import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def ico1_ops():
    from oracle.assemble import Operators
    from synth import meshes
    V, F = meshes.icosphere(1)
    return Operators(V, F, dt=0.4)


@pytest.fixture(scope="session")
def ico1_fm(ico1_ops):
    from oracle.formulation import Formulation
    return Formulation(ico1_ops)


@pytest.fixture(scope="session")
def torus_ops():
    from oracle.assemble import Operators
    from synth import meshes
    V, F = meshes.torus(1.0, 0.4, 12, 6)
    return Operators(V, F, dt=0.5)


@pytest.fixture(scope="session")
def torus_fm(torus_ops):
    from oracle.formulation import Formulation
    return Formulation(torus_ops)
