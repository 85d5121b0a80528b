import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (parity and device tests)")


@pytest.fixture(scope="session")
def barrel_geom():
    import lst_synth
    return lst_synth.geometry(True)


@pytest.fixture(scope="session")
def full_geom():
    import lst_synth
    return lst_synth.geometry(False)


@pytest.fixture(scope="session")
def ora_barrel(barrel_geom):
    import oracle
    return oracle.Geometry(barrel_geom.modules)


@pytest.fixture(scope="session")
def ora_full(full_geom):
    import oracle
    return oracle.Geometry(full_geom.modules)


@pytest.fixture(scope="session")
def tilted_geom():
    import lst_synth
    return lst_synth.geometry(False, True)


@pytest.fixture(scope="session")
def ora_tilted(tilted_geom):
    import oracle
    return oracle.Geometry(tilted_geom.modules)


@pytest.fixture(scope="session")
def ec2s_geom():
    import lst_synth
    return lst_synth.geometry(False, False, True)


@pytest.fixture(scope="session")
def ora_ec2s(ec2s_geom):
    import oracle
    return oracle.Geometry(ec2s_geom.modules)
