"""Shared test setup: the ``gpu`` marker, import paths and oracle fixtures."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU run (still part of the default suite)")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as O
    O.lib()
    return O


@pytest.fixture(scope="session")
def analytic():
    from oracle import analytic as A
    return A


@pytest.fixture(scope="session")
def built_library():
    """Builds libLeMC.so in tree (nvcc) and returns the imported package."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("le_mc_build", os.path.join(ROOT, "paper_1206_3316_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_1206_3316_gb300 as pkg
    return pkg
