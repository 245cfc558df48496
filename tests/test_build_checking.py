"""The checking build (-DLEMC_DEBUG) of the library compiles.

Its range checks rewrite data-dependent indices in device code, so a
construct that only the release build accepts (an index declared const, for
instance) is caught here, on the CPU; the GPU tests run that build.
"""
import importlib.util
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checking_build_compiles(tmp_path):
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("needs nvcc")
    spec = importlib.util.spec_from_file_location("le_mc_build_check",
                                                  os.path.join(ROOT, "paper_1206_3316_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    # into a scratch directory: the in-tree libraries are left as they are
    mod.OBJ = str(tmp_path / "obj")
    mod.LIB_DEBUG = str(tmp_path / "libLeMC_debug.so")
    lib = mod.build(force=True, debug=True)
    assert os.path.getsize(lib) > 0
