import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_sessionstart(session):
    # The compiled pieces are build outputs, not sources: build what is
    # missing or stale (nvcc cross-compiles for sm_103a without a GPU).
    import importlib.util

    import oracle
    import synth
    synth.build()
    oracle.build()
    # load the build script by path: importing the package itself needs the library
    spec = importlib.util.spec_from_file_location(
        "_dvl_build", os.path.join(ROOT, "paper_2306_11612_b300", "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
