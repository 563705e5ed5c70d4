import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle_polys():
    """Minimal polynomials and squaring chains of the three variants (oracle side)."""
    import oracle
    oracle.prepare_all()
    return oracle


@pytest.fixture(scope="session")
def stdmt():
    """Path of a tiny program printing std::mt19937 / std::mt19937_64 outputs."""
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler for the libstdc++ pin")
    d = tempfile.mkdtemp(prefix="stdmt")
    exe = os.path.join(d, "stdmt")
    subprocess.check_call([cxx, "-O1", "-std=c++17", "-o", exe,
                           os.path.join(ROOT, "tests", "helpers", "stdmt.cpp")])
    yield exe
    shutil.rmtree(d, ignore_errors=True)


def run_stdmt(exe, bits, seed, skip, count):
    out = subprocess.check_output([exe, str(bits), str(seed), str(skip), str(count)], text=True)
    return [int(x) for x in out.split()]
