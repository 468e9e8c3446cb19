import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session", autouse=True)
def _library_current():
    """Build libdmrg_gb300.so in-tree if it is missing or older than its sources (nvcc
    cross-compiles without a GPU), so every test runs the current library."""
    import glob
    import shutil
    from paper_2001_04890_gb300 import build as b
    srcs = glob.glob(os.path.join(ROOT, "paper_2001_04890_gb300", "csrc", "*")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    stale = not os.path.exists(b.OUT) or any(os.path.getmtime(f) > os.path.getmtime(b.OUT) for f in srcs)
    if stale and (os.path.exists(b.NVCC) or shutil.which("nvcc")):
        b.build()
    yield
