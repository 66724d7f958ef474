import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def semlib():
    """libsem initialised on cuda:0 (GPU tests only); torch's current stream is
    set to libsem's stream so tensor set-up and kernels are ordered."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2606_12650_gb300 import build, sem
    build.build()
    sem.init(["--device=0"])
    torch.cuda.set_stream(sem.stream())
    yield sem
    torch.cuda.synchronize()
    sem.finalize()
