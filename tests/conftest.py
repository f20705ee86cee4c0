import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libpbdr.so")
    config.addinivalue_line("markers", "slow: longer CPU-only checks")


@pytest.fixture(scope="session")
def orc():
    """The FP64 oracle (built in place on first use)."""
    from oracle import oracle as O
    O.build()
    return O


@pytest.fixture(scope="session")
def pbdr_lib():
    """The sm_103a library (built in place); loading fails loudly if missing."""
    from paper_2603_14634_gb300 import build as B
    B.build()
    from paper_2603_14634_gb300 import binding
    return binding


@pytest.fixture(params=["resident", "streaming"])
def ctx(pbdr_lib, request):
    """A context running the scene-resident kernel (default) or the streaming
    kernels for every scene."""
    c = pbdr_lib.Context(0)
    c.set_path(streaming=request.param == "streaming")
    c.path_name = request.param
    yield c
    c.close()
