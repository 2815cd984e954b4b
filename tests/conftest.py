import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def pytest_sessionstart(session):
    # The CUDA library cross-compiles without a GPU; build it (if stale) so the
    # boundary tests can load it.  No fallback exists if the build fails.
    from paper_2604_15765_gb300 import build as _b
    _b.build()


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
