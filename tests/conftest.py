import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libsmg library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


LATE_MODULES = ("test_gpu_solve_coarse_forms.py", "test_gpu_boundary.py")
LAST_MODULES = ("test_zz_no_alloc.py",)


def pytest_collection_modifyitems(config, items):
    """The coarse-level form and boundary-condition tests (the newest GPU
    paths) run after the rest of the suite, so that under -x a failure there
    cannot hide the results of the established tests; the no-allocation entry
    point's test runs after everything else."""
    def module(it):
        path = getattr(it, "path", None)
        return path.name if path is not None else os.path.basename(str(it.fspath))

    rank = {m: 1 for m in LATE_MODULES}
    rank.update({m: 2 for m in LAST_MODULES})
    items[:] = sorted(items, key=lambda it: rank.get(module(it), 0))   # stable: file order within a rank


@pytest.fixture(scope="session")
def lib():
    """The C-ABI library, loaded once (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_12559_gb300 import binding
    return binding.load()
