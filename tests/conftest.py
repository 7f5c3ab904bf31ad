import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# BLAS threads of the oracle checks: at most half the cores.  OpenBLAS
# threads spin while they wait, and a 192 x 192 dense LU slows down from
# about a millisecond to more than half a second when they share busy
# cores.  The variables reach the ranks and pool workers the tests spawn;
# threadpoolctl (where installed) limits this process, whose BLAS may
# already be loaded.
_BLAS_THREADS = str(max(1, (os.cpu_count() or 2) // 2))
for _k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_k, _BLAS_THREADS)
try:
    from threadpoolctl import threadpool_limits

    threadpool_limits(int(_BLAS_THREADS))
except ImportError:  # pragma: no cover - not installed on every host
    pass


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built CUDA library")
    config.addinivalue_line("markers", "slow: oracle checks that take more than a few seconds")


def pytest_collection_modifyitems(config, items):
    # GPU tests cannot run without a device: skip them cleanly when absent.
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)
