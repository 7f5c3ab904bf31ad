"""Helpers for the GPU parity tests: build/load the CUDA library and move
numpy fields to and from the device."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def lib_api():
    from paper_1112_1243_gb300 import build
    build.build()
    from paper_1112_1243_gb300 import api
    return api


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_err(a, b):
    return float(np.linalg.norm((a - b).reshape(-1)) / max(np.linalg.norm(b.reshape(-1)), 1e-300))
