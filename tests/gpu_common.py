"""Shared fixtures for the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

KAPPA, MU, EPS = 0.16, 0.1, 0.11


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_09584_gb300 import _build
    _build.build()
    import paper_1805_09584_gb300 as tm
    tm.lib()  # raises if the library is missing: no fallback
    return tm


def rel_err(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
