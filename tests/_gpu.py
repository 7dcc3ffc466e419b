"""Helpers for the GPU tests: skip cleanly without a GPU, fail loudly without the library."""
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA GPU")
    from paper_1705_02028_gb300 import binding
    binding.load()  # raises if the CUDA library cannot be built or loaded
    return torch


def rel_max_err(a, b):
    """Per-component max|a-b| / max(max|b_k|, max|b_E|) (max norm, relative)."""
    import numpy as np
    scale = np.maximum(np.abs(b).max(axis=1), np.abs(b[3]).max())
    return float((np.abs(a - b).max(axis=1) / scale).max())
