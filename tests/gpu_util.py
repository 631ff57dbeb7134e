"""Helpers shared by the GPU tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def cuda_or_skip():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_04100_gb300 import build
    build.build()
    return torch.device("cuda:0")


def row_relerr(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """max_s |a - b| / max_s |b| per row."""
    return np.abs(a - b).max(1) / np.maximum(np.abs(b).max(1), 1e-300)
