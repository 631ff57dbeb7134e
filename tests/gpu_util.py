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


def rows_to_sell(a: np.ndarray, w: int) -> np.ndarray:
    """[n][w] rows -> sliced-ELL storage (slice height 32, slot-major inside a slice), zero padded."""
    from paper_1603_04100_gb300 import api
    n = a.shape[0]
    npad = api.n_padded(n)
    full = np.zeros((npad, w), dtype=a.dtype)
    full[:n] = a
    return np.ascontiguousarray(full.reshape(npad // api.SLICE, api.SLICE, w).transpose(0, 2, 1)).ravel()


def operator_from_rows(nbr: np.ndarray, val: np.ndarray, prec: int, device):
    """An operator uploaded from host rows in their own order (the tests feed the
    oracle's own rows to the GPU hierarchy): nbr [n][k] int32, val [n][k+1] FP64
    with slot 0 the row itself; the mixed format stores each weight as its FP32
    rounding hi plus the FP32 rounding of the rest."""
    from paper_1603_04100_gb300 import api
    n, k = nbr.shape
    col, v, lo = api.ell_alloc(n, k, prec, device)
    c = rows_to_sell(np.ascontiguousarray(nbr, dtype=np.int32), k)
    col[: c.size].copy_(torch.from_numpy(c))
    if prec == api.FP64:
        vv = rows_to_sell(np.asarray(val, dtype=np.float64), k + 1)
        v[: vv.size].copy_(torch.from_numpy(vv))
    else:
        hi = np.asarray(val, dtype=np.float64).astype(np.float32)
        rest = (np.asarray(val, dtype=np.float64) - hi.astype(np.float64)).astype(np.float32)
        h = rows_to_sell(hi, k + 1)
        r = rows_to_sell(rest, k + 1)
        v[: h.size].copy_(torch.from_numpy(h))
        lo[: r.size].copy_(torch.from_numpy(r))
    return api.Operator(n, k, prec, col, v, lo, None)
