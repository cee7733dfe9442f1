"""Shared helpers for the GPU parity tests (not a test module)."""
import numpy as np
import pytest

import oracle


def lib_and_device():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device (run with -m 'not gpu' on CPU-only hosts)")
    import paper_2405_01599_gb300 as xb
    xb.build()
    xb.lib()
    return xb, torch.device("cuda:0")


def row_bound(A, x, alpha=1.0, beta=0.0, y0=None):
    """sum_j |a_ij||x_j| * |alpha| (+ |beta||y0_i|): the per-row scale of the
    1e-12 SpMV tolerance, from the oracle on |A| and |x|."""
    Aabs = dict(A)
    Aabs["val"] = np.abs(A["val"])
    s = abs(alpha) * oracle.spmv(Aabs, np.abs(x))
    if beta != 0.0 and y0 is not None:
        s = s + abs(beta) * np.abs(y0)
    return s


def assert_rows_close(y, yref, bound, rel=1e-12, what=""):
    err = np.abs(y - yref)
    bad = err > rel * bound
    # rows whose scale is 0 must match exactly
    if np.any(bad):
        i = int(np.flatnonzero(bad)[0])
        raise AssertionError(f"{what}: {bad.sum()} rows exceed tolerance; row {i}: "
                             f"gpu={y[i]!r} oracle={yref[i]!r} bound={rel * bound[i]:.3e}")


def row_subset(A, rows):
    """CRS of the given rows of A (index bookkeeping only; columns unchanged)."""
    rp = A["rowptr"].astype(np.int64)
    lens = rp[rows + 1] - rp[rows]
    idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows]) if len(rows) else np.zeros(0, np.int64)
    sub_rp = np.zeros(len(rows) + 1, np.int64)
    np.cumsum(lens, out=sub_rp[1:])
    return dict(n=len(rows), nnz=int(sub_rp[-1]), rowptr=sub_rp.astype(np.int32),
                col=A["col"][idx], val=A["val"][idx], sym_upper=False)


def sampled_rows_oracle(A, x, rows):
    """Oracle y_i for the sampled rows only: the oracle's SpMV on the row subset
    (the subset's column indices still address the full x)."""
    S = row_subset(A, rows)
    y = np.zeros(len(rows))
    import ctypes
    L = oracle.lib()
    n_sub = S["n"]
    L.orc_spmv(n_sub, S["rowptr"], S["col"].astype(np.int32), S["val"].astype(np.float64),
               1.0, np.ascontiguousarray(x, np.float64), 0.0, y)
    return y
