"""The allocation-free SpMV entry point (spmv_segscan_noalloc), called through
the C ABI, against the oracle and the plan-based spmv_segscan on the same
inputs.

It serves callers that cannot allocate device memory (their memory belongs
to another allocator, or allocation is not allowed where they call), so it
takes the CRS arrays directly and keeps its scratch in an array compiled into
the library.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen
from tests._gpu import assert_rows_close, lib_and_device, row_bound

pytestmark = pytest.mark.gpu


def _fn(xb):
    f = xb.lib().spmv_segscan_noalloc
    f.restype = C.c_int32
    f.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                  C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]
    return f


def _call(xb, f, rp, ci, va, alpha, x, beta, y):
    import torch
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: C.c_void_p(t.data_ptr()) if t.numel() else C.c_void_p(0)
    return f(rp.numel() - 1, ci.numel(), p(rp), p(ci), p(va), alpha, p(x), beta, p(y), s)


def _adversarial():
    rng = np.random.default_rng(42)
    n = 6000
    L = rng.choice([0, 0, 1, 2, 5, 31, 32, 33, 63, 64, 65, 127, 129], size=n)
    L[3000] = 5999
    L[-40:] = 0
    return gen.random_general(n, L, seed=7)


@pytest.mark.parametrize("make", [lambda: gen.powerlaw(n=300_000, seed=3), _adversarial,
                                  lambda: gen.poisson2d(64)])
def test_noalloc_matches_oracle_and_plan_segscan_twice(make):
    """Two calls in a row (they share the scratch array) each match the
    oracle row by row at 1e-12 * (|alpha| sum_j |a_ij||x_j| + |beta||y_i|), and
    the plan-based spmv_segscan on the same inputs meets the same bound."""
    xb, dev = lib_and_device()
    import torch
    A = make()
    n = A["n"]
    f = _fn(xb)
    rp = torch.as_tensor(A["rowptr"], device=dev)
    ci = torch.as_tensor(A["col"], device=dev)
    va = torch.as_tensor(A["val"], device=dev)
    plan = xb.Plan(rp, ci, va)
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, n)
    y0 = rng.uniform(-1, 1, n)
    xt = torch.tensor(x, device=dev)
    for alpha, beta in [(1.0, 0.0), (-2.0, 0.5)]:
        want = oracle.spmv(A, x, alpha, beta, y0)
        bound = row_bound(A, x, alpha, beta, y0)
        ref = torch.tensor(y0, device=dev)
        plan.spmv_segscan(xt, ref, alpha=alpha, beta=beta)
        assert_rows_close(ref.cpu().numpy(), want, bound, what="plan segscan")
        for call in range(2):
            y = torch.tensor(y0, device=dev)
            assert _call(xb, f, rp, ci, va, alpha, xt, beta, y) == 0, xb.last_error()
            assert_rows_close(y.cpu().numpy(), want, bound, what=f"noalloc call {call}")


def test_noalloc_matrix_without_entries():
    """n > 0 rows and nnz = 0: only the empty-row pass runs; y = 0 when
    beta = 0 and y = beta * y otherwise, exactly."""
    xb, dev = lib_and_device()
    import torch
    f = _fn(xb)
    n = 1000
    rp = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    ci = torch.zeros(0, dtype=torch.int32, device=dev)
    va = torch.zeros(0, dtype=torch.float64, device=dev)
    y0 = np.random.default_rng(3).uniform(-1, 1, n)
    xt = torch.ones(n, dtype=torch.float64, device=dev)
    for alpha, beta in [(1.0, 0.0), (-2.0, 0.5)]:
        y = torch.tensor(y0, device=dev)
        assert _call(xb, f, rp, ci, va, alpha, xt, beta, y) == 0, xb.last_error()
        np.testing.assert_array_equal(y.cpu().numpy(), beta * y0 if beta else np.zeros(n))


def test_noalloc_rejects_overlapping_x_and_y():
    xb, dev = lib_and_device()
    import torch
    f = _fn(xb)
    A = gen.poisson2d(8)
    rp = torch.as_tensor(A["rowptr"], device=dev)
    ci = torch.as_tensor(A["col"], device=dev)
    va = torch.as_tensor(A["val"], device=dev)
    buf = torch.zeros(2 * A["n"], dtype=torch.float64, device=dev)
    rc = _call(xb, f, rp, ci, va, 1.0, buf[: A["n"]], 0.0, buf[A["n"] // 2: A["n"] // 2 + A["n"]])
    assert rc == xb.XB_EINVAL and "overlap" in xb.last_error()


def test_noalloc_rejects_oversize_without_launching():
    xb, dev = lib_and_device()
    import torch
    f = _fn(xb)
    rp = torch.zeros(2, dtype=torch.int32, device=dev)
    one = torch.zeros(1, dtype=torch.float64, device=dev)
    ci = torch.zeros(1, dtype=torch.int32, device=dev)
    y = torch.zeros(1, dtype=torch.float64, device=dev)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # nnz far beyond the built-in scratch: rejected on the host before any launch
    rc = f(1, 2_000_000_000, C.c_void_p(rp.data_ptr()), C.c_void_p(ci.data_ptr()),
           C.c_void_p(one.data_ptr()), 1.0, C.c_void_p(one.data_ptr()), 0.0,
           C.c_void_p(y.data_ptr()), s)
    assert rc == xb.XB_EINVAL
    assert "scratch" in xb.last_error()
