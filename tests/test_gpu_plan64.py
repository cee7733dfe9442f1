"""Plans over 64-bit row offsets (xb_plan_create64) against the oracle.

Below 2^31 - 64 non-zeros the plan narrows rowptr and is an ordinary plan.
Beyond it the plan runs every SpMV row block by row block; a 2^31-entry
matrix is not needed to test that path: XB_PLAN_SPLIT_NNZ lowers the block
limit so that a small matrix is split into several blocks."""
import os

import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen
from tests._gpu import assert_rows_close, lib_and_device, row_bound

pytestmark = pytest.mark.gpu


def _plan64(xb, dev, A):
    import torch
    return xb.Plan(torch.as_tensor(np.asarray(A["rowptr"], np.int64), device=dev),
                   torch.as_tensor(A["col"], dtype=torch.int32, device=dev),
                   torch.as_tensor(A["val"], dtype=torch.float64, device=dev))


def _check_spmv(xb, dev, plan, A, shapes):
    import torch
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, A["n"])
    y0 = rng.uniform(-1, 1, A["n"])
    xt = torch.tensor(x, device=dev)
    for alpha, beta in [(1.0, 0.0), (-1.5, 0.5)]:
        want = oracle.spmv(A, x, alpha, beta, y0)
        bound = row_bound(A, x, alpha, beta, y0)
        for v, b, i in shapes:
            y = torch.tensor(y0, device=dev)
            plan.spmv(xt, y, alpha=alpha, beta=beta, variant=v, block=b, ipt=i)
            assert_rows_close(y.cpu().numpy(), want, bound, what=f"v{v} b{b} i{i} a{alpha}")
        y = torch.tensor(y0, device=dev)
        plan.spmv_crs(xt, y, alpha=alpha, beta=beta)
        assert_rows_close(y.cpu().numpy(), want, bound, what="spmv_crs")


def _solves(xb, dev, plan, A):
    import torch
    b_h = oracle.spmv(A, np.ones(A["n"]))
    b = torch.tensor(b_h, device=dev)
    _, io = oracle.gmres(A, b_h, m=30, tol=1e-8)
    for kw in (dict(), dict(precision=xb.PREC_MIXED, tol_inner=1e-4)):
        x = torch.zeros_like(b)
        info = plan.gmres(b, x, m=30, tol=1e-8, small_n=0, **kw)
        rel = np.linalg.norm(b_h - oracle.spmv(A, x.cpu().numpy())) / np.linalg.norm(b_h)
        assert info["status"] == 0 and rel <= 1e-8, (kw, info)
        if not kw:
            assert abs(info["iters"] - io["iters"]) <= max(3, 0.05 * io["iters"])
    x = torch.zeros_like(b)
    info = plan.bicgstab(b, x, tol=1e-8)
    rel = np.linalg.norm(b_h - oracle.spmv(A, x.cpu().numpy())) / np.linalg.norm(b_h)
    assert info["status"] == 0 and rel <= 1e-8, info


def _powerlaw_dominant(n=20000, seed=6):
    """Lognormal row lengths (as the power-law recipe) with a dominant
    diagonal, so that the solves converge in a few dozen steps."""
    L = np.clip(np.rint(np.random.default_rng(seed).lognormal(1.36, 1.5, n)), 1, 2000).astype(np.int64)
    return gen.random_general(n, L, seed=seed, diag=1.0)


SHAPES = [(0, 256, 1), (1, 128, 8), (1, 256, 4), (2, 128, 8), (2, 256, 16), (5, 128, 32)]


def test_plan64_below_the_limit_is_an_ordinary_plan():
    xb, dev = lib_and_device()
    A = _powerlaw_dominant()
    plan = _plan64(xb, dev, A)
    _check_spmv(xb, dev, plan, A, SHAPES)
    _solves(xb, dev, plan, A)
    plan.ilu0_setup()  # everything an int32 plan supports


@pytest.mark.parametrize("make,extra", [
    (_powerlaw_dominant, []),
    (lambda: gen.block_stencil3d(14, 3), [(8, 128, 3), (8, 256, 2)]),
])
def test_plan64_split_into_row_blocks(make, extra):
    xb, dev = lib_and_device()
    import torch
    A = make()
    os.environ["XB_PLAN_SPLIT_NNZ"] = str(A["nnz"] // 5)
    try:
        plan = _plan64(xb, dev, A)
    finally:
        del os.environ["XB_PLAN_SPLIT_NNZ"]
    # SELL is left out: its padding rule (3 nnz + 32 per slice) rejects the
    # small last block the greedy split leaves, and a variant rejected on one
    # block is rejected for the plan
    _check_spmv(xb, dev, plan, A, [t for t in SHAPES if t[0] != 5] + extra)
    _solves(xb, dev, plan, A)
    ch = plan.tune()
    assert ch["variant"] in (xb.VAR_ROW, xb.VAR_NNZ, xb.VAR_SEGSCAN, xb.VAR_SELL, xb.VAR_BCSR)
    _check_spmv(xb, dev, plan, A, [(-1, 0, 0)])  # the tuned choice on every block
    b = torch.ones(A["n"], dtype=torch.float64, device=dev)
    with pytest.raises(xb.XbError):
        plan.gmres(b, torch.zeros_like(b), precond=xb.PRECOND_ILU0)
    with pytest.raises(xb.XbError):
        plan.ilu0_setup()


def test_plan64_rejects_bad_input():
    xb, dev = lib_and_device()
    import torch
    A = gen.poisson2d(8)
    rp = np.asarray(A["rowptr"], np.int64).copy()
    rp[-1] += 1  # rowptr[n] != nnz
    with pytest.raises(xb.XbError):
        xb.Plan(torch.as_tensor(rp, device=dev), torch.as_tensor(A["col"], device=dev),
                torch.as_tensor(A["val"], device=dev))
