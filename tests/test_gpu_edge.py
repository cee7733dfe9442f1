"""Degenerate shapes for the preconditioner, the eigensolver and the policy
path through the C ABI: a 1 x 1 system, a diagonal matrix (ILU(0) exact, one
preconditioned step), a Lanczos cycle as long as the matrix (the Krylov space
is the whole space, Ritz values exact), nev = 1, and n = 0 solves."""
import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen
from tests._gpu import lib_and_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


def _diag(d):
    n = len(d)
    return dict(n=n, nnz=n, rowptr=np.arange(n + 1, dtype=np.int32),
                col=np.arange(n, dtype=np.int32), val=np.asarray(d, np.float64), sym_upper=False)


def test_ilu_on_one_by_one_and_diagonal(env):
    xb, dev = env
    import torch
    for A in (_diag([4.0]), _diag(np.arange(1.0, 301.0))):
        plan = xb.Plan.from_host(A, dev)
        b = torch.tensor(oracle.spmv(A, np.ones(A["n"])), device=dev)
        for fn in (plan.gmres, plan.bicgstab):
            x = torch.zeros_like(b)
            info = fn(b, x, tol=1e-12, precond=xb.PRECOND_ILU0)
            assert info["status"] == 0 and info["iters"] <= 1, info
            np.testing.assert_allclose(x.cpu().numpy(), np.ones(A["n"]), rtol=1e-13)


def test_lanczos_full_length_cycle_is_exact(env):
    xb, dev = env
    import torch
    n = 24
    A = gen.laplace1d(n)
    ref = 2 + 2 * np.cos(np.arange(1, 4) * np.pi / (n + 1))
    plan = xb.Plan.from_host(A, dev)
    v0 = torch.tensor(np.random.default_rng(4).standard_normal(n), device=dev)
    ev, _, info = plan.lanczos(nev=3, m=n, tol=1e-10, v0=v0, vectors=False)
    # m = n: the first cycle spans the whole space unless the start vector
    # lies in an invariant subspace; then a breakdown is the right answer
    assert info["status"] in (0, xb.XB_EBREAKDOWN)
    if info["status"] == 0:
        np.testing.assert_allclose(ev, ref, atol=1e-10)
    ev1, _, info1 = plan.lanczos(nev=1, m=12, tol=1e-10, v0=v0, vectors=False)
    assert info1["status"] == 0 and abs(ev1[0] - ref[0]) <= 1e-10


def test_empty_system_under_policies(env):
    xb, dev = env
    import torch
    A = dict(n=0, nnz=0, rowptr=np.zeros(1, np.int32), col=np.zeros(0, np.int32),
             val=np.zeros(0), sym_upper=False)
    plan = xb.Plan.from_host(A, dev)
    b = torch.zeros(0, dtype=torch.float64, device=dev)
    for pol in (xb.POLICY_TIME, xb.POLICY_ACCURACY, xb.POLICY_MEMORY, xb.POLICY_STABLE):
        info = plan.gmres(b, torch.zeros_like(b), policy=pol)
        assert info["status"] == 0
