"""GPU thick-restart Lanczos (OpenATI_EIGENSOLVE, restarted Lanczos) against
the CPU oracle and the mathematics: with the same start vector the GPU's nev
largest eigenvalues equal the oracle's and the closed form / dense spectrum
within 1e-9 (relative to the largest), every Ritz residual meets the
tolerance, the eigenvectors satisfy ||A y - theta y|| <= 1e-6 |theta| on the
oracle's SpMV, and symmetric upper storage gives the same spectrum."""
import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen
from tests._gpu import lib_and_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


def _check(xb, dev, A, nev, m, tol, ref=None):
    import torch
    n = A["n"]
    v0 = np.random.default_rng(5).standard_normal(n)
    plan = xb.Plan.from_host(A, dev)
    ev, Y, info = plan.lanczos(nev=nev, m=m, tol=tol, v0=torch.tensor(v0, device=dev))
    assert info["status"] == 0, info
    eo, _, io = oracle.lanczos(A, nev=nev, m=m, tol=tol, v0=v0, vectors=False)
    assert io["status"] == 0
    scale = np.max(np.abs(eo))
    np.testing.assert_allclose(ev, eo, atol=1e-9 * scale)
    if ref is not None:
        np.testing.assert_allclose(ev, ref, atol=1e-9 * scale)
    assert np.all(info["resid"] <= tol * np.abs(ev) * (1 + 1e-12))
    Yh = Y.cpu().numpy()
    for i in range(nev):
        r = oracle.spmv(A, Yh[:, i]) - ev[i] * Yh[:, i]
        assert np.linalg.norm(r) <= 1e-6 * abs(ev[i]) + 1e-12, i
        assert abs(np.linalg.norm(Yh[:, i]) - 1.0) <= 1e-8
    return ev, info


def test_lanczos_1d_laplacian(env):
    xb, dev = env
    n = 200
    ref = 2 + 2 * np.cos(np.arange(1, 6) * np.pi / (n + 1))
    _check(xb, dev, gen.laplace1d(n), 5, 40, 1e-10, ref)


def test_lanczos_random_symmetric_full_and_upper(env):
    xb, dev = env
    U = gen.random_sym_upper(3000, seed=7)
    F = gen.full_from_upper(U)
    e1, _ = _check(xb, dev, F, 8, 40, 1e-10)
    e2, _ = _check(xb, dev, U, 8, 40, 1e-10)
    np.testing.assert_allclose(e1, e2, atol=1e-9 * np.max(np.abs(e1)))


def test_lanczos_limits_and_arguments(env):
    xb, dev = env
    import torch
    plan = xb.Plan.from_host(gen.laplace1d(100), dev)
    ev, _, info = plan.lanczos(nev=4, m=12, tol=1e-14, maxrestart=1, vectors=False)
    assert info["status"] == xb.XB_ENOCONV and info["restarts"] == 1 and len(ev) == 4
    for bad in (dict(nev=0, m=10), dict(nev=5, m=5), dict(nev=2, m=101)):
        with pytest.raises(xb.XbError):
            plan.lanczos(**bad)
    # a start vector spanning an invariant subspace (a unit vector of a diagonal
    # matrix: A v0 - (A v0, v0) v0 is exactly 0) breaks down
    n = 50
    D = dict(n=n, nnz=n, rowptr=np.arange(n + 1, dtype=np.int32),
             col=np.arange(n, dtype=np.int32), val=np.arange(1.0, n + 1), sym_upper=False)
    v = torch.zeros(n, dtype=torch.float64, device=dev)
    v[3] = 1.0
    _, _, info = xb.Plan.from_host(D, dev).lanczos(nev=2, m=10, v0=v, vectors=False)
    assert info["status"] == xb.XB_EBREAKDOWN


def test_lanczos_restart_rule(env):
    """The restart rule grows a too-short cycle on the GPU as in the oracle:
    same closed-form eigenvalues, m grown in steps of 5, far fewer SpMVs than
    the fixed cycle."""
    xb, dev = env
    import torch
    n = 400
    A = gen.laplace1d(n)
    v0 = torch.tensor(np.random.default_rng(1).standard_normal(n), device=dev)
    ref = 2 + 2 * np.cos(np.arange(1, 7) * np.pi / (n + 1))
    plan = xb.Plan.from_host(A, dev)
    ev0, _, fixed = plan.lanczos(nev=6, m=10, tol=1e-10, v0=v0, maxrestart=5000, vectors=False)
    ev1, _, grown = plan.lanczos(nev=6, m=10, tol=1e-10, v0=v0, maxrestart=5000, vectors=False,
                                 m_max=60)
    assert fixed["status"] == 0 and grown["status"] == 0
    assert fixed["m_final"] == 10 and 10 < grown["m_final"] <= 60
    assert (grown["m_final"] - 10) % 5 == 0
    assert grown["steps"] < fixed["steps"] / 4
    np.testing.assert_allclose(ev0, ref, atol=1e-10)
    np.testing.assert_allclose(ev1, ref, atol=1e-10)


def test_lanczos_policies(env):
    """The numerical computation policies on the Lanczos eigensolver (the
    paper's Table 4 counts Lanczos runs per policy): every policy but NONE
    checks the true residuals of a claimed convergence; each policy's
    settings (SpMV, cycle, memory) as defined, DGKS throughout; every policy
    gives the oracle's eigenvalues."""
    xb, dev = env
    import torch
    U = gen.random_sym_upper(3000, seed=7)
    F = gen.full_from_upper(U)
    nev, tol = 8, 1e-8
    v0h = np.random.default_rng(5).standard_normal(U["n"])
    eo, _, io = oracle.lanczos(F, nev=nev, m=40, tol=1e-12, v0=v0h, vectors=False)
    scale = np.max(np.abs(eo))
    plan = xb.Plan.from_host(U, dev)
    out = {}
    for pol in (xb.POLICY_NONE, xb.POLICY_TIME, xb.POLICY_ACCURACY, xb.POLICY_MEMORY,
                xb.POLICY_STABLE):
        ev, _, info = plan.lanczos(nev=nev, m=40, tol=tol, policy=pol, maxrestart=3000,
                                   v0=torch.tensor(v0h, device=dev), vectors=False)
        out[pol] = info
        assert info["status"] in (xb.XB_OK, xb.XB_EFAULT), (pol, info)
        np.testing.assert_allclose(ev, eo, atol=1e-6 * scale)
        if pol == xb.POLICY_NONE:
            assert info["true_resid"] == -1.0 and info["ortho_used"] == xb.ORTHO_DGKS
        elif info["status"] == xb.XB_OK:
            assert 0.0 <= info["true_resid"] <= tol, (pol, info)
        else:
            assert info["true_resid"] > tol and pol != xb.POLICY_ACCURACY, (pol, info)
    t, mem, stb = out[xb.POLICY_TIME], out[xb.POLICY_MEMORY], out[xb.POLICY_STABLE]
    # the thick restart needs an orthonormal basis: DGKS under every policy
    assert all(out[p]["ortho_used"] == xb.ORTHO_DGKS for p in out)
    assert 40 <= t["m_final"] <= 128 and mem["m_final"] == 20 and stb["m_final"] == 40
    assert out[xb.POLICY_ACCURACY]["status"] == xb.XB_OK
    assert mem["mem_bytes"] < t["mem_bytes"] / 3
