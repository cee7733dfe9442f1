"""Pins for the oracle's Krylov solvers (GMRES(m) and BiCGStab of Sec. 2.2 /
4.3; fault-convergence handling of Sec. 3.1 / 3.3.2; mixed-precision
refinement) against dense LU (numpy and textbook), finite termination, the
Arnoldi relation, closed-form solutions and degenerate cases."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")))
TOL = GOLD["solver_tolerance"]["value"]


def _rhs_ones(A):
    return oracle.spmv(A, np.ones(A["n"]))


def test_lu_matches_numpy():
    rng = np.random.default_rng(0)
    D = rng.standard_normal((30, 30)) + 10 * np.eye(30)
    b = rng.standard_normal(30)
    np.testing.assert_allclose(oracle.lu_solve(D, b), np.linalg.solve(D, b), rtol=1e-12, atol=1e-13)


def test_gmres_random200_vs_lu():
    A = gen.random200()
    D = gen.to_dense(A)
    b = _rhs_ones(A)
    x, info = oracle.gmres(A, b, m=30, tol=TOL)
    assert info["status"] == 0 and info["res_true"] <= TOL
    xs = np.linalg.solve(D, b)
    kappa = np.linalg.cond(D)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * TOL
    np.testing.assert_allclose(xs, np.ones(200), atol=1e-12)


def test_gmres_full_dimension_is_direct():
    # m = n, no restart: GMRES terminates with the exact solution (to rounding)
    rng = np.random.default_rng(4)
    A = gen.random_general(40, rng.integers(1, 8, size=40), seed=4, diag=0.5)
    b = rng.standard_normal(40)
    x, info = oracle.gmres(A, b, m=40, tol=1e-14, maxiter=40)
    xs = oracle.lu_solve(gen.to_dense(A), b)
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
    assert info["restarts"] <= 2


def test_arnoldi_relation_and_orthogonality():
    A = gen.poisson2d(12)
    D = gen.to_dense(A)
    m = 20
    v0 = np.random.default_rng(1).standard_normal(A["n"])
    k, V, H = oracle.arnoldi(A, v0, m)
    assert k == m
    Vm, Vm1 = V[:m].T, V[: m + 1].T
    R = D @ Vm - Vm1 @ H
    assert np.linalg.norm(R) <= 1e-12 * np.linalg.norm(D, 2)
    assert np.linalg.norm(np.eye(m) - Vm.T @ Vm) <= 1e-10
    # H is upper Hessenberg
    assert np.all(np.tril(H, -2) == 0)


def test_identity_converges_in_one_step():
    n = 50
    I = dict(n=n, nnz=n, rowptr=np.arange(n + 1, dtype=np.int32),
             col=np.arange(n, dtype=np.int32), val=np.ones(n), sym_upper=False)
    b = np.random.default_rng(0).standard_normal(n)
    x, info = oracle.gmres(I, b, m=10)
    assert info["iters"] == 1 and info["status"] == 0
    np.testing.assert_allclose(x, b, rtol=1e-15)
    x, info = oracle.bicgstab(I, b)
    assert info["iters"] == 1
    np.testing.assert_allclose(x, b, rtol=1e-14)


def test_gmres_poisson64_solution_is_ones():
    # config 1: 64x64 Poisson, b = A*ones, x0 = 0, GMRES(30) to 1e-8
    A = gen.poisson2d(64)
    b = _rhs_ones(A)
    x, info = oracle.gmres(A, b, m=30, tol=TOL)
    assert info["status"] == 0 and info["res_true"] <= TOL
    lam_min = 8 * np.sin(np.pi / (2 * 65)) ** 2  # smallest eigenvalue, closed form
    # ||x - 1|| <= ||A^-1|| ||r|| = ||r|| / lam_min
    assert np.linalg.norm(x - 1) <= TOL * np.linalg.norm(b) / lam_min * 1.01
    # implicit residual never increases within a cycle -> monotone restarts
    x2, inf2 = oracle.gmres(A, b, m=30, tol=TOL, hist_cap=100)
    h = inf2["hist"]
    assert np.all(np.diff(h) <= 1e-14)


def test_bicgstab_vs_lu_nonsymmetric():
    A = gen.convdiff3d(N=10, pe=10.0)
    D = gen.to_dense(A)
    b = _rhs_ones(A)
    x, info = oracle.bicgstab(A, b, tol=TOL)
    assert info["status"] == 0 and info["res_true"] <= TOL
    xs = np.linalg.solve(D, b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= np.linalg.cond(D) * TOL
    np.testing.assert_allclose(xs, 1.0, atol=1e-12)


def test_bicgstab_random200_and_powerlaw_small():
    for A in (gen.random200(), gen.powerlaw(n=3000, seed=9)):
        b = _rhs_ones(A)
        x, info = oracle.bicgstab(A, b, tol=TOL)
        assert info["status"] == 0 and info["res_true"] <= TOL
        r = b - gen.to_dense(A) @ x
        assert np.linalg.norm(r) / np.linalg.norm(b) <= TOL * 1.0001


def test_gmres_symmetric_upper_storage():
    U = gen.laplace3d(8, upper=True)
    F = gen.laplace3d(8)
    b = _rhs_ones(F)
    xu, iu = oracle.gmres(U, b, m=20, tol=TOL)
    xf, if_ = oracle.gmres(F, b, m=20, tol=TOL)
    assert iu["status"] == 0 and abs(iu["iters"] - if_["iters"]) <= 2
    np.testing.assert_allclose(xu, xf, atol=1e-7)


def test_maxiter_reports_noconv():
    A = gen.poisson2d(32)
    b = _rhs_ones(A)
    x, info = oracle.gmres(A, b, m=5, tol=1e-12, maxiter=20)
    assert info["status"] == -4 and info["iters"] == 20 and info["res_true"] > 1e-12
    x, info = oracle.bicgstab(A, b, tol=1e-14, maxiter=3)
    assert info["status"] == -4 and info["iters"] == 3


def test_breakdown_on_singular():
    n = 6
    Z = dict(n=n, nnz=0, rowptr=np.zeros(n + 1, np.int32), col=np.zeros(0, np.int32),
             val=np.zeros(0), sym_upper=False)
    b = np.ones(n)
    assert oracle.gmres(Z, b)[1]["status"] == -5
    assert oracle.bicgstab(Z, b)[1]["status"] == -5


def test_zero_rhs_gives_zero():
    A = gen.poisson2d(5)
    x, info = oracle.gmres(A, np.zeros(25), x0=np.ones(25))
    assert info["status"] == 0 and np.all(x == 0)
    x, info = oracle.bicgstab(A, np.zeros(25), x0=np.ones(25))
    assert info["status"] == 0 and np.all(x == 0)


def test_mixed_refinement_reaches_fp64_accuracy():
    for A in (gen.poisson2d(32), gen.random200(), gen.convdiff3d(N=12)):
        b = _rhs_ones(A)
        x, info = oracle.gmres_ir(A, b, m=30, tol=TOL, tol_in=1e-4)
        assert info["status"] == 0 and info["res_true"] <= TOL
        # re-evaluated independently of the oracle (numpy dense)
        r = b - gen.to_dense(A) @ x
        assert np.linalg.norm(r) / np.linalg.norm(b) <= TOL * 1.0001
        assert info["outer"] >= 2  # FP32 inner alone cannot reach 1e-8


def test_refinement_steps_contract_by_the_inner_tolerance():
    """The plain refinement loop, step by step: the inner FP32 solve leaves
    ||r/||r|| - A d|| <= tol_in (up to FP32 rounding), and x += ||r|| d makes
    that the next FP64 residual, so each step shrinks ||b - A x|| by at most
    about tol_in.  Residuals are recomputed densely here, independently of the
    oracle; a dropped ||r|| scale, a wrong sign in the update or a residual
    taken against float(A) breaks the bound."""
    A = gen.poisson2d(32)
    D = gen.to_dense(A)
    b = _rhs_ones(A)
    for tin in (0.3, 0.5):
        res = []
        for k in range(5):
            x, info = oracle.gmres_ir(A, b, m=30, tol=1e-14, tol_in=tin, max_outer=k)
            assert info["status"] == -4 and info["outer"] == k
            res.append(np.linalg.norm(b - D @ x) / np.linalg.norm(b))
            assert abs(res[-1] - info["res_true"]) <= 1e-12
        assert res[0] == 1.0
        for k in range(1, 5):
            assert res[k] <= tin * (1 + 1e-3) * res[k - 1] + 1e-6, (tin, k, res)


def test_stagnating_refinement_stays_plain():
    """One inner Arnoldi step per refinement step contracts slowly (the
    residual ratio climbs above 1/2); the plain loop keeps refining until
    max_outer and never hands over to another solver: one inner step per
    outer step, residual decreasing, ENOCONV at the cap."""
    A = gen.poisson2d(32)
    D = gen.to_dense(A)
    b = _rhs_ones(A)
    x, info = oracle.gmres_ir(A, b, m=30, tol=1e-8, tol_in=1e-4, maxit_in=1, max_outer=6)
    assert info["status"] == -4 and info["outer"] == 6 and info["inner_iters"] == 6
    prev = 1.0
    for k in range(1, 7):
        xk, _ = oracle.gmres_ir(A, b, m=30, tol=1e-8, tol_in=1e-4, maxit_in=1, max_outer=k)
        rk = np.linalg.norm(b - D @ xk) / np.linalg.norm(b)
        assert rk < prev
        prev = rk
    assert prev > 0.5 ** 6  # no FP64 solve took over
    np.testing.assert_array_equal(x, xk)


def test_inner_f32_solve_contracts_residual():
    A = gen.poisson2d(16)
    r = np.random.default_rng(0).standard_normal(A["n"]).astype(np.float32)
    r /= np.linalg.norm(r)
    d, it = oracle.gmres_f32_inner(A, r, m=20, tol_in=1e-4, maxit=500)
    res = np.linalg.norm(r.astype(np.float64) - gen.to_dense(A) @ d.astype(np.float64))
    assert res <= 2e-4 and it > 0
