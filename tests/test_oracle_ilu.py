"""Pins of the oracle's ILU(0) preconditioner (the paper's solver runs use
ILU(0), Sec. 4.3) and of its right-preconditioned GMRES / BiCGStab:
  - the defining property of ILU(0): (L U)_ij = a_ij on A's pattern;
  - a tridiagonal matrix has no fill, so ILU(0) is its exact LU: L U = A
    everywhere and the preconditioned solvers finish in one iteration;
  - the triangular solves equal dense forward / backward substitution;
  - a zero pivot is reported as a breakdown;
  - preconditioning keeps the true residual of A x = b and cuts iterations."""
import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen


def _dense_lu(A, lu):
    n = A["n"]
    L = np.eye(n)
    U = np.zeros((n, n))
    rp, ci = A["rowptr"], A["col"]
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            j = ci[p]
            if j < i:
                L[i, j] = lu[p]
            else:
                U[i, j] = lu[p]
    return L, U


@pytest.mark.parametrize("make", [gen.random200, lambda: gen.powerlaw(n=400, seed=9),
                                  lambda: gen.convdiff3d(N=5), lambda: gen.poisson2d(9)])
def test_ilu0_matches_A_on_its_pattern(make):
    A = make()
    lu, st = oracle.ilu0(A)
    assert st == 0
    L, U = _dense_lu(A, lu)
    P = L @ U
    D = gen.to_dense(A)
    mask = np.zeros_like(D, dtype=bool)
    rp, ci = A["rowptr"], A["col"]
    for i in range(A["n"]):
        mask[i, ci[rp[i]:rp[i + 1]]] = True
    scale = np.max(np.abs(D))
    assert np.max(np.abs((P - D)[mask])) <= 1e-12 * scale
    # and it is not the exact LU where the pattern has fill (2D stencil)
    if A.get("kind") == "poisson2d":
        assert np.max(np.abs((P - D)[~mask])) > 1e-3


def test_tridiagonal_ilu0_is_exact_lu():
    A = gen.laplace1d(50)
    lu, st = oracle.ilu0(A)
    L, U = _dense_lu(A, lu)
    np.testing.assert_allclose(L @ U, gen.to_dense(A), atol=1e-13)
    b = oracle.spmv(A, np.ones(50))
    x, g = oracle.gmres(A, b, m=10, tol=1e-10, ilu=True)
    assert g["status"] == 0 and g["iters"] == 1
    x, bi = oracle.bicgstab(A, b, tol=1e-10, ilu=True)
    assert bi["status"] == 0 and bi["iters"] == 1
    np.testing.assert_allclose(x, np.ones(50), rtol=1e-10)


def test_ilu0_solve_is_forward_then_backward_substitution():
    A = gen.powerlaw(n=300, seed=4)
    lu, _ = oracle.ilu0(A)
    L, U = _dense_lu(A, lu)
    r = np.random.default_rng(2).standard_normal(300)
    z = oracle.ilu0_solve(A, lu, r)
    zr = np.linalg.solve(U, np.linalg.solve(L, r))
    np.testing.assert_allclose(z, zr, rtol=1e-10, atol=1e-12 * np.max(np.abs(zr)))


def test_ilu0_zero_pivot_is_a_breakdown():
    A = dict(n=2, nnz=3, rowptr=np.array([0, 1, 3], np.int32), col=np.array([1, 0, 1], np.int32),
             val=np.array([1.0, 1.0, 2.0]), sym_upper=False)
    _, st = oracle.ilu0(A)
    assert st == -5


@pytest.mark.parametrize("make", [lambda: gen.poisson2d(64), lambda: gen.convdiff3d(N=16),
                                  lambda: gen.powerlaw(n=3000, seed=9)])
def test_preconditioned_solvers_converge_faster_on_the_true_residual(make):
    A = make()
    b = oracle.spmv(A, np.ones(A["n"]))
    for solve in (lambda **k: oracle.gmres(A, b, m=30, tol=1e-8, maxiter=200000, **k),
                  lambda **k: oracle.bicgstab(A, b, tol=1e-8, maxiter=200000, **k)):
        x0, plain = solve()
        x1, prec = solve(ilu=True)
        assert prec["status"] == 0
        rel = np.linalg.norm(b - oracle.spmv(A, x1)) / np.linalg.norm(b)
        assert rel <= 1e-8 and abs(rel - prec["res_true"]) <= 1e-3 * rel
        assert prec["iters"] <= plain["iters"] / 2
