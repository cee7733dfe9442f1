"""Pins of the oracle's eigensolver path (OpenATI_EIGENSOLVE, restarted
Lanczos, Sec. 2.2 / 4.3):
  - the dense symmetric eigen-decomposition (Jacobi) equals numpy's eigh and
    satisfies A S = S diag(w), S^T S = I;
  - thick-restart Lanczos reproduces the closed-form eigenvalues of the 1D
    Laplacian, 2 + 2 cos(j pi / (n + 1)), and the brute-force dense spectrum
    of random sparse symmetric matrices (full and upper storage);
  - its eigenvectors satisfy A y = theta y;
  - a starting vector that spans an invariant subspace ends in a breakdown."""
import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen


@pytest.mark.parametrize("seed", [0, 1])
def test_jacobi_eigendecomposition(seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((30, 30))
    M = M + M.T
    w, S = oracle.sym_eig(M)
    np.testing.assert_allclose(w, np.sort(np.linalg.eigvalsh(M))[::-1], atol=1e-12)
    assert np.max(np.abs(M @ S - S * w)) <= 1e-12 * np.max(np.abs(w))
    np.testing.assert_allclose(S.T @ S, np.eye(30), atol=1e-13)
    # repeated eigenvalues
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    d = np.array([3.0, 3.0, 3.0, 1.0, 1.0, -2.0, -2.0, 5.0, 0.0, 0.0, 7.0, 7.0])
    w, S = oracle.sym_eig(Q @ np.diag(d) @ Q.T)
    np.testing.assert_allclose(w, np.sort(d)[::-1], atol=1e-12)


def test_lanczos_1d_laplacian_closed_form():
    n = 200
    A = gen.laplace1d(n)
    ev, Y, info = oracle.lanczos(A, nev=5, m=40, tol=1e-10,
                                 v0=np.random.default_rng(1).standard_normal(n))
    assert info["status"] == 0
    ref = 2 + 2 * np.cos(np.arange(1, 6) * np.pi / (n + 1))
    np.testing.assert_allclose(ev, ref, atol=1e-10)
    D = gen.to_dense(A)
    for i in range(5):
        assert np.linalg.norm(D @ Y[:, i] - ev[i] * Y[:, i]) <= 1e-8
        assert abs(np.linalg.norm(Y[:, i]) - 1.0) <= 1e-10


def test_lanczos_random_symmetric_brute_force():
    U = gen.random_sym_upper(300, seed=2)
    F = gen.full_from_upper(U)
    ref = np.sort(np.linalg.eigvalsh(gen.to_dense(F)))[::-1][:6]
    v0 = np.random.default_rng(2).standard_normal(300)
    for A in (F, U):
        ev, _, info = oracle.lanczos(A, nev=6, m=30, tol=1e-12, v0=v0, vectors=False)
        assert info["status"] == 0
        np.testing.assert_allclose(ev, ref, atol=1e-10)


def test_lanczos_invariant_start_breaks_down():
    n = 50
    A = dict(n=n, nnz=n, rowptr=np.arange(n + 1, dtype=np.int32), col=np.arange(n, dtype=np.int32),
             val=np.arange(1.0, n + 1), sym_upper=False)
    v0 = np.zeros(n)
    v0[3] = 1.0
    _, _, info = oracle.lanczos(A, nev=2, m=10, tol=1e-10, v0=v0)
    assert info["status"] == -5
    ev, _, info = oracle.lanczos(A, nev=3, m=20, tol=1e-12, v0=np.ones(n))
    assert info["status"] == 0
    np.testing.assert_allclose(ev, [50.0, 49.0, 48.0], atol=1e-9)


def test_lanczos_restart_rule_grows_m():
    """With m_max > m the restart rule (Eq. 1 over 5 samples of the worst
    relative Ritz residual, m += 5 on stagnation) grows a too-short cycle and
    converges in far fewer steps, to the same closed-form eigenvalues."""
    n = 400
    A = gen.laplace1d(n)
    v0 = np.random.default_rng(1).standard_normal(n)
    ref = 2 + 2 * np.cos(np.arange(1, 7) * np.pi / (n + 1))
    ev0, _, fixed = oracle.lanczos(A, nev=6, m=10, tol=1e-10, v0=v0, vectors=False,
                                   maxrestart=5000)
    ev1, _, grown = oracle.lanczos(A, nev=6, m=10, tol=1e-10, v0=v0, vectors=False,
                                   maxrestart=5000, m_max=60)
    assert fixed["status"] == 0 and grown["status"] == 0
    assert fixed["m_final"] == 10 and 10 < grown["m_final"] <= 60
    assert (grown["m_final"] - 10) % 5 == 0
    assert grown["steps"] < fixed["steps"] / 4
    np.testing.assert_allclose(ev0, ref, atol=1e-10)
    np.testing.assert_allclose(ev1, ref, atol=1e-10)
