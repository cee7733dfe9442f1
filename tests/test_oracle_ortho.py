"""Pins of the oracle's orthogonalisations (Sec. 3.2.2: CGS, DGKS, MGS, BCGS
with block length 4) and of the accuracy policy that chooses among them
(Sec. 3.3.2), against what the mathematics fixes:
  - Gram-Schmidt QR reconstructs X, and the loss of orthogonality follows the
    textbook orders: DGKS (CGS twice) ~ eps, MGS ~ eps*kappa, CGS ~ eps*kappa^2;
  - BCGS with block length 1 is MGS and with one block is CGS, bit for bit;
  - k Arnoldi steps span the Krylov space: V and H equal numpy's QR of the
    Krylov matrix [v0, A v0, ..., A^k v0] (R's diagonal made positive) and
    Q^T A Q;
  - GMRES with every orthogonalisation solves the 64x64 Poisson problem;
  - the policy picks MGS for tol <= 1e-10, BCGS otherwise, DGKS after a fault
    convergence."""
import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen

ORTHOS = {"mgs": oracle.MGS, "cgs": oracle.CGS, "dgks": oracle.DGKS, "bcgs": oracle.BCGS}


def _ill_conditioned(n, k, kappa, seed=0):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, k)))
    W, _ = np.linalg.qr(rng.standard_normal((k, k)))
    return U @ np.diag(np.logspace(0, -np.log10(kappa), k)) @ W.T


def _orth_err(Q):
    return np.max(np.abs(Q.T @ Q - np.eye(Q.shape[1])))


def test_gram_schmidt_qr_reconstructs_and_loses_orthogonality_as_theory_says():
    X = _ill_conditioned(300, 20, 1e6)
    err = {}
    for name, o in ORTHOS.items():
        Q, R, done = oracle.gs_qr(X, o)
        assert done == 20
        assert np.allclose(np.tril(R, -1), 0.0)
        assert np.max(np.abs(Q @ R - X)) <= 1e-14 * np.max(np.abs(X)), name
        err[name] = _orth_err(Q)
    eps = np.finfo(float).eps
    assert err["dgks"] <= 100 * eps                      # ~ eps
    assert 100 * eps < err["mgs"] <= 1e-8                # ~ eps * kappa
    assert err["cgs"] >= 1e3 * err["mgs"]                # ~ eps * kappa^2
    assert err["bcgs"] <= 1e-8


def test_block_length_limits_of_bcgs():
    X = _ill_conditioned(120, 9, 1e5, seed=3)
    Qm, Rm, _ = oracle.gs_qr(X, oracle.MGS)
    Qc, Rc, _ = oracle.gs_qr(X, oracle.CGS)
    Q1, R1, _ = oracle.gs_qr(X, oracle.BCGS, bl=1)
    Q9, R9, _ = oracle.gs_qr(X, oracle.BCGS, bl=9)
    np.testing.assert_array_equal(Q1, Qm)
    np.testing.assert_array_equal(R1, Rm)
    np.testing.assert_array_equal(Q9, Qc)
    np.testing.assert_array_equal(R9, Rc)
    # block length 4 is neither
    Q4, _, _ = oracle.gs_qr(X, oracle.BCGS, bl=4)
    assert not np.array_equal(Q4, Qm) and not np.array_equal(Q4, Qc)


@pytest.mark.parametrize("name", list(ORTHOS))
def test_arnoldi_equals_qr_of_the_krylov_matrix(name):
    A = gen.random200()
    n, k = A["n"], 6
    v0 = np.random.default_rng(5).standard_normal(n)
    steps, V, H = oracle.arnoldi(A, v0, k, ortho=ORTHOS[name])
    assert steps == k
    Ad = gen.to_dense(A)
    K = np.empty((n, k + 1))
    K[:, 0] = v0
    for j in range(k):
        K[:, j + 1] = Ad @ K[:, j]
    K /= np.linalg.norm(K, axis=0)
    Q, R = np.linalg.qr(K)
    Q *= np.sign(np.diag(R))
    np.testing.assert_allclose(V.T, Q, atol=1e-10)
    Href = Q.T @ Ad @ Q[:, :k]
    np.testing.assert_allclose(H, Href, atol=1e-9 * np.max(np.abs(Href)))


@pytest.mark.parametrize("name", list(ORTHOS))
def test_gmres_every_orthogonalisation_solves_poisson64(name):
    A = gen.poisson2d(64)
    b = oracle.spmv(A, np.ones(A["n"]))
    x, info = oracle.gmres(A, b, m=30, tol=1e-8, ortho=ORTHOS[name])
    _, ref = oracle.gmres(A, b, m=30, tol=1e-8, ortho=oracle.MGS)
    assert info["status"] == 0 and info["res_true"] <= 1e-8
    r = b - oracle.spmv(A, x)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b)
    assert abs(info["iters"] - ref["iters"]) <= 0.03 * ref["iters"]
    assert info["ortho"] == ORTHOS[name]


def test_accuracy_policy_chooses_the_orthogonalisation():
    A = gen.poisson2d(64)
    b = oracle.spmv(A, np.ones(A["n"]))
    _, loose = oracle.gmres(A, b, m=30, tol=1e-8, ortho=oracle.AUTO)
    _, tight = oracle.gmres(A, b, m=30, tol=1e-12, ortho=oracle.AUTO)
    assert loose["status"] == 0 and loose["faults"] == 0 and loose["ortho"] == oracle.BCGS
    assert tight["status"] == 0 and tight["faults"] == 0 and tight["ortho"] == oracle.MGS
    # at 1e-14 the implicit residual claims convergence the true one misses
    _, fault = oracle.gmres(A, b, m=30, tol=1e-14, ortho=oracle.AUTO, maxiter=20000)
    assert fault["faults"] >= 1 and fault["ortho"] == oracle.DGKS
    assert fault["status"] == 0 and fault["res_true"] <= 1e-14


def test_fault_check_off_stops_at_the_false_claim():
    """Without the accuracy mechanism (the time / memory / stable policies of
    Sec. 2.3.2 do not recompute the error) the solve ends at the first claimed
    convergence: the implicit residual meets tol, the true one does not
    (fault convergence, status -7); with it the same solve reaches tol."""
    A = gen.poisson2d(64)
    b = oracle.spmv(A, np.ones(A["n"]))
    x, off = oracle.gmres(A, b, m=30, tol=1e-14, maxiter=20000, fault_check=False)
    assert off["status"] == -7 and off["faults"] == 1
    assert off["res_implicit"] <= 1e-14 < off["res_true"]
    r = np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)
    assert abs(r - off["res_true"]) <= 1e-3 * r
    _, on = oracle.gmres(A, b, m=30, tol=1e-14, maxiter=20000, fault_check=True)
    assert on["status"] == 0 and on["res_true"] <= 1e-14 and on["faults"] == 1
