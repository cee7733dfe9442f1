"""Pins of the oracle's restarted Arnoldi eigensolver (OpenATI_EIGENSOLVE,
restarted Arnoldi for unsymmetric matrices, Sec. 2.2 / 4.3), and of the
library's host-side dense eigen step against numpy:
  - block upper-triangular matrices whose spectrum is fixed by construction
    (1 x 1 blocks a, 2 x 2 blocks [[a, b], [-b, a]] -> a +- ib): the wanted
    eigenvalues, largest real part and largest modulus, complex pairs included;
    every returned eigenvalue is one of the matrix's;
  - the tridiagonal Toeplitz closed form d + 2 sqrt(l u) cos(j pi / (n + 1));
  - the symmetric special case: the 1D Laplacian closed form;
  - brute force: the dense spectrum of a random sparse nonsymmetric matrix;
  - returned Ritz vectors satisfy A y = theta y to the requested tolerance
    (so the restart keeps a valid Arnoldi relation), and the residual
    estimate |beta e_m^T s| equals the true residual;
  - the restart rule grows m on a stagnating problem; an invariant start
    vector ends in a breakdown."""
import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen


def spectrum(A):
    e = []
    for a, b in A["blocks"]:
        e += [complex(a, b), complex(a, -b)] if b else [complex(a, 0.0)]
    return np.array(e)


def same_multiset(a, b, tol):
    """Every value of a matched to a distinct value of b within tol (greedy,
    nearest first): the two lists hold the same eigenvalues."""
    b = list(np.asarray(b))
    for x in np.asarray(a):
        d = [abs(x - y) for y in b]
        i = int(np.argmin(d))
        if d[i] > tol:
            return False
        b.pop(i)
    return not b


def true_resid(A, ev, X):
    D = gen.to_dense(A)
    return np.array([np.linalg.norm(D @ X[:, i] - ev[i] * X[:, i]) for i in range(len(ev))])


@pytest.mark.parametrize("which", [oracle.EIG_LR, oracle.EIG_LM])
def test_quasi_triangular_known_spectrum(which):
    n, nev = 400, 8
    A = gen.quasi_triangular(n, seed=2, signed=which == oracle.EIG_LM)
    v0 = np.random.default_rng(3).standard_normal(n)
    ev, X, info = oracle.arnoldi_eig(A, nev=nev, m=30, tol=1e-10, v0=v0, which=which)
    assert info["status"] == 0 and info["restarts"] > 0
    e = spectrum(A)
    ref = e[oracle.wanted_order(e, which)[:nev]]
    np.testing.assert_allclose(ev, ref, atol=1e-8)
    assert np.any(np.abs(ev.imag) > 0.1)  # complex pairs among the wanted ones
    assert np.all(np.min(np.abs(e[:, None] - ev[None, :]), axis=0) <= 1e-8)
    r = true_resid(A, ev, X)
    assert np.all(r <= 1e-9 * np.abs(ev))
    # the estimate the stopping test uses is the true residual
    np.testing.assert_allclose(r, info["resid"], rtol=1e-3, atol=1e-11)
    np.testing.assert_allclose(np.linalg.norm(X, axis=0), 1.0, atol=1e-12)


@pytest.mark.parametrize("which", [oracle.EIG_LR, oracle.EIG_LM])
def test_restart_basis_spans_the_wanted_invariant_subspace(which):
    """The restart step on its own: Q is orthonormal, H Q = Q T_k (an
    invariant subspace), and T_k carries exactly the kk wanted eigenvalues,
    conjugate pairs whole."""
    from oracle.eig import restart_basis
    rng = np.random.default_rng(21 + which)
    for m in (12, 30):
        H = np.triu(rng.standard_normal((m, m)), -1)  # upper Hessenberg, like H_m
        lam = np.linalg.eigvals(H)
        order = oracle.wanted_order(lam, which)
        kk = m // 2
        if lam[order[kk - 1]].imag > 0:
            kk += 1
        Q, Tk = restart_basis(H, lam, order, kk, which)
        assert Q.shape == (m, kk)
        np.testing.assert_allclose(Q.T @ Q, np.eye(kk), atol=1e-13)
        assert np.max(np.abs(H @ Q - Q @ Tk)) <= 1e-12 * np.max(np.abs(H))
        got = np.sort_complex(np.linalg.eigvals(Tk))
        want = np.sort_complex(lam[order[:kk]])
        np.testing.assert_allclose(got, want, atol=1e-10)


def test_toeplitz_closed_form():
    n, l, d, u = 100, 1.0, 2.0, 1.2
    A = gen.toeplitz3(n, l, d, u)
    ev, X, info = oracle.arnoldi_eig(A, nev=5, m=30, tol=1e-10,
                                     v0=np.random.default_rng(1).standard_normal(n))
    assert info["status"] == 0
    ref = d + 2 * np.sqrt(l * u) * np.cos(np.arange(1, 6) * np.pi / (n + 1))
    np.testing.assert_allclose(ev.real, ref, atol=1e-8)
    np.testing.assert_allclose(ev.imag, 0.0, atol=1e-8)


def test_symmetric_special_case_laplacian():
    n = 200
    A = gen.laplace1d(n)
    ev, X, info = oracle.arnoldi_eig(A, nev=4, m=30, tol=1e-10,
                                     v0=np.random.default_rng(1).standard_normal(n))
    assert info["status"] == 0
    ref = 2 + 2 * np.cos(np.arange(1, 5) * np.pi / (n + 1))
    np.testing.assert_allclose(ev, ref, atol=1e-9)


def test_random_sparse_brute_force():
    A = gen.random200(200, per_row=5, diag=0.0, seed=4)
    e = np.linalg.eigvals(gen.to_dense(A))
    ref = e[oracle.wanted_order(e, oracle.EIG_LR)[:6]]
    ev, X, info = oracle.arnoldi_eig(A, nev=6, m=24, tol=1e-10,
                                     v0=np.random.default_rng(5).standard_normal(200))
    assert info["status"] == 0
    np.testing.assert_allclose(ev, ref, atol=1e-8)
    assert np.all(true_resid(A, ev, X) <= 1e-9 * np.abs(ev))


def test_restart_rule_grows_m():
    A = gen.quasi_triangular(3000, seed=7, ratio=0.999)  # top real parts 0.01 apart
    v0 = np.random.default_rng(2).standard_normal(A["n"])
    fixed = oracle.arnoldi_eig(A, nev=10, m=20, tol=1e-8, v0=v0, vectors=False,
                               maxrestart=3000)[2]
    rule = oracle.arnoldi_eig(A, nev=10, m=20, m_max=60, tol=1e-8, v0=v0, vectors=False,
                              maxrestart=3000)[2]
    assert fixed["status"] == 0 and rule["status"] == 0
    assert fixed["m_final"] == 20 and rule["m_final"] > 20
    assert rule["restarts"] < fixed["restarts"]


def test_invariant_start_vector_breaks_down():
    n = 50  # diag(1..50): A e_3 = 4 e_3 exactly, so the first step leaves w = 0
    A = dict(n=n, nnz=n, rowptr=np.arange(n + 1, dtype=np.int32),
             col=np.arange(n, dtype=np.int32), val=np.arange(1.0, n + 1), sym_upper=False)
    v0 = np.zeros(50)
    v0[3] = 1.0
    ev, X, info = oracle.arnoldi_eig(A, nev=2, m=6, tol=1e-10, v0=v0)
    assert info["status"] == -5


@pytest.mark.parametrize("which", [0, 1])
def test_library_restart_basis(which):
    """The library's own restart step (host logic, the one xb_arnoldi runs):
    an orthonormal real basis of the invariant subspace of the k wanted
    eigenvalues, pairs whole; it spans the oracle's restart subspace."""
    import paper_2405_01599_gb300 as xb
    try:
        xb.lib()
    except ImportError:
        pytest.skip("CUDA library not built")
    from oracle.eig import restart_basis
    rng = np.random.default_rng(31 + which)
    for m in (10, 25, 40):
        H = np.triu(rng.standard_normal((m, m)), -1)
        lam = np.linalg.eigvals(H)
        order = oracle.wanted_order(lam, which)
        k0 = m // 2
        Q = xb.dense_restart_basis(H, k0, which)
        kk = Q.shape[1]
        want_k = k0 + 1 if lam[order[k0 - 1]].imag > 0 else k0
        assert kk == want_k
        np.testing.assert_allclose(Q.T @ Q, np.eye(kk), atol=1e-12)
        Tk = Q.T @ H @ Q
        assert np.max(np.abs(H @ Q - Q @ Tk)) <= 1e-11 * np.max(np.abs(H))
        assert same_multiset(np.linalg.eigvals(Tk), lam[order[:kk]], 1e-9)
        Qo, _ = restart_basis(H, lam, order, kk, which)  # the oracle's subspace
        s = np.linalg.svd(Qo.T @ Q, compute_uv=False)
        np.testing.assert_allclose(s, 1.0, atol=1e-9)  # same subspace: all cosines 1


def test_dense_eig_special_matrices():
    """Host dense step on matrices with a known spectrum: zero, 1 x 1, a
    rotation (+-2i), a Jordan block (defective, all 2), the cyclic
    permutation (roots of unity), extreme scalings."""
    import paper_2405_01599_gb300 as xb
    try:
        xb.lib()
    except ImportError:
        pytest.skip("CUDA library not built")
    w, V = xb.dense_eig(np.zeros((5, 5)))
    assert np.all(w == 0)
    w, V = xb.dense_eig(np.array([[3.0]]))
    assert w[0] == 3.0 and V[0, 0] == 1.0
    w, V = xb.dense_eig(np.array([[0.0, 2.0], [-2.0, 0.0]]))
    np.testing.assert_allclose(w, [2j, -2j], atol=1e-15)
    J = np.diag(np.full(6, 2.0)) + np.diag(np.ones(5), 1)
    w, V = xb.dense_eig(J)
    np.testing.assert_allclose(w, 2.0, atol=1e-14)
    assert np.max(np.abs(J @ V - V * w)) <= 1e-14
    n = 30
    P = np.roll(np.eye(n), 1, axis=1)
    w, V = xb.dense_eig(P, xb.EIG_LR)
    roots = np.exp(2j * np.pi * np.arange(n) / n)
    assert same_multiset(w, roots, 1e-13)
    R = np.random.default_rng(0).standard_normal((40, 40))
    ref = np.linalg.eigvals(R)
    for scale in (1e150, 1e-150):
        w, V = xb.dense_eig(R * scale)
        assert same_multiset(w / scale, ref, 1e-12)
        assert np.max(np.abs(R @ V - V * (w / scale))) <= 1e-12


def test_dense_eig_host_step_matches_numpy():
    """The library's host-side dense eigen step (Schur form, ordering,
    eigenvectors) against numpy: host logic only, no device work."""
    import paper_2405_01599_gb300 as xb
    try:
        xb.lib()
    except ImportError:
        pytest.skip("CUDA library not built")
    rng = np.random.default_rng(11)
    for trial in range(60):
        n = int(rng.integers(1, 50))
        kind = trial % 4
        if kind == 0:
            D = rng.standard_normal((n, n))
        elif kind == 1:
            D = np.triu(rng.standard_normal((n, n)), -1)
        elif kind == 2:
            B = rng.standard_normal((n, n))
            D = B + B.T
        else:
            D = np.diag(rng.integers(-3, 3, n).astype(float))  # repeated eigenvalues
        for which in (xb.EIG_LR, xb.EIG_LM):
            w, V = xb.dense_eig(D, which)
            e = np.linalg.eigvals(D)
            ref = e[oracle.wanted_order(e, which)]
            sc = max(1.0, np.max(np.abs(e)))
            key = lambda z: sorted(z, key=lambda c: (round(c.real, 7), round(c.imag, 7)))
            assert np.max(np.abs(np.array(key(w)) - np.array(key(ref)))) <= 1e-10 * sc
            k = np.abs(w) if which == xb.EIG_LM else w.real
            assert np.all(np.diff(k) <= 1e-9 * sc)
            assert np.max(np.abs(D @ V - V * w)) <= 1e-10 * sc
            np.testing.assert_allclose(np.linalg.norm(V, axis=0), 1.0, atol=1e-12)
            for t in range(n):  # conjugate pairs adjacent, positive imaginary part first
                if w[t].imag > 0:
                    assert t + 1 < n and w[t + 1] == np.conj(w[t])
