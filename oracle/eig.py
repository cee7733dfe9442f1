"""Restarted Arnoldi eigensolver: the CPU oracle (test infrastructure only).

Plain numpy / scipy in FP64, written from the mathematics of the method the
paper names for unsymmetric eigenproblems (OpenATI_EIGENSOLVE, restarted
Arnoldi, Sec. 2.2; 10 eigenpairs to 1e-8, Sec. 4.3; restart-frequency rule,
Eq. 1 and Sec. 4.3).  The paper gives no restart scheme, so this follows the
Krylov-Schur restart: after a cycle of m Arnoldi steps,

    A V_m = V_m H_m + beta v_m e_m^T,

the real Schur form H_m = Z T Z^T is ordered with the k wanted Ritz values
leading (library routine: scipy.linalg.schur with a sort rule), and the
relation is cut to

    A (V_m Z_k) = (V_m Z_k) T_k + v_m (beta e_m^T Z_k),

from which the next cycle continues.  The SpMV is the oracle's C CRS kernel;
the Gram-Schmidt step is classical Gram-Schmidt applied twice (DGKS) in plain
numpy; the Ritz pairs of each cycle come from numpy.linalg.eig.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

LR, LM = 0, 1


def _key(z, which):
    return np.abs(z) if which == LM else np.real(z)


def wanted_order(vals, which=LR):
    """Indices of vals in wanted order: key descending, ties by imaginary
    part descending (a conjugate pair: positive imaginary part first)."""
    vals = np.asarray(vals)
    return sorted(range(len(vals)), key=lambda i: (-_key(vals[i], which), -vals[i].imag))


def restart_basis(Hm, lam, order, kk, which=LR):
    """The restart step: an orthonormal real basis Q (m x k) of the invariant
    subspace of Hm belonging to its kk wanted eigenvalues (lam[order[:kk]],
    conjugate pairs kept whole), from scipy's real Schur form ordered by a
    threshold between the kk-th and (kk+1)-th keys, and T_k = Q^T Hm Q (the
    leading quasi-triangular block).  k = kk unless keys tie at the threshold."""
    thr = 0.5 * (_key(lam[order[kk - 1]], which) + _key(lam[order[kk]], which))
    T, Z, sdim = scipy.linalg.schur(
        Hm, output="real", sort=lambda re, im: _key(complex(re, im), which) > thr)
    return Z[:, :sdim], T[:sdim, :sdim]


def arnoldi_eig(A, nev=10, m=20, tol=1e-8, maxrestart=1000, v0=None, which=LR, m_max=None,
                theta=10.0, vectors=True):
    """nev eigenvalues of the general CRS matrix A at the wanted end (LR:
    largest real part, LM: largest modulus) and their unit Ritz vectors;
    returns (evals (complex, nev), evecs (n x nev complex) or None, info).
    Convergence: |beta e_m^T y_i| <= tol |theta_i| for every wanted pair.
    m_max > m turns on the restart rule: the worst relative wanted residual of
    each cycle is a sample; every 5 samples, if the MM ratio of the last 5 is
    below theta, m grows by 5 (up to m_max)."""
    from . import dafrt, spmv  # the oracle's C CRS SpMV and restart judgement
    n = A["n"]
    if m < nev + 2 or m > n:
        raise ValueError("need nev + 2 <= m <= n")
    M = m if m_max is None else max(m, m_max)
    v = np.ones(n) if v0 is None else np.array(v0, dtype=np.float64)
    V = np.zeros((M + 1, n))
    Hb = np.zeros((M + 1, M))
    V[0] = v / np.linalg.norm(v)
    k = steps = restarts = 0
    samples = []
    status = -4
    while True:
        for j in range(k, m):
            w = spmv(A, V[j])
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            h2 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h2
            Hb[:j + 1, j] = h + h2
            Hb[j + 1, j] = np.linalg.norm(w)
            steps += 1
            if not Hb[j + 1, j] > 0.0:
                info = dict(status=-5, steps=steps, restarts=restarts, m_final=m,
                            resid=np.full(nev, np.nan))
                return np.full(nev, np.nan + 0j), None, info
            V[j + 1] = w / Hb[j + 1, j]
        Hm = Hb[:m, :m].copy()
        beta = Hb[m, m - 1]
        lam, Y = np.linalg.eig(Hm)
        order = wanted_order(lam, which)
        want = order[:nev]
        resid = np.abs(beta) * np.abs(Y[m - 1, want])
        vals = lam[want]
        conv = bool(np.all(resid <= tol * np.abs(vals)))
        if conv or restarts >= maxrestart:
            status = 0 if conv else -4
            evecs = V[:m].T @ Y[:, want] if vectors else None
            break
        m_next = m
        if M > m or samples:
            samples.append(float(np.max(resid / np.abs(vals))))
            if len(samples) == 5:
                if dafrt(samples, theta):
                    m_next = min(m + 5, M)
                samples = []
        kk = nev + (m - nev) // 2
        if lam[order[kk - 1]].imag > 0:  # first of a conjugate pair: keep both
            kk = kk + 1 if kk + 1 <= m - 1 else kk - 1
        Q, Tk = restart_basis(Hm, lam, order, kk, which)
        sdim = Q.shape[1]
        V[:sdim] = Q.T @ V[:m]
        V[sdim] = V[m]
        Hb[:] = 0.0
        Hb[:sdim, :sdim] = Tk
        Hb[sdim, :sdim] = beta * Q[m - 1, :]
        k = sdim
        m = m_next
        restarts += 1
    info = dict(status=status, steps=steps, restarts=restarts, m_final=m, resid=resid)
    return vals, evecs, info
