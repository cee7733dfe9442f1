"""Pins for the restart-frequency rule (Eq. 1, Fig. 2, Sec. 4.3), the matrix
features and the tuner MLP (finite differences, Adam's closed-form first
step) in the oracle."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen

HERE = os.path.dirname(__file__)
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))


def _mm_cases():
    out = []
    for line in open(os.path.join(HERE, "golden", "mm_ratio_cases.txt")):
        if line.startswith("#") or not line.strip():
            continue
        head, seq = line.split("|")
        s, t, exp = head.split()
        out.append((int(s), int(t), float(exp), [float(v) for v in seq.split()]))
    return out


@pytest.mark.parametrize("s,t,expected,seq", _mm_cases())
def test_mm_ratio_hand_cases(s, t, expected, seq):
    assert oracle.mm_ratio(seq, s, t) == expected


def test_dafrt_judgement():
    # Halving residuals over I=5 samples -> R = 16: no stagnation at theta=10
    assert oracle.dafrt([1, 0.5, 0.25, 0.125, 0.0625], 10.0) == 0
    # flat residuals -> R = 1: stagnation, increase the restart frequency
    assert oracle.dafrt([1, 1, 1, 1, 1], 10.0) == 1
    assert oracle.dafrt([1, 0.5, 0.25, 0.125, 0.0625], 20.0) == 1


def test_dafrt_cadence_in_gmres():
    # Poisson with a tiny restart length stagnates; the rule samples the true
    # residual at every restart (Sec. 4.3), judges every I=5 samples (Fig. 2)
    # and grows m by 5 (Sec. 4.3) up to m_max.
    I = GOLD["dafrt_fig2"]["judgement_period_I"]
    dm = GOLD["dafrt_sec43"]["increment"]
    A = gen.poisson2d(24)
    b = oracle.spmv(A, np.ones(A["n"]))
    x, info = oracle.gmres(A, b, m=2, m_max=17, tol=1e-8, maxiter=3000, dafrt=True,
                           theta=10.0, window=I, dm=dm, hist_cap=400)
    mh, h = info["mhist"], info["hist"]
    assert mh[0] == 2
    changes = np.flatnonzero(np.diff(mh)) + 1
    assert changes.size >= 1
    for c in changes:
        assert c % I == 0                      # only at judgement points
        assert mh[c] - mh[c - 1] == dm or mh[c] == 17
        # the judgement saw stagnation over the last I samples (cycles c-I+1..c)
        w = h[c - I + 1:c + 1]
        assert w.max() / w.min() < 10.0
    assert mh.max() <= 17
    # without the rule, m stays fixed
    x2, i2 = oracle.gmres(A, b, m=2, tol=1e-8, maxiter=3000, hist_cap=400)
    assert np.all(i2["mhist"] == 2)
    # and the rule pays off on this stagnating problem
    assert info["iters"] < i2["iters"] or i2["status"] != 0


def test_features_hand_built():
    # 4x4: rows lengths 2,1,3,0; entries (0,0),(0,3),(1,1),(2,0),(2,2),(2,3)
    A = dict(n=4, nnz=6, rowptr=np.array([0, 2, 3, 6, 6], np.int32),
             col=np.array([0, 3, 1, 0, 2, 3], np.int32),
             val=np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0]), sym_upper=False)
    raw, f = oracle.features(A)
    assert list(raw) == [4, 6, 1.5, 1.25, 3, 3, 0]
    np.testing.assert_allclose(f, [np.log(5), np.log(7), np.log(2.5), np.log(2.25),
                                   np.log(4), np.log(4), 0, np.log(4) - np.log(2.5)])
    F = gen.poisson2d(4)
    raw, f = oracle.features(F)
    assert raw[6] == 1 and raw[5] == 4 and raw[4] == 5 and raw[1] == 5 * 16 - 16
    U = gen.laplace3d(3, upper=True)
    assert oracle.features(U)[0][6] == 1
    P = gen.powerlaw(n=500, seed=1)
    assert oracle.features(P)[0][6] == 0


DIMS = (8, 16, 12, (4, 3, 5))


def _params(seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(oracle.mlp_param_count(*DIMS[:3], DIMS[3])) * 0.4


def test_mlp_gradient_finite_differences():
    P = _params()
    rng = np.random.default_rng(1)
    X = rng.standard_normal((7, 8))
    lab = np.stack([rng.integers(0, k, 7) for k in DIMS[3]], axis=1)
    loss, g = oracle.mlp_loss_grad(P, DIMS, X, lab)
    assert loss > 0
    eps = 1e-6
    idx = rng.choice(P.size, 60, replace=False)
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += eps
        Pm[i] -= eps
        fd = (oracle.mlp_loss_grad(Pp, DIMS, X, lab)[0] - oracle.mlp_loss_grad(Pm, DIMS, X, lab)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd))


def test_mlp_forward_matches_numpy():
    P = _params(3)
    d, h1, h2, heads = DIMS
    o = sum(heads)
    X = np.random.default_rng(2).standard_normal((5, d))
    W1 = P[:h1 * d].reshape(h1, d); p = h1 * d
    b1 = P[p:p + h1]; p += h1
    W2 = P[p:p + h2 * h1].reshape(h2, h1); p += h2 * h1
    b2 = P[p:p + h2]; p += h2
    W3 = P[p:p + o * h2].reshape(o, h2); p += o * h2
    b3 = P[p:p + o]
    ref = np.maximum(np.maximum(X @ W1.T + b1, 0) @ W2.T + b2, 0) @ W3.T + b3
    np.testing.assert_allclose(oracle.mlp_forward(P, DIMS, X), ref, rtol=1e-12, atol=1e-12)


def test_adam_first_step_closed_form():
    # t = 1 from zero moments: m_hat = g, v_hat = g^2 -> p -= lr * g / (|g| + eps)
    P = np.array([1.0, -2.0, 0.5, 3.0])
    G = np.array([0.3, -1e-3, 0.0, 5.0])
    M, V = np.zeros(4), np.zeros(4)
    P0 = P.copy()
    oracle.adam(P, G, M, V, 1, lr=0.01)
    np.testing.assert_allclose(P, P0 - 0.01 * G / (np.abs(G) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(M, 0.1 * G)
    np.testing.assert_allclose(V, 0.001 * G * G)


def test_adam_training_reduces_loss():
    P = _params(5)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((32, 8))
    lab = np.stack([(X[:, 0] > 0).astype(int), (X[:, 1] > 0).astype(int),
                    (X[:, 2] > 0).astype(int)], axis=1)
    M, V = np.zeros_like(P), np.zeros_like(P)
    l0 = oracle.mlp_loss_grad(P, DIMS, X, lab)[0]
    for t in range(1, 201):
        _, g = oracle.mlp_loss_grad(P, DIMS, X, lab)
        oracle.adam(P, g, M, V, t, lr=1e-2)
    assert oracle.mlp_loss_grad(P, DIMS, X, lab)[0] < 0.2 * l0
