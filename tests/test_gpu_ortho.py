"""GPU re-orthogonalisations (Sec. 3.2.2: MGS, CGS, DGKS, BCGS with block
length 4) and the accuracy policy (Sec. 3.3.2) against the CPU oracle, through
the C ABI.

xb_orth: V is the oracle's Gram-Schmidt Q of a seeded matrix X (kappa 1e3)
with the same orthogonalisation, w the next column of X; the GPU's projection
coefficients and norm must equal the oracle's R column within 1e-11 of
||x|| (dot-product rounding over n terms, amplified at most by kappa for the
classical variants), on even n (16-byte vector path) and odd n (scalar
path), with more basis vectors than one launch's 16 dots and a partial last
block of 4.  GMRES with each orthogonalisation reaches the true residual and
the oracle's iteration count within max(3, 5 %)."""
import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen
from tests._gpu import lib_and_device

pytestmark = pytest.mark.gpu
NAMES = {"mgs": 0, "cgs": 1, "dgks": 2, "bcgs": 3}


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


def _X(n, k, kappa, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, k)))
    W, _ = np.linalg.qr(rng.standard_normal((k, k)))
    return U @ np.diag(np.logspace(0, -np.log10(kappa), k)) @ W.T


@pytest.mark.parametrize("name", list(NAMES))
@pytest.mark.parametrize("n,k", [(6000, 21), (5003, 9), (4096, 1), (130, 4)])
def test_orth_matches_oracle(env, name, n, k):
    xb, dev = env
    import torch
    o = NAMES[name]
    X = _X(n, k + 1, 1e3, seed=n + k)
    Q, R, done = oracle.gs_qr(X, o)
    assert done == k + 1
    plan = xb.Plan.from_host(gen.laplace1d(n), dev)
    V = torch.tensor(np.ascontiguousarray(Q[:, :k].T), device=dev)
    w = torch.tensor(X[:, k].copy(), device=dev)
    h = plan.orth(V, w, o).cpu().numpy()
    scale = np.linalg.norm(X[:, k])
    np.testing.assert_allclose(h[:k], R[:k, k], rtol=0, atol=1e-11 * scale)
    assert abs(h[k] - R[k, k]) <= 1e-11 * scale
    # w left orthogonal to the basis, with the reported norm
    wn = w.cpu().numpy()
    assert abs(np.linalg.norm(wn) - h[k]) <= 1e-12 * scale
    assert np.max(np.abs(Q[:, :k].T @ wn)) <= 1e-10 * scale


def test_orth_rejects_bad_arguments(env):
    xb, dev = env
    import torch
    plan = xb.Plan.from_host(gen.laplace1d(64), dev)
    V = torch.zeros((3, 64), dtype=torch.float64, device=dev)
    w = torch.ones(64, dtype=torch.float64, device=dev)
    for o in (4, -1, 7):
        with pytest.raises(RuntimeError):
            plan.orth(V, w, o)


def _gmres(xb, dev, A, **opt):
    import torch
    plan = xb.Plan.from_host(A, dev)
    b = oracle.spmv(A, np.ones(A["n"]))
    x = torch.zeros(A["n"], dtype=torch.float64, device=dev)
    info = plan.gmres(torch.tensor(b, device=dev), x, **opt)
    xh = x.cpu().numpy()
    return info, np.linalg.norm(b - oracle.spmv(A, xh)) / np.linalg.norm(b), b


@pytest.mark.parametrize("name", list(NAMES))
@pytest.mark.parametrize("mat,make,m", [
    ("poisson64", lambda: gen.poisson2d(64), 30),
    ("convdiff12", lambda: gen.convdiff3d(N=12), 20),
    ("random200", lambda: gen.random200(), 30),
])
def test_gmres_each_orthogonalisation_matches_oracle(env, name, mat, make, m):
    xb, dev = env
    A = make()
    info, rel, b = _gmres(xb, dev, A, m=m, tol=1e-8, ortho=NAMES[name])
    _, io = oracle.gmres(A, b, m=m, tol=1e-8, ortho=NAMES[name])
    assert info["status"] == 0 and rel <= 1e-8, info
    assert info["ortho_used"] == NAMES[name]
    assert abs(info["iters"] - io["iters"]) <= max(3, 0.05 * io["iters"]), (info["iters"], io["iters"])


def test_accuracy_policy(env):
    xb, dev = env
    A = gen.poisson2d(64)
    loose, rel, _ = _gmres(xb, dev, A, m=30, tol=1e-8, ortho=4)
    assert loose["status"] == 0 and rel <= 1e-8 and loose["ortho_used"] == 3
    tight, rel, _ = _gmres(xb, dev, A, m=30, tol=1e-12, ortho=4)
    assert tight["status"] == 0 and rel <= 1e-12
    assert tight["ortho_used"] == (2 if tight["faults"] else 0)
    fault, rel, _ = _gmres(xb, dev, A, m=30, tol=1e-14, ortho=4, maxiter=20000)
    assert fault["ortho_used"] == (2 if fault["faults"] else 0)
    assert fault["status"] == 0 and rel <= 1e-14


@pytest.mark.parametrize("name", ["cgs", "dgks", "bcgs"])
def test_mixed_refinement_with_block_orthogonalisations(env, name):
    xb, dev = env
    A = gen.convdiff3d(N=16)
    info, rel, _ = _gmres(xb, dev, A, m=30, tol=1e-8, precision=xb.PREC_MIXED, tol_inner=1e-4,
                          ortho=NAMES[name])
    assert info["status"] == 0 and rel <= 1e-8, info
    assert info["ortho_used"] == NAMES[name]
