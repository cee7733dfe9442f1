"""GPU restarted Arnoldi (OpenATI_EIGENSOLVE, restarted Arnoldi for
unsymmetric matrices) against the CPU oracle and the mathematics.  With the
same start vector the GPU's wanted eigenvalues (largest real part or largest
modulus, complex pairs included) equal the oracle's and the spectrum fixed by
construction within 1e-8; every Ritz residual meets the tolerance; the
returned Ritz vectors satisfy ||A y - theta y|| <= 1e-6 |theta| on the
oracle's SpMV; the number of restarts matches the oracle's within one (both
keep the same invariant subspace at each restart, so only rounding differs);
every Gram-Schmidt variant converges to the same eigenvalues; the restart
rule grows m; an invariant start vector ends in a breakdown; bad arguments
are rejected."""
import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen
from tests._gpu import lib_and_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


def spectrum(A):
    e = []
    for a, b in A["blocks"]:
        e += [complex(a, b), complex(a, -b)] if b else [complex(a, 0.0)]
    return np.array(e)


def _run(xb, dev, A, nev, m, tol, which=0, ortho=None, m_max=None, seed=3, maxrestart=1000):
    import torch
    v0 = np.random.default_rng(seed).standard_normal(A["n"])
    plan = xb.Plan.from_host(A, dev)
    kw = {} if ortho is None else dict(ortho=ortho)
    ev, Y, info = plan.arnoldi(nev=nev, m=m, tol=tol, which=which, m_max=m_max,
                              maxrestart=maxrestart, v0=torch.tensor(v0, device=dev), **kw)
    eo, _, io = oracle.arnoldi_eig(A, nev=nev, m=m, tol=tol, which=which, m_max=m_max,
                                   maxrestart=maxrestart, v0=v0, vectors=False)
    return ev, Y, info, eo, io


def _check_vectors(A, ev, Y, info, tol):
    assert np.all(info["resid"] <= tol * np.abs(ev) * (1 + 1e-12))
    Yh = Y.cpu().numpy()
    for i in range(len(ev)):
        y = Yh[:, i]
        r = oracle.spmv(A, y.real) + 1j * oracle.spmv(A, y.imag) - ev[i] * y
        assert np.linalg.norm(r) <= 1e-6 * abs(ev[i]) + 1e-12, i
        assert abs(np.linalg.norm(y) - 1.0) <= 1e-8


@pytest.mark.parametrize("which", [0, 1])
def test_arnoldi_known_spectrum_matches_oracle(env, which):
    xb, dev = env
    A = gen.quasi_triangular(4000, seed=2, signed=which == 1)
    nev, tol = 10, 1e-10
    ev, Y, info, eo, io = _run(xb, dev, A, nev, 40, tol, which=which)
    assert info["status"] == 0 and io["status"] == 0, (info, io)
    e = spectrum(A)
    ref = e[oracle.wanted_order(e, which)[:nev]]
    np.testing.assert_allclose(ev, eo, atol=1e-8)
    np.testing.assert_allclose(ev, ref, atol=1e-8)
    assert np.any(np.abs(ev.imag) > 0.1)
    assert abs(info["restarts"] - io["restarts"]) <= 1, (info, io)
    _check_vectors(A, ev, Y, info, tol)


def test_arnoldi_toeplitz_closed_form(env):
    xb, dev = env
    n, l, d, u = 100, 1.0, 2.0, 1.2
    A = gen.toeplitz3(n, l, d, u)
    ev, Y, info, eo, io = _run(xb, dev, A, 5, 30, 1e-10)
    assert info["status"] == 0
    ref = d + 2 * np.sqrt(l * u) * np.cos(np.arange(1, 6) * np.pi / (n + 1))
    np.testing.assert_allclose(ev.real, ref, atol=1e-8)
    np.testing.assert_allclose(ev.imag, 0.0, atol=1e-8)
    np.testing.assert_allclose(ev, eo, atol=1e-8)


def test_arnoldi_convdiff_dense_spectrum(env):
    """Brute force: the wanted end of the dense spectrum of a small
    convection-diffusion matrix (7 x 8 x 9 grid), the paper's matrix class."""
    xb, dev = env
    A = gen.convdiff3d(8, pe=40.0, dims=(7, 8, 9))
    e = np.linalg.eigvals(gen.to_dense(A))
    ref = e[oracle.wanted_order(e, 0)[:6]]
    ev, Y, info, eo, io = _run(xb, dev, A, 6, 40, 1e-10)
    assert info["status"] == 0
    np.testing.assert_allclose(ev, ref, atol=1e-8 * np.max(np.abs(ref)))
    np.testing.assert_allclose(ev, eo, atol=1e-8 * np.max(np.abs(ref)))
    _check_vectors(A, ev, Y, info, 1e-10)


@pytest.mark.parametrize("ortho", [0, 1, 2, 3, 4])
def test_arnoldi_gram_schmidt_variants(env, ortho):
    xb, dev = env
    A = gen.quasi_triangular(3000, seed=5)
    ev, Y, info, eo, io = _run(xb, dev, A, 8, 30, 1e-9, ortho=ortho)
    assert info["status"] == 0, info
    e = spectrum(A)
    cgs = ortho == xb.ORTHO_CGS  # one classical pass: orthogonality only to ~1e-7
    np.testing.assert_allclose(ev, e[oracle.wanted_order(e, 0)[:8]], atol=1e-6 if cgs else 1e-7)
    if not cgs:
        assert abs(info["restarts"] - io["restarts"]) <= 2, (info, io)
        _check_vectors(A, ev, Y, info, 1e-9)


def test_arnoldi_restart_rule(env):
    xb, dev = env
    A = gen.quasi_triangular(3000, seed=7, ratio=0.999)  # top real parts 0.01 apart
    f = _run(xb, dev, A, 10, 20, 1e-8, seed=2, maxrestart=3000)
    r = _run(xb, dev, A, 10, 20, 1e-8, m_max=60, seed=2, maxrestart=3000)
    assert f[2]["status"] == 0 and r[2]["status"] == 0
    assert f[2]["m_final"] == 20 and r[2]["m_final"] > 20
    assert abs(r[2]["m_final"] - r[4]["m_final"]) <= 5, (r[2], r[4])
    assert r[2]["restarts"] < f[2]["restarts"]
    e = spectrum(A)
    np.testing.assert_allclose(r[0], e[oracle.wanted_order(e, 0)[:10]], atol=1e-7)
    np.testing.assert_allclose(r[0], r[3], atol=1e-7)


def test_arnoldi_breakdown_and_arguments(env):
    import torch
    xb, dev = env
    n = 50  # diag(1..50): A e_3 = 4 e_3 exactly, so the first step leaves w = 0
    A = dict(n=n, nnz=n, rowptr=np.arange(n + 1, dtype=np.int32),
             col=np.arange(n, dtype=np.int32), val=np.arange(1.0, n + 1), sym_upper=False)
    plan = xb.Plan.from_host(A, dev)
    v0 = torch.zeros(50, dtype=torch.float64, device=dev)
    v0[3] = 1.0
    ev, Y, info = plan.arnoldi(nev=2, m=6, tol=1e-10, v0=v0)
    assert info["status"] == xb.XB_EBREAKDOWN
    B = gen.quasi_triangular(200, seed=1)
    pb = xb.Plan.from_host(B, dev)
    for kw in (dict(nev=5, m=6), dict(nev=0, m=10), dict(nev=2, m=300),
               dict(nev=2, m=10, which=2), dict(nev=2, m=10, ortho=5),
               dict(nev=2, m=10, tol=0.0)):
        with pytest.raises(xb.XbError):
            pb.arnoldi(**kw)
    # restart limit: XB_ENOCONV with the current Ritz values
    ev, Y, info = pb.arnoldi(nev=4, m=8, tol=1e-14, maxrestart=2, vectors=False)
    assert info["status"] == xb.XB_ENOCONV and info["restarts"] == 2
    assert np.all(np.isfinite(ev))


def test_arnoldi_policies(env):
    """Numerical computation policies (Sec. 2.3.2, 3.3) on the eigensolver:
    every policy but NONE checks the true residuals of a claimed convergence;
    TIME / STABLE give the oracle's eigenvalues for their settings; MEMORY
    uses a short cycle and far less memory; ACCURACY ends within tol."""
    import torch
    xb, dev = env
    A = gen.quasi_triangular(20000, seed=11)
    n, nev, tol = A["n"], 10, 1e-8
    v0h = np.random.default_rng(4).standard_normal(n)
    v0 = torch.tensor(v0h, device=dev)
    e = spectrum(A)
    plan = xb.Plan.from_host(A, dev)
    out = {}
    for pol in (xb.POLICY_NONE, xb.POLICY_TIME, xb.POLICY_ACCURACY, xb.POLICY_MEMORY,
                xb.POLICY_STABLE):
        ev, Y, info = plan.arnoldi(nev=nev, m=40, tol=tol, v0=v0, policy=pol, maxrestart=3000,
                                   ortho=xb.ORTHO_DGKS)
        out[pol] = (ev, info)
        assert info["status"] in (xb.XB_OK, xb.XB_EFAULT), (pol, info)
        # every returned value is an eigenvalue of A (a short cycle may miss a wanted one)
        assert np.all(np.min(np.abs(e[:, None] - ev[None, :]), axis=0) <= 1e-6), pol
        if pol == xb.POLICY_NONE:
            assert info["true_resid"] == -1.0 and info["outer"] == 1
            continue
        if info["status"] == xb.XB_OK:
            assert 0.0 <= info["true_resid"] <= tol, (pol, info)
        else:
            assert info["true_resid"] > tol and pol != xb.POLICY_ACCURACY, (pol, info)
    t, a, mem, stb = (out[p][1] for p in (xb.POLICY_TIME, xb.POLICY_ACCURACY,
                                           xb.POLICY_MEMORY, xb.POLICY_STABLE))
    assert t["ortho_used"] == xb.ORTHO_BCGS and stb["ortho_used"] == xb.ORTHO_MGS
    assert mem["ortho_used"] == xb.ORTHO_MGS and mem["m_final"] == 20
    assert stb["m_final"] == 40 and 40 <= t["m_final"] <= 128
    assert a["status"] == xb.XB_OK
    assert mem["mem_bytes"] < t["mem_bytes"] / 3
    ref = e[oracle.wanted_order(e, 0)[:nev]]
    np.testing.assert_allclose(out[xb.POLICY_TIME][0], ref, atol=1e-7)
    np.testing.assert_allclose(out[xb.POLICY_STABLE][0], ref, atol=1e-7)
    # STABLE = the arguments with MGS and no rule: the oracle's iteration
    eo, _, io = oracle.arnoldi_eig(A, nev=nev, m=40, tol=tol, v0=v0h, vectors=False)
    np.testing.assert_allclose(out[xb.POLICY_STABLE][0], eo, atol=1e-7)
    assert abs(stb["restarts"] - io["restarts"]) <= 1, (stb, io)
