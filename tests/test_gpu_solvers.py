"""GPU Krylov solvers and vector kernels against the CPU oracle (C ABI).

Solver parity: both reach the true residual ||b - A x|| / ||b|| <= tol (the
GPU's x re-evaluated by the oracle's SpMV), FP64 iteration counts agree
within max(3, 5 %) for GMRES and max(3, 10 %) for BiCGStab (rounding order
differs; BiCGStab's recurrences amplify it more)."""
import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen
from tests._gpu import lib_and_device

pytestmark = pytest.mark.gpu
TOL = 1e-8


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


def _true_rel(A, x, b):
    return np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)


# the three GMRES paths: one launch from one cluster's shared memory, one
# launch of the batched kernel (basis in global memory), and the multi-launch
# Arnoldi loop
PATHS = ["resident", "batched", "multi"]


def _path(monkeypatch, path):
    """Select a GMRES path; returns the small_n option for it."""
    monkeypatch.setenv("XB_RESIDENT_CL", "0" if path == "batched" else "")
    if path != "batched":
        monkeypatch.delenv("XB_RESIDENT_CL")
    return 0 if path == "multi" else 8192


def _persistent(path, A):
    if path == "multi" or A["sym_upper"]:
        return 0
    return 2 if path == "resident" else 1


def _solve(xb, dev, A, which, b=None, x0=None, **opt):
    import torch
    plan = xb.Plan.from_host(A, dev)
    if b is None:
        b = oracle.spmv(A, np.ones(A["n"]))
    bt = torch.tensor(b, device=dev)
    xt = torch.zeros(A["n"], dtype=torch.float64, device=dev) if x0 is None else torch.tensor(x0, device=dev)
    info = (plan.gmres if which == "gmres" else plan.bicgstab)(bt, xt, **opt)
    return info, xt.cpu().numpy(), b


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("name,make,m", [
    ("poisson64", lambda: gen.poisson2d(64), 30),
    ("random200", lambda: gen.random200(), 30),
    ("convdiff10", lambda: gen.convdiff3d(N=10), 20),
    ("laplace3d_10_upper", lambda: gen.laplace3d(10, upper=True), 25),
])
def test_gmres_matches_oracle(env, monkeypatch, name, make, m, path):
    """Every GMRES path: one persistent launch for small general systems
    (small_n = 8192, the default), from shared memory or through the batched
    kernel, and the multi-launch path (small_n = 0; symmetric storage always
    takes it)."""
    xb, dev = env
    A = make()
    small_n = _path(monkeypatch, path)
    info, x, b = _solve(xb, dev, A, "gmres", m=m, tol=TOL, small_n=small_n)
    xo, io = oracle.gmres(A, b, m=m, tol=TOL)
    assert info["persistent"] == _persistent(path, A)
    assert info["status"] == 0, info
    assert _true_rel(A, x, b) <= TOL
    assert abs(info["iters"] - io["iters"]) <= max(3, 0.05 * io["iters"]), (info["iters"], io["iters"])
    assert np.linalg.norm(x - xo) <= 1e-5 * np.linalg.norm(xo)


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_gmres_each_spmv_variant(env, variant):
    xb, dev = env
    A = gen.powerlaw(n=4000, seed=4)
    info, x, b = _solve(xb, dev, A, "gmres", m=40, tol=TOL, variant=variant, maxiter=20000,
                        small_n=0)
    assert info["status"] == 0 and _true_rel(A, x, b) <= TOL
    assert info["variant_used"] == variant


def test_gmres_check_every_is_transparent(env):
    xb, dev = env
    A = gen.poisson2d(40)
    i1, x1, b = _solve(xb, dev, A, "gmres", m=30, tol=TOL, check_every=1, small_n=0)
    i4, x4, _ = _solve(xb, dev, A, "gmres", m=30, tol=TOL, check_every=7, small_n=0)
    assert i1["iters"] == i4["iters"] and i1["restarts"] == i4["restarts"]
    np.testing.assert_array_equal(x1, x4)


@pytest.mark.parametrize("path", PATHS)
def test_gmres_dafrt_matches_oracle(env, monkeypatch, path):
    xb, dev = env
    A = gen.poisson2d(24)
    small_n = _path(monkeypatch, path)
    info, x, b = _solve(xb, dev, A, "gmres", m=2, m_max=17, tol=TOL, dafrt=1, dafrt_theta=10.0,
                        dafrt_window=5, dafrt_dm=5, maxiter=3000, small_n=small_n)
    assert info["persistent"] == _persistent(path, A)
    xo, io = oracle.gmres(A, b, m=2, m_max=17, tol=TOL, maxiter=3000, dafrt=True, theta=10.0,
                          window=5, dm=5)
    assert info["m_final"] == io["m_final"] and info["m_final"] > 2
    assert abs(info["iters"] - io["iters"]) <= max(3, 0.05 * io["iters"])
    assert info["status"] == io["status"]


@pytest.mark.parametrize("path", PATHS)
def test_gmres_edge_cases(env, monkeypatch, path):
    xb, dev = env
    small_n = _path(monkeypatch, path)
    A = gen.poisson2d(10)
    n = A["n"]
    info, x, _ = _solve(xb, dev, A, "gmres", b=np.zeros(n), x0=np.ones(n), small_n=small_n)
    assert info["status"] == 0 and np.all(x == 0)
    info, x, b = _solve(xb, dev, A, "gmres", m=5, tol=1e-12, maxiter=20, small_n=small_n)
    assert info["status"] == xb.XB_ENOCONV and info["iters"] == 20 and info["res_true"] > 1e-12
    I = dict(n=50, nnz=50, rowptr=np.arange(51, dtype=np.int32), col=np.arange(50, dtype=np.int32),
             val=np.ones(50), sym_upper=False)
    info, x, b = _solve(xb, dev, I, "gmres", b=np.random.default_rng(0).standard_normal(50),
                        small_n=small_n)
    assert info["status"] == 0 and info["iters"] == 1
    np.testing.assert_allclose(x, b, rtol=1e-15)
    Z = dict(n=6, nnz=0, rowptr=np.zeros(7, np.int32), col=np.zeros(0, np.int32), val=np.zeros(0),
             sym_upper=False)
    info, x, b = _solve(xb, dev, Z, "gmres", b=np.ones(6), small_n=small_n)
    assert info["status"] == xb.XB_EBREAKDOWN
    info, x, b = _solve(xb, dev, Z, "bicgstab", b=np.ones(6))
    assert info["status"] == xb.XB_EBREAKDOWN


@pytest.mark.parametrize("ncl,mat,m", [
    (2, "convdiff9", 23), (4, "convdiff9", 23), (8, "convdiff9", 23), (16, "convdiff9", 23),
    (2, "poisson44", 10), (16, "poisson44", 10), (16, "poisson90", 30)])
@pytest.mark.parametrize("ortho", ["mgs", "bcgs"])
def test_gmres_resident_cluster_sizes(env, monkeypatch, ncl, mat, m, ortho):
    """The shared-memory path on each cluster size and rows-per-thread count
    (convdiff9, n = 729: 365 / 183 / 92 / 46 rows per CTA, 4 / 2 / 1 / 1 rows
    per thread; poisson44, n = 1936: 968 rows per CTA, 8 per thread, or 121;
    poisson90, n = 8100: 507 rows per CTA, 4 per thread, near the shared-
    memory limit; the last CTA holds fewer rows than the others), both
    Gram-Schmidt forms, against the oracle's GMRES with the same
    orthogonalisation."""
    xb, dev = env
    monkeypatch.setenv("XB_RESIDENT_CL", str(ncl))
    A = {"convdiff9": lambda: gen.convdiff3d(N=9), "poisson44": lambda: gen.poisson2d(44),
         "poisson90": lambda: gen.poisson2d(90)}[mat]()
    oc = xb.ORTHO_MGS if ortho == "mgs" else xb.ORTHO_BCGS
    info, x, b = _solve(xb, dev, A, "gmres", m=m, tol=1e-10, ortho=oc, maxiter=20000)
    xo, io = oracle.gmres(A, b, m=m, tol=1e-10, maxiter=20000,
                          ortho=oracle.MGS if ortho == "mgs" else oracle.BCGS)
    assert info["persistent"] == 2 and info["status"] == 0, info
    assert _true_rel(A, x, b) <= 1e-10
    assert abs(info["iters"] - io["iters"]) <= max(3, 0.05 * io["iters"]), (info["iters"], io["iters"])
    assert np.linalg.norm(x - xo) <= 1e-7 * np.linalg.norm(xo)


@pytest.mark.parametrize("ortho", ["mgs", "bcgs"])
def test_gmres_resident_is_repeatable(env, monkeypatch, ortho):
    """The shared-memory path sums in one fixed order whatever the timing of
    the exchanges, so repeated solves give the same iterate bit for bit."""
    xb, dev = env
    monkeypatch.delenv("XB_RESIDENT_CL", raising=False)
    A = gen.poisson2d(64)
    oc = xb.ORTHO_MGS if ortho == "mgs" else xb.ORTHO_BCGS
    runs = [_solve(xb, dev, A, "gmres", m=30, tol=1e-8, ortho=oc) for _ in range(4)]
    assert all(i["persistent"] == 2 and i["status"] == 0 for i, _, _ in runs)
    assert len({i["iters"] for i, _, _ in runs}) == 1
    for _, x, _ in runs[1:]:
        np.testing.assert_array_equal(x, runs[0][1])


def test_gmres_resident_fault_convergence_and_time_budget(env, monkeypatch):
    """The shared-memory path's true-residual check after an implicit
    convergence claim (Sec. 3.3.2: at tol 1e-14 the oracle claims once too
    early and narrows its threshold) and its time budget (a deadline the
    first restart check already sees ends the solve with XB_ENOCONV)."""
    xb, dev = env
    monkeypatch.delenv("XB_RESIDENT_CL", raising=False)
    A = gen.poisson2d(64)
    info, x, b = _solve(xb, dev, A, "gmres", m=30, tol=1e-14, maxiter=20000, ortho=xb.ORTHO_MGS)
    _, io = oracle.gmres(A, b, m=30, tol=1e-14, maxiter=20000)
    assert io["faults"] >= 1
    assert info["persistent"] == 2 and info["status"] == 0, info
    assert _true_rel(A, x, b) <= 1e-14
    assert abs(info["iters"] - io["iters"]) <= max(3, 0.05 * io["iters"]), (info["iters"], io["iters"])
    info, x, b = _solve(xb, dev, A, "gmres", m=30, tol=1e-8, maxtime_s=1e-6)
    assert info["persistent"] == 2 and info["status"] == xb.XB_ENOCONV, info
    assert info["iters"] <= 30


def test_gmres_resident_cta_without_rows_and_tiny_systems(env, monkeypatch):
    """A cluster CTA that owns no rows still takes part in every exchange
    (n = 130 on 16 CTAs: 9 rows per CTA, the last CTA none); a 1 x 1 system
    and a 2 x 2 one converge in one and two steps."""
    xb, dev = env
    monkeypatch.setenv("XB_RESIDENT_CL", "16")
    A = gen.laplace1d(130)
    info, x, b = _solve(xb, dev, A, "gmres", m=30, tol=1e-10, maxiter=5000)
    _, io = oracle.gmres(A, b, m=30, tol=1e-10, maxiter=5000)
    assert info["persistent"] == 2 and info["status"] == 0, info
    assert _true_rel(A, x, b) <= 1e-10
    assert abs(info["iters"] - io["iters"]) <= max(3, 0.05 * io["iters"]), (info["iters"], io["iters"])
    monkeypatch.delenv("XB_RESIDENT_CL")
    one = dict(n=1, nnz=1, rowptr=np.array([0, 1], np.int32), col=np.array([0], np.int32),
               val=np.array([3.0]), sym_upper=False)
    info, x, b = _solve(xb, dev, one, "gmres", b=np.array([6.0]))
    assert info["persistent"] == 2 and info["status"] == 0 and info["iters"] == 1
    np.testing.assert_allclose(x, [2.0], rtol=1e-15)
    two = dict(n=2, nnz=3, rowptr=np.array([0, 2, 3], np.int32), col=np.array([0, 1, 1], np.int32),
               val=np.array([2.0, 1.0, 3.0]), sym_upper=False)
    info, x, b = _solve(xb, dev, two, "gmres", b=np.array([3.0, 3.0]), tol=1e-12)
    assert info["persistent"] == 2 and info["status"] == 0 and info["iters"] <= 2
    np.testing.assert_allclose(x, [1.0, 1.0], rtol=1e-12)


def test_gmres_resident_declines_long_rows(env, monkeypatch):
    """Rows longer than 64 entries do not take the shared-memory path: the
    batched kernel runs the system instead."""
    xb, dev = env
    monkeypatch.delenv("XB_RESIDENT_CL", raising=False)
    A = gen.powerlaw(n=3000, seed=9)
    assert np.diff(A["rowptr"]).max() > 64
    info, x, b = _solve(xb, dev, A, "gmres", m=30, tol=TOL, maxiter=20000)
    assert info["persistent"] == 1 and info["status"] == 0
    assert _true_rel(A, x, b) <= TOL
    # rows longer than 1024 entries: summed by the whole cluster CTA
    A = gen.poisson2d_dense_rows(60, count=3, length=1500, seed=1)
    info, x, b = _solve(xb, dev, A, "gmres", m=30, tol=TOL, maxiter=20000)
    _, io = oracle.gmres(A, b, m=30, tol=TOL)
    assert info["persistent"] == 1 and info["status"] == 0
    assert _true_rel(A, x, b) <= TOL
    assert abs(info["iters"] - io["iters"]) <= max(3, 0.05 * io["iters"]), (info["iters"], io["iters"])


@pytest.mark.parametrize("name,make", [
    ("convdiff12", lambda: gen.convdiff3d(N=12)),
    ("powerlaw3000", lambda: gen.powerlaw(n=3000, seed=9)),
    ("random200", lambda: gen.random200()),
])
def test_bicgstab_matches_oracle(env, name, make):
    xb, dev = env
    A = make()
    info, x, b = _solve(xb, dev, A, "bicgstab", tol=TOL, maxiter=200000)
    xo, io = oracle.bicgstab(A, b, tol=TOL, maxiter=200000)
    assert info["status"] == 0, info
    assert _true_rel(A, x, b) <= TOL
    assert abs(info["iters"] - io["iters"]) <= max(3, 0.10 * io["iters"]), (info["iters"], io["iters"])


def test_bicgstab_limits(env):
    xb, dev = env
    A = gen.poisson2d(20)
    n = A["n"]
    info, x, _ = _solve(xb, dev, A, "bicgstab", b=np.zeros(n), x0=np.ones(n))
    assert info["status"] == 0 and np.all(x == 0)
    info, x, b = _solve(xb, dev, A, "bicgstab", tol=1e-14, maxiter=3)
    assert info["status"] == xb.XB_ENOCONV and info["iters"] == 3


@pytest.mark.parametrize("name,make", [
    ("poisson64", lambda: gen.poisson2d(64)),
    ("convdiff16", lambda: gen.convdiff3d(N=16)),
    ("random200", lambda: gen.random200()),
])
def test_mixed_refinement_reaches_fp64(env, name, make):
    """Plain refinement (ir_fallback = 0) against the oracle's loop: same
    number of refinement steps (within one: the FP32 inner solves round
    differently), both true residuals <= tol, no FP64 hand-over."""
    xb, dev = env
    A = make()
    info, x, b = _solve(xb, dev, A, "gmres", m=30, tol=TOL, precision=xb.PREC_MIXED,
                        tol_inner=1e-4, ir_fallback=0)
    assert info["status"] == 0, info
    assert info["fallback"] == 0 and info["iters"] == 0
    rel = _true_rel(A, x, b)
    assert rel <= TOL
    assert info["outer"] >= 2
    xo, io = oracle.gmres_ir(A, b, m=30, tol=TOL, tol_in=1e-4)
    assert io["status"] == 0
    assert abs(info["outer"] - io["outer"]) <= 1, (info["outer"], io["outer"])
    # both solutions solve the system to the same accuracy class
    assert np.linalg.norm(x - xo) <= 1e-4 * np.linalg.norm(xo)


def test_mixed_refinement_fallback_continues_as_fp64_gmres(env):
    """The library's safeguard (ir_fallback = 1, not part of the method):
    with one inner Arnoldi step per refinement step on a 32 x 32 Poisson
    matrix the residual ratios are ~0.46, ~0.71, ~0.82, so the third residual
    check sees two steps in a row that failed to halve it and the solve goes
    on as FP64 GMRES(30) from that x.  Checked against the oracle: three plain
    refinement steps, then the oracle's FP64 GMRES(30) from the resulting x;
    Arnoldi step counts within max(3, 5 %), both true residuals <= tol."""
    xb, dev = env
    A = gen.poisson2d(32)
    info, x, b = _solve(xb, dev, A, "gmres", m=30, tol=TOL, precision=xb.PREC_MIXED,
                        tol_inner=1e-4, maxiter_inner=1, ir_fallback=1)
    assert info["status"] == 0, info
    assert info["fallback"] == 1 and info["outer"] == 3 and info["inner_iters"] == 3, info
    assert _true_rel(A, x, b) <= TOL
    x3, i3 = oracle.gmres_ir(A, b, m=30, tol=TOL, tol_in=1e-4, maxit_in=1, max_outer=3)
    assert i3["outer"] == 3
    xo, io = oracle.gmres(A, b, x0=x3, m=30, tol=TOL)
    assert io["status"] == 0
    assert abs(info["iters"] - io["iters"]) <= max(3, 0.05 * io["iters"]), (info["iters"], io["iters"])
    # without the safeguard the same settings keep refining to max_outer
    info0, _, _ = _solve(xb, dev, A, "gmres", m=30, tol=TOL, precision=xb.PREC_MIXED,
                         tol_inner=1e-4, maxiter_inner=1, ir_fallback=0, max_outer=6)
    assert info0["status"] == -4 and info0["fallback"] == 0 and info0["outer"] == 6, info0


def test_dot_and_axpy(env):
    xb, dev = env
    import torch
    rng = np.random.default_rng(0)
    for n in (0, 1, 1000, 1_000_003):
        a, c = rng.standard_normal(n), rng.standard_normal(n)
        plan = xb.Plan.from_host(gen.poisson2d(4), dev)
        d = plan.dot(torch.tensor(a, device=dev), torch.tensor(c, device=dev)).item()
        ref = float(np.dot(a, c))
        assert abs(d - ref) <= 1e-13 * (np.abs(a) @ np.abs(c) + 1e-300)
        yt = torch.tensor(c, device=dev)
        xb.axpy(0.5, torch.tensor(a, device=dev), yt)
        np.testing.assert_allclose(yt.cpu().numpy(), c + 0.5 * a, rtol=1e-15, atol=1e-15)


def test_mgs_sweep_matches_oracle_arnoldi(env):
    """One MGS sweep (h_ij = (w, v_i); w -= h_ij v_i; h_{j+1,j} = ||w||) on the
    oracle's Arnoldi basis reproduces the oracle's Hessenberg column."""
    xb, dev = env
    import torch
    A = gen.poisson2d(20)
    m = 12
    v0 = np.random.default_rng(3).standard_normal(A["n"])
    k, V, H = oracle.arnoldi(A, v0, m)
    plan = xb.Plan.from_host(A, dev)
    for j in (0, 5, m - 1):
        w = torch.tensor(oracle.spmv(A, V[j]), device=dev)
        Vt = torch.tensor(V[: j + 1], device=dev)
        h = plan.mgs(Vt, w).cpu().numpy()
        np.testing.assert_allclose(h, H[: j + 2, j], rtol=1e-10, atol=1e-12)


def test_tuner_choice_is_valid_and_exact(env):
    xb, dev = env
    import torch
    A = gen.powerlaw(n=200000, seed=6)
    plan = xb.Plan.from_host(A, dev)
    ch = plan.tune()
    assert ch["variant"] in (0, 1, 2, 5) and ch["ms"] > 0  # a general-storage variant
    x = np.random.default_rng(1).uniform(-1, 1, A["n"])
    y = torch.empty(A["n"], dtype=torch.float64, device=dev)
    plan.spmv(torch.tensor(x, device=dev), y)
    from tests._gpu import assert_rows_close, row_bound
    assert_rows_close(y.cpu().numpy(), oracle.spmv(A, x), row_bound(A, x), what="tuned")
    U = gen.laplace3d(30, upper=True)
    pu = xb.Plan.from_host(U, dev)
    assert pu.tune()["variant"] in (3, 4)


def test_mm_ratio_and_dafrt_host(env):
    xb, dev = env
    assert xb.mm_ratio([1.0, 0.5, 0.25, 0.125, 0.0625], 5, 5) == 16.0
    assert xb.dafrt([1, 1, 1, 1, 1], 10.0) == 1
    assert xb.dafrt([1, 0.5, 0.25, 0.125, 0.0625], 10.0) == 0
