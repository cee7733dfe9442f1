"""GPU ILU(0) preconditioner (Sec. 4.3) against the CPU oracle: the factors
(same IKJ order per row; the device contracts a*b+c into FMAs, so entries
agree to rounding, 1e-11 relative to the row's largest factor), the two
substitutions (1e-10 of max |z|), and right-preconditioned GMRES and
BiCGStab (true residual <= 1e-8, iteration counts within max(3, 10 %)).
Both substitution paths run every case: the captured graph of level
launches (mode 0) and the persistent cooperative launch (mode 1); a test
makes the persistent path's bounded barrier wait run out."""
import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen
from tests._gpu import lib_and_device

pytestmark = pytest.mark.gpu
MATS = [("random200", gen.random200), ("poisson30", lambda: gen.poisson2d(30)),
        ("convdiff12", lambda: gen.convdiff3d(N=12)),
        ("powerlaw3000", lambda: gen.powerlaw(n=3000, seed=9)),
        ("powerlaw20k", lambda: gen.powerlaw(n=20000, seed=2))]


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name,make", MATS)
def test_factors_and_apply_match_oracle(env, name, make, mode):
    xb, dev = env
    import torch
    A = make()
    lu_o, st = oracle.ilu0(A)
    assert st == 0
    plan = xb.Plan.from_host(A, dev)
    plan.ilu0_config(mode)
    lu = plan.ilu0_factors().cpu().numpy()
    rp = A["rowptr"]
    for i in range(A["n"]):
        a, b = rp[i], rp[i + 1]
        scale = np.max(np.abs(lu_o[a:b]))
        assert np.max(np.abs(lu[a:b] - lu_o[a:b])) <= 1e-11 * scale, i
    r = np.random.default_rng(1).standard_normal(A["n"])
    z = plan.ilu0_apply(torch.tensor(r, device=dev),
                        torch.empty(A["n"], dtype=torch.float64, device=dev)).cpu().numpy()
    zo = oracle.ilu0_solve(A, lu_o, r)
    assert np.max(np.abs(z - zo)) <= 1e-10 * np.max(np.abs(zo))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name,make", MATS)
@pytest.mark.parametrize("which", ["gmres", "bicgstab"])
def test_preconditioned_solvers_match_oracle(env, name, make, which, mode):
    xb, dev = env
    import torch
    A = make()
    b = oracle.spmv(A, np.ones(A["n"]))
    plan = xb.Plan.from_host(A, dev)
    plan.ilu0_config(mode)
    x = torch.zeros(A["n"], dtype=torch.float64, device=dev)
    fn = plan.gmres if which == "gmres" else plan.bicgstab
    info = fn(torch.tensor(b, device=dev), x, tol=1e-8, precond=xb.PRECOND_ILU0)
    xh = x.cpu().numpy()
    rel = np.linalg.norm(b - oracle.spmv(A, xh)) / np.linalg.norm(b)
    assert info["status"] == 0 and rel <= 1e-8, info
    ofn = oracle.gmres if which == "gmres" else oracle.bicgstab
    _, io = ofn(A, b, tol=1e-8, ilu=True)
    assert abs(info["iters"] - io["iters"]) <= max(3, 0.10 * io["iters"]), (info["iters"], io["iters"])


def test_ilu_argument_errors(env):
    xb, dev = env
    import torch
    with pytest.raises(xb.XbError):  # symmetric upper storage has no L part stored
        xb.Plan.from_host(gen.laplace3d(6, upper=True), dev).ilu0_setup()
    A = gen.poisson2d(10)
    plan = xb.Plan.from_host(A, dev)
    b = torch.ones(A["n"], dtype=torch.float64, device=dev)
    with pytest.raises(xb.XbError):  # FP64 only
        plan.gmres(b, torch.zeros_like(b), precond=xb.PRECOND_ILU0, precision=xb.PREC_MIXED)
    with pytest.raises(xb.XbError):
        plan.gmres(b, torch.zeros_like(b), precond=7)
    # a row without a stored diagonal
    Z = dict(n=2, nnz=3, rowptr=np.array([0, 1, 3], np.int32), col=np.array([1, 0, 1], np.int32),
             val=np.array([1.0, 1.0, 2.0]), sym_upper=False)
    with pytest.raises(xb.XbError) as e:
        xb.Plan.from_host(Z, dev).ilu0_setup()
    assert e.value.code == xb.XB_EBREAKDOWN


def test_persistent_barrier_wait_runs_out(env):
    """The persistent substitution's level barrier with a one-poll limit: a
    CTA that finds the barrier not yet released gives up, flags the error and
    returns, the rest return at their next barrier, and the host reports
    XB_ETIMEOUT (a bounded wait, no fault).  The plan stays usable: with the
    default limit the next application matches the oracle."""
    xb, dev = env
    import torch
    A = gen.poisson2d(40)  # 79 dependency levels per triangle
    plan = xb.Plan.from_host(A, dev)
    plan.ilu0_setup()
    r = np.random.default_rng(3).standard_normal(A["n"])
    rt = torch.tensor(r, device=dev)
    z = torch.empty_like(rt)
    plan.ilu0_config(1, barrier_polls=1)
    with pytest.raises(xb.XbError) as e:
        plan.ilu0_apply(rt, z)
    assert e.value.code == xb.XB_ETIMEOUT
    b = torch.tensor(oracle.spmv(A, np.ones(A["n"])), device=dev)
    for fn in (plan.gmres, plan.bicgstab):  # both stop at their next check of the flag
        info = fn(b, torch.zeros_like(b), tol=1e-8, precond=xb.PRECOND_ILU0, maxiter=2000)
        assert info["status"] == xb.XB_ETIMEOUT, info
        assert info["iters"] <= 60, info  # stopped early, not at maxiter
    plan.ilu0_config(1, barrier_polls=0)
    zo = oracle.ilu0_solve(A, oracle.ilu0(A)[0], r)
    z = plan.ilu0_apply(rt, z).cpu().numpy()
    assert np.max(np.abs(z - zo)) <= 1e-10 * np.max(np.abs(zo))


def test_ilu_config_rejects_bad_arguments(env):
    xb, dev = env
    plan = xb.Plan.from_host(gen.poisson2d(6), dev)
    for mode, polls in ((2, 0), (-2, 0), (0, -1)):
        with pytest.raises(xb.XbError):
            plan.ilu0_config(mode, polls)
