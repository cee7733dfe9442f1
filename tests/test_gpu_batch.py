"""Batched persistent GMRES(m) (one graph-captured launch for many uneven
systems) against the CPU oracle: every system reaches the true residual
tolerance, iteration counts agree with the oracle's GMRES(m), replays are
bit-identical, and the time budget ends the launch with a status, not a hang."""
import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen
from tests._gpu import lib_and_device

pytestmark = pytest.mark.gpu


def _systems(dev, specs):
    import torch
    out, mats = [], []
    for A, m, mode in specs:
        b = oracle.spmv(A, np.ones(A["n"]))
        out.append(dict(rowptr=torch.as_tensor(A["rowptr"], device=dev),
                        col=torch.as_tensor(A["col"], device=dev),
                        val=torch.as_tensor(A["val"], device=dev),
                        b=torch.tensor(b, device=dev),
                        x=torch.zeros(A["n"], dtype=torch.float64, device=dev), m=m, mode=mode))
        mats.append((A, b))
    return out, mats


SPECS = [
    (lambda: gen.poisson2d(130), 30, 0), (lambda: gen.powerlaw(n=20000, mean=20, sigma=0.6, seed=3), 30, 1),
    (lambda: gen.powerlaw(n=20000, mean=12, sigma=0.5, seed=8), 30, 0),
    (lambda: gen.laplace3d(28), 40, 0),
    (lambda: gen.poisson2d(40), 30, 0), (lambda: gen.poisson2d(33), 20, 1),
    (lambda: gen.laplace3d(12), 30, 0), (lambda: gen.convdiff3d(N=14), 10, 0),
    (lambda: gen.powerlaw(n=6000, mean=12, sigma=0.6, seed=4), 30, 1), (lambda: gen.powerlaw(n=3000, seed=5), 50, 0),
    (lambda: gen.random200(), 30, 0), (lambda: gen.poisson2d(8), 5, 1),
] * 3


@pytest.mark.parametrize("coop_min", ["16384", "1000000000"])
def test_batch_matches_oracle_and_replays(coop_min, monkeypatch):
    """coop_min 16384: the systems with n >= 16384 go to whole clusters
    (distributed-shared-memory reductions, cluster barriers); 1e9: every
    system to a single CTA."""
    monkeypatch.setenv("XB_BATCH_COOP_MIN_N", coop_min)
    xb, dev = lib_and_device()
    specs = [(f(), m, mode) for f, m, mode in SPECS]
    systems, mats = _systems(dev, specs)
    bt = xb.Batch(systems, tol=1e-8, maxiter=20000, maxtime_s=60.0)
    bt.run()
    res = bt.results()
    xs = [q["x"].cpu().numpy().copy() for q in systems]
    for (A, b), r, x, (_, m, mode) in zip(mats, res, xs, specs):
        assert r["status"] == 0, r
        rel = np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)
        assert rel <= 1e-8 and abs(r["res_true"] - rel) <= 1e-9
        _, io = oracle.gmres(A, b, m=m, tol=1e-8)
        assert abs(r["iters"] - io["iters"]) <= max(3, 0.05 * io["iters"]), (r, io["iters"])
        assert r["m"] == m and r["mode"] == mode
    # a replay of the captured graph (x restarts from 0) gives identical results
    bt.run()
    res2 = bt.results()
    for q, x, r, r2 in zip(systems, xs, res, res2):
        np.testing.assert_array_equal(q["x"].cpu().numpy(), x)
        assert r["iters"] == r2["iters"]


@pytest.mark.parametrize("coop_min", ["16384", "1000000000"])
def test_batch_long_rows_summed_by_the_cta(coop_min, monkeypatch):
    """Mode 1 with rows longer than 1024 entries: the CTA (or each CTA of a
    cluster, for the long rows in its slice) sums them after its warp blocks;
    the solves match the oracle and replays are bit-identical."""
    monkeypatch.setenv("XB_BATCH_COOP_MIN_N", coop_min)
    xb, dev = lib_and_device()
    specs = [(gen.poisson2d_dense_rows(60, count=3, length=1500, seed=1), 30, 1),
             (gen.poisson2d_dense_rows(130, count=5, length=3000, seed=3), 30, 1),
             (gen.poisson2d_dense_rows(45, count=2, length=1100, seed=5), 20, 1)]
    assert all(np.diff(A["rowptr"]).max() > 1024 for A, _, _ in specs)
    systems, mats = _systems(dev, specs)
    bt = xb.Batch(systems, tol=1e-8, maxiter=20000, maxtime_s=60.0)
    bt.run()
    res = bt.results()
    xs = [q["x"].cpu().numpy().copy() for q in systems]
    for (A, b), r, x, (_, m, _) in zip(mats, res, xs, specs):
        assert r["status"] == 0, r
        rel = np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)
        assert rel <= 1e-8
        _, io = oracle.gmres(A, b, m=m, tol=1e-8)
        assert abs(r["iters"] - io["iters"]) <= max(3, 0.05 * io["iters"]), (r, io["iters"])
    bt.run()
    for q, x in zip(systems, xs):
        np.testing.assert_array_equal(q["x"].cpu().numpy(), x)


def test_batch_restart_rule_grows_m(monkeypatch):
    """With the MM-ratio rule on, a stagnating GMRES(5) grows its restart
    length at run time (Eq. 1, Sec. 4.3) and still converges; the same
    system from the cluster path and the single-CTA path agrees."""
    monkeypatch.setenv("XB_BATCH_COOP_MIN_N", "16384")
    xb, dev = lib_and_device()
    specs = [(gen.poisson2d(140), 5, 0), (gen.poisson2d(60), 5, 0)]
    systems, mats = _systems(dev, specs)
    bt = xb.Batch(systems, tol=1e-8, maxiter=200000, maxtime_s=60.0, dafrt=1, m_max=60,
                  dafrt_theta=10.0)
    bt.run()
    res = bt.results()
    for (A, b), r, q in zip(mats, res, systems):
        assert r["status"] == 0 and r["m"] > 5, r
        x = q["x"].cpu().numpy()
        assert np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b) <= 1e-8


def test_batch_time_budget_returns_status():
    xb, dev = lib_and_device()
    systems, _ = _systems(dev, [(gen.poisson2d(150), 5, 0)] * 4)
    bt = xb.Batch(systems, tol=1e-14, maxiter=10 ** 7, maxtime_s=0.05)
    bt.run()
    res = bt.results()
    assert all(r["status"] == xb.XB_ENOCONV for r in res)


def test_batch_empty_and_bad_args():
    xb, dev = lib_and_device()
    bt = xb.Batch([])
    bt.run()
    assert bt.results() == []
    systems, _ = _systems(dev, [(gen.poisson2d(5), 0, 0)])
    with pytest.raises(xb.XbError):
        xb.Batch(systems)


@pytest.mark.parametrize("coop_min", ["16384", "1000000000"])
@pytest.mark.parametrize("ortho", [3, 4])
def test_batch_bcgs_matches_oracle(coop_min, ortho, monkeypatch):
    """BCGS with block length 4 inside the batched launch (explicitly, and as
    the accuracy policy's choice at tol 1e-8): every system reaches the true
    residual and the oracle's BCGS GMRES(m) iteration count within
    max(3, 5 %), on the cluster and the single-CTA paths."""
    monkeypatch.setenv("XB_BATCH_COOP_MIN_N", coop_min)
    xb, dev = lib_and_device()
    specs = [(f(), m, mode) for f, m, mode in SPECS[:12]]
    systems, mats = _systems(dev, specs)
    bt = xb.Batch(systems, tol=1e-8, maxiter=20000, maxtime_s=60.0, ortho=ortho)
    bt.run()
    res = bt.results()
    for (A, b), r, q, (_, m, _) in zip(mats, res, systems, specs):
        assert r["status"] == 0, r
        x = q["x"].cpu().numpy()
        assert np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b) <= 1e-8
        _, io = oracle.gmres(A, b, m=m, tol=1e-8, ortho=oracle.BCGS)
        assert abs(r["iters"] - io["iters"]) <= max(3, 0.05 * io["iters"]), (r, io["iters"])


def test_batch_rejects_unsupported_orthogonalisation():
    xb, dev = lib_and_device()
    systems, _ = _systems(dev, [(gen.poisson2d(5), 5, 0)])
    for o in (1, 2):
        with pytest.raises(xb.XbError):
            xb.Batch(systems, ortho=o)
