"""GPU parity of every SpMV kernel against the CPU oracle, through the C ABI.

Tolerance (per row): |y_gpu - y_oracle| <= 1e-12 * sum_j |a_ij||x_j|
(FP64); rows whose scale is zero must match exactly.  Matrices span many
tiles/segments with ragged tails, plus the degenerate shapes (empty rows,
n = 1, nnz = 0, one row holding most entries, rows of length 31/32/33...).
"""
import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen
from tests._gpu import assert_rows_close, lib_and_device, row_bound, sampled_rows_oracle

pytestmark = pytest.mark.gpu

GENERAL = {
    "row": (0, [(64, 1), (256, 1)]),
    "nnz": (1, [(64, 4), (128, 4), (256, 8), (512, 16), (128, 16)]),
    "segscan": (2, [(64, 4), (128, 4), (256, 8), (128, 16), (256, 16), (128, 32)]),
    "sell": (5, [(64, 1), (256, 1), (128, 8), (512, 32)]),
    "bcsr": (8, [(128, 2), (256, 3), (64, 4)]),
}


def bcsr_accepts(A, r):
    """The BCSR copy is built unless its r x r blocks hold more than 2 nnz +
    16 r entries (blocks = distinct column blocks of each block row)."""
    rp = np.asarray(A["rowptr"], np.int64)
    col = np.asarray(A["col"], np.int64)
    n = A["n"]
    nb = sum(np.unique(col[rp[b * r]:rp[min(n, b * r + r)]] // r).size
             for b in range((n + r - 1) // r))
    return nb * r * r <= 2 * A["nnz"] + 16 * r


def sell_accepts(A, sigma):
    """The SELL-32-sigma copy is built unless its padding exceeds 3 nnz + 32
    per slice (the format's definition: rows sorted by length inside windows
    of sigma rows, slices of 32 as wide as their longest row)."""
    L = np.diff(np.asarray(A["rowptr"], np.int64))
    n = A["n"]
    order = np.concatenate([w0 + np.argsort(-L[w0:w0 + sigma], kind="stable")
                            for w0 in range(0, n, sigma)]) if n else np.zeros(0, np.int64)
    Ls = np.zeros(((n + 31) // 32) * 32, np.int64)
    Ls[:n] = L[order]
    total = 32 * Ls.reshape(-1, 32).max(axis=1).sum() if n else 0
    return total <= 3 * A["nnz"] + 32 * ((n + 31) // 32)


def _adversarial():
    rng = np.random.default_rng(42)
    n = 6000
    L = rng.choice([0, 0, 1, 2, 5, 31, 32, 33, 63, 64, 65, 127, 129], size=n)
    L[17] = 2047
    L[18] = 2048
    L[19] = 2049
    L[3000] = 5999  # a full row
    L[-40:] = 0     # ragged empty tail
    L[:5] = 0       # empty head
    return gen.random_general(n, L, seed=7)


def _one_huge_row():
    n = 30000
    L = np.zeros(n, np.int64)
    L[n // 2] = n - 1
    L[::97] = 3
    return gen.random_general(n, L, seed=8)


MATS = {
    "random200": lambda: gen.random200(),
    "poisson64": lambda: gen.poisson2d(64),
    "laplace3d_20": lambda: gen.laplace3d(20),
    "convdiff12": lambda: gen.convdiff3d(N=12),
    "powerlaw30k": lambda: gen.powerlaw(n=30000, seed=3),
    "block3d_10_dof3": lambda: gen.block_stencil3d(10, 3),
    "block3d_7_dof2": lambda: gen.block_stencil3d(7, 2),
    "adversarial": _adversarial,
    "one_huge_row": _one_huge_row,
    "n1": lambda: dict(n=1, nnz=1, rowptr=np.array([0, 1], np.int32), col=np.array([0], np.int32),
                       val=np.array([2.5]), sym_upper=False),
    "empty": lambda: dict(n=7, nnz=0, rowptr=np.zeros(8, np.int32), col=np.zeros(0, np.int32),
                          val=np.zeros(0), sym_upper=False),
}


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


@pytest.mark.parametrize("mname", list(MATS))
def test_general_variants_match_oracle(env, mname):
    xb, dev = env
    import torch
    A = MATS[mname]()
    n = A["n"]
    plan = xb.Plan.from_host(A, dev)
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, n)
    y0 = rng.uniform(-1, 1, n)
    xt = torch.tensor(x, device=dev)
    for alpha, beta in [(1.0, 0.0), (-0.75, 0.0), (1.5, -2.0)]:
        yref = oracle.spmv(A, x, alpha, beta, y0)
        bound = row_bound(A, x, alpha, beta, y0)
        for vname, (v, shapes) in GENERAL.items():
            for block, ipt in shapes:
                y = torch.tensor(y0, device=dev) if beta != 0 else torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
                if ((v == xb.VAR_SELL and not sell_accepts(A, 32 * ipt)) or
                        (v == xb.VAR_BCSR and not bcsr_accepts(A, ipt))):
                    with pytest.raises(xb.XbError):
                        plan.spmv(xt, y, alpha=alpha, beta=beta, variant=v, block=block, ipt=ipt)
                    continue
                plan.spmv(xt, y, alpha=alpha, beta=beta, variant=v, block=block, ipt=ipt)
                assert_rows_close(y.cpu().numpy(), yref, bound,
                                  what=f"{mname}/{vname}/b{block}i{ipt}/a{alpha}b{beta}")


def test_named_entry_points(env):
    xb, dev = env
    import torch
    A = gen.powerlaw(n=20000, seed=11)
    plan = xb.Plan.from_host(A, dev)
    x = np.random.default_rng(2).uniform(-1, 1, A["n"])
    yref = oracle.spmv(A, x)
    bound = row_bound(A, x)
    xt = torch.tensor(x, device=dev)
    for fn in (plan.spmv_crs, plan.spmv_segscan):
        y = torch.empty(A["n"], dtype=torch.float64, device=dev)
        fn(xt, y)
        assert_rows_close(y.cpu().numpy(), yref, bound, what=fn.__name__)
    with pytest.raises(xb.XbError):
        plan.spmv_sym(xt, torch.empty_like(xt))


def test_segscan_deterministic(env):
    xb, dev = env
    import torch
    A = gen.powerlaw(n=50000, seed=5)
    plan = xb.Plan.from_host(A, dev)
    xt = torch.tensor(np.random.default_rng(3).standard_normal(A["n"]), device=dev)
    ys = []
    for _ in range(3):
        y = torch.empty_like(xt)
        plan.spmv_segscan(xt, y)
        ys.append(y.cpu().numpy())
    np.testing.assert_array_equal(ys[0], ys[1])
    np.testing.assert_array_equal(ys[0], ys[2])


def _arrow(U):
    """Upper storage plus a dense last column (every row couples to row n-1):
    all lanes of a warp send a transpose term to the same row, the case the
    warp-aggregated atomics combine."""
    n = U["n"]
    rp = np.asarray(U["rowptr"], np.int64)
    rows, cols, vals = [], [], []
    for i in range(n):
        a, b = rp[i], rp[i + 1]
        c = list(U["col"][a:b])
        v = list(U["val"][a:b])
        if i < n - 1 and c[-1] != n - 1:
            c.append(n - 1)
            v.append(0.01)
        rows.append(len(c))
        cols += c
        vals += v
    rp2 = np.concatenate([[0], np.cumsum(rows)])
    return dict(n=n, nnz=int(rp2[-1]), rowptr=rp2.astype(np.int32), col=np.array(cols, np.int32),
                val=np.array(vals), sym_upper=True)


def _sym_long_row():
    n = 4000
    U = gen.random_sym_upper(n, per_row=3, seed=21)
    # add a dense first row (columns 0..n-1) by bookkeeping on the CRS arrays
    rp, col, val = U["rowptr"].astype(np.int64), U["col"], U["val"]
    first_cols = np.arange(n)
    first_vals = np.random.default_rng(5).uniform(-1, 1, n)
    first_vals[0] = 4.0 * n
    rest = slice(rp[1], rp[-1])
    col2 = np.concatenate([first_cols, col[rest]])
    val2 = np.concatenate([first_vals, val[rest]])
    rp2 = np.concatenate([[0], rp[1:] - rp[1] + n])
    return dict(n=n, nnz=int(rp2[-1]), rowptr=rp2.astype(np.int32), col=col2.astype(np.int32),
                val=val2, sym_upper=True)


def s3_accepts(U, block, ipt):
    """The S3 layout exists unless some tile (at most `block` rows and
    block*ipt entries, a longer row alone) reaches more than 8 granules of 256
    rows beyond its last row."""
    rp = np.asarray(U["rowptr"], np.int64)
    col = np.asarray(U["col"], np.int64)
    n = U["n"]
    r = 0
    while r < n:
        r1 = r + 1
        if rp[r + 1] - rp[r] <= block * ipt:
            while r1 < n and r1 - r < block and rp[r1 + 1] - rp[r] <= block * ipt:
                r1 += 1
        c = col[rp[r]:rp[r1]]
        if np.unique(c[c >= r1] // 256).size > 8:
            return False
        r = r1
    return True


SYM = {
    "laplace3d_20_upper": lambda: gen.laplace3d(20, upper=True),
    "laplace3d_24_upper_arrow": lambda: _arrow(gen.laplace3d(24, upper=True)),
    "randsym3000": lambda: gen.random_sym_upper(3000, per_row=6, seed=3),
    "sym_long_row": _sym_long_row,
    "poisson2d_50_upper": lambda: gen.poisson2d(50, upper=True),
}


@pytest.mark.parametrize("mname", list(SYM))
def test_sym_variants_match_oracle(env, mname):
    xb, dev = env
    import torch
    U = SYM[mname]()
    F = gen.full_from_upper(U)
    n = U["n"]
    plan = xb.Plan.from_host(U, dev)
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, n)
    y0 = rng.uniform(-1, 1, n)
    xt = torch.tensor(x, device=dev)
    for alpha, beta in [(1.0, 0.0), (2.0, 0.5)]:
        yref = oracle.spmv(U, x, alpha, beta, y0)
        bound = row_bound(F, x, alpha, beta, y0)
        # the symmetric-storage identity: oracle sym == oracle full
        assert_rows_close(oracle.spmv(F, x, alpha, beta, y0), yref, bound, what="oracle sym==full")
        for v, shapes in ((3, [(128, 1), (256, 1)]), (4, [(128, 4), (256, 8), (512, 16), (64, 1)]),
                          (6, [(128, 4), (256, 8), (512, 16), (64, 1)]), (7, [(64, 1), (256, 1)])):
            for block, ipt in shapes:
                y = torch.tensor(y0, device=dev)
                if v == 6 and not s3_accepts(U, block, ipt):
                    with pytest.raises(xb.XbError):
                        plan.spmv(xt, y, alpha=alpha, beta=beta, variant=v, block=block, ipt=ipt)
                    continue
                plan.spmv(xt, y, alpha=alpha, beta=beta, variant=v, block=block, ipt=ipt)
                assert_rows_close(y.cpu().numpy(), yref, bound, what=f"{mname}/v{v}/b{block}i{ipt}")
        y = torch.tensor(y0, device=dev)
        plan.spmv_sym(xt, y, alpha=alpha, beta=beta)
        assert_rows_close(y.cpu().numpy(), yref, bound, what=f"{mname}/spmv_sym")


def test_f32_path(env):
    xb, dev = env
    import torch
    for A in (gen.poisson2d(40), gen.powerlaw(n=8000, seed=2)):
        plan = xb.Plan.from_host(A, dev)
        x = np.random.default_rng(4).uniform(-1, 1, A["n"]).astype(np.float32)
        yo = oracle.spmv_f32(A, x)
        Aabs = dict(A)
        Aabs["val"] = np.abs(A["val"])
        bound = oracle.spmv(Aabs, np.abs(x.astype(np.float64)))
        k = np.diff(A["rowptr"]).astype(np.float64)
        for v in (0, 1, 2, 5):
            y = torch.empty(A["n"], dtype=torch.float32, device=dev)
            if v == xb.VAR_SELL:
                plan.set_choice(xb.VAR_SELL, 256, 32)  # SELL-32-1024 (FP32 values)
                if not sell_accepts(A, 1024):
                    continue
            plan.spmv_f32(torch.tensor(x, device=dev), y, variant=v)
            err = np.abs(y.cpu().numpy().astype(np.float64) - yo.astype(np.float64))
            assert np.all(err <= 2 * (k + 2) * 6e-8 * bound + 1e-30), v


def test_full_size_powerlaw_sampled(env):
    """Config-3 size (n = 4M, lognormal rows): the tuned launch shape and each
    general variant, checked on 3000 sampled rows that the oracle computes one
    by one, plus exact agreement between the deterministic variants' checksums."""
    xb, dev = env
    import torch
    A = gen.powerlaw(n=4_000_000, seed=3)
    plan = xb.Plan.from_host(A, dev)
    choice = plan.tune()
    x = np.random.default_rng(12).uniform(-1, 1, A["n"])
    xt = torch.tensor(x, device=dev)
    rows = np.sort(np.random.default_rng(13).choice(A["n"], 3000, replace=False))
    rows = np.unique(np.concatenate([rows, [0, A["n"] - 1], [int(np.argmax(np.diff(A["rowptr"])))]]))
    yref = sampled_rows_oracle(A, x, rows)
    S = {k: A[k] for k in A}
    Aabs = dict(A)
    Aabs["val"] = np.abs(A["val"])
    bound = sampled_rows_oracle(Aabs, np.abs(x), rows)
    for v, b, i in [(-1, 0, 0), (0, 256, 1), (1, 256, 8), (2, 256, 8), (2, 128, 16), (2, 256, 32)]:
        y = torch.empty_like(xt)
        plan.spmv(xt, y, variant=v, block=b, ipt=i)
        assert_rows_close(y.cpu().numpy()[rows], yref, bound, what=f"C3 v{v} b{b} i{i} ({choice})")


def test_full_size_sym_laplace128_sampled(env):
    """Config-2 size (128^3 Laplacian, upper storage): sym SpMV vs the oracle on
    sampled rows of the independently generated full-storage matrix."""
    xb, dev = env
    import torch
    U = gen.laplace3d(128, upper=True)
    plan = xb.Plan.from_host(U, dev)
    x = np.random.default_rng(5).uniform(-1, 1, U["n"])
    xt = torch.tensor(x, device=dev)
    F = gen.laplace3d(128)
    rows = np.unique(np.concatenate([np.random.default_rng(6).choice(U["n"], 3000, replace=False),
                                     [0, 127, 128 * 128, U["n"] - 1]]))
    yref = sampled_rows_oracle(F, x, rows)
    Fabs = dict(F)
    Fabs["val"] = np.abs(F["val"])
    bound = sampled_rows_oracle(Fabs, np.abs(x), rows)
    for v, b, i in [(3, 256, 1), (4, 256, 8), (4, 512, 4)]:
        y = torch.empty_like(xt)
        plan.spmv(xt, y, variant=v, block=b, ipt=i)
        assert_rows_close(y.cpu().numpy()[rows], yref, bound, what=f"C2 v{v}")


def test_features_match_oracle(env):
    xb, dev = env
    import torch
    for A in (gen.poisson2d(30), gen.powerlaw(n=5000, seed=1), gen.laplace3d(8, upper=True),
              gen.random200(), _adversarial()):
        raw_o, feat_o = oracle.features(A)
        t = [torch.as_tensor(A[k], device=dev) for k in ("rowptr", "col", "val")]
        raw_g, feat_g = xb.features(t[0].int(), t[1].int(), t[2].double(), A["sym_upper"])
        np.testing.assert_array_equal(raw_g[[0, 1, 4, 5, 6]], raw_o[[0, 1, 4, 5, 6]])
        np.testing.assert_allclose(raw_g[[2, 3]], raw_o[[2, 3]], rtol=1e-12)
        np.testing.assert_allclose(feat_g, feat_o, rtol=1e-6, atol=1e-6)


def test_bad_arguments_rejected(env):
    xb, dev = env
    import torch
    A = gen.poisson2d(8)
    plan = xb.Plan.from_host(A, dev)
    x = torch.ones(A["n"], dtype=torch.float64, device=dev)
    with pytest.raises(xb.XbError):
        plan.spmv(x, x)  # aliasing
    with pytest.raises(xb.XbError):
        plan.spmv(x, torch.empty_like(x), variant=3)  # sym variant on general storage
    with pytest.raises(xb.XbError):
        plan.spmv(x, torch.empty_like(x), variant=1, block=100)
    bad = dict(A)
    bad["rowptr"] = A["rowptr"].copy()
    bad["rowptr"][-1] += 1
    with pytest.raises(xb.XbError):
        xb.Plan.from_host(bad, dev)


def test_sell_layout_and_solvers(env):
    """Format conversion (SELL-32-sigma): bit-identical to the thread-per-row
    CRS kernel (same summation order, padding never read); a padding-heavy
    matrix is rejected at sigma = 32 and accepted at sigma = 1024; GMRES in
    FP64 and mixed precision run on the SELL copy and meet tol."""
    xb, dev = env
    import torch
    A = gen.convdiff3d(N=24)
    plan = xb.Plan.from_host(A, dev)
    xt = torch.tensor(np.random.default_rng(9).uniform(-1, 1, A["n"]), device=dev)
    y_row = torch.empty_like(xt)
    plan.spmv(xt, y_row, variant=xb.VAR_ROW, block=256, ipt=1)
    for ipt in (1, 8, 32):
        y = torch.empty_like(xt)
        plan.spmv(xt, y, variant=xb.VAR_SELL, block=256, ipt=ipt)
        assert torch.equal(y, y_row), ipt
    P = gen.powerlaw(n=3000, seed=1, cap=300)
    pp = xb.Plan.from_host(P, dev)
    assert not sell_accepts(P, 32) and sell_accepts(P, 1024)
    xp = torch.tensor(np.random.default_rng(3).uniform(-1, 1, P["n"]), device=dev)
    with pytest.raises(xb.XbError):
        pp.spmv(xp, torch.empty_like(xp), variant=xb.VAR_SELL, block=256, ipt=1)
    y = torch.empty_like(xp)
    pp.spmv(xp, y, variant=xb.VAR_SELL, block=256, ipt=32)
    y2 = torch.empty_like(xp)
    pp.spmv(xp, y2, variant=xb.VAR_ROW, block=256, ipt=1)
    assert torch.equal(y, y2)
    # solvers on the converted copy
    Q = gen.poisson2d(64)
    pq = xb.Plan.from_host(Q, dev)
    pq.set_choice(xb.VAR_SELL, 256, 32)
    b_h = oracle.spmv(Q, np.ones(Q["n"]))
    b = torch.tensor(b_h, device=dev)
    _, oinfo = oracle.gmres(Q, b_h, m=30, tol=1e-8)
    for prec in (xb.PREC_FP64, xb.PREC_MIXED):
        x = torch.zeros_like(b)
        info = pq.gmres(b, x, m=30, tol=1e-8, precision=prec)
        assert info["status"] == 0 and info["res_true"] <= 1e-8, (prec, info)
        assert info["variant_used"] == xb.VAR_SELL
        if prec == xb.PREC_FP64:
            assert abs(info["iters"] - oinfo["iters"]) <= max(3, 0.05 * oinfo["iters"])


def test_bcsr_is_bit_identical_to_row_kernel_and_solves(env):
    """BCSR adds its zero fill as fma(0, x, s) and walks columns in ascending
    order, so y equals the row kernel's bit for bit; GMRES runs on it in FP64
    and mixed precision; the exhaustive tuner may pick it."""
    xb, dev = env
    import torch
    A = gen.block_stencil3d(12, 3)
    plan = xb.Plan.from_host(A, dev)
    xt = torch.tensor(np.random.default_rng(3).uniform(-1, 1, A["n"]), device=dev)
    y_row = torch.empty_like(xt)
    plan.spmv(xt, y_row, variant=xb.VAR_ROW, block=256, ipt=1)
    for r in (2, 3, 4):
        y = torch.empty_like(xt)
        if not bcsr_accepts(A, r):  # 4 x 4 blocks over 3 x 3 node blocks: too much fill
            with pytest.raises(xb.XbError):
                plan.spmv(xt, y, variant=xb.VAR_BCSR, block=128, ipt=r)
            continue
        plan.spmv(xt, y, variant=xb.VAR_BCSR, block=128, ipt=r)
        assert torch.equal(y, y_row), r
    b_h = oracle.spmv(A, np.ones(A["n"]))
    b = torch.tensor(b_h, device=dev)
    _, oinfo = oracle.gmres(A, b_h, m=30, tol=1e-8)
    for prec in (xb.PREC_FP64, xb.PREC_MIXED):
        x = torch.zeros_like(b)
        info = plan.gmres(b, x, m=30, tol=1e-8, precision=prec, variant=xb.VAR_BCSR, block=128,
                          ipt=3, small_n=0)
        rel = np.linalg.norm(b_h - oracle.spmv(A, x.cpu().numpy())) / np.linalg.norm(b_h)
        assert info["status"] == 0 and rel <= 1e-8, info
        assert info["variant_used"] == xb.VAR_BCSR
        if prec == xb.PREC_FP64:
            assert abs(info["iters"] - oinfo["iters"]) <= max(3, 0.05 * oinfo["iters"])
    ch = plan.tune()
    assert ch["variant"] in (xb.VAR_ROW, xb.VAR_NNZ, xb.VAR_SEGSCAN, xb.VAR_SELL, xb.VAR_BCSR)
