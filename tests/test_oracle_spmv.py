"""Pins for the oracle's SpMV routines against facts outside the oracle:
numpy dense products, closed-form Laplacian eigenpairs, the symmetric-storage
identity, and hand-checked edge cases (CRS of Sec. 4.2; SpMV of Sec. 3.2.2)."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_01599_gb300 import gen


def _norm_err(y, yref, A, x):
    """max_i |y_i - yref_i| / sum_j |a_ij||x_j| (row-normalised error)."""
    D = np.abs(gen.to_dense(A))
    s = D @ np.abs(x)
    s[s == 0] = 1.0
    return np.max(np.abs(y - yref) / s)


def test_spmv_random200_vs_dense_bitexact():
    # config-1 companion matrix: 200 rows, 5 random off-diagonals U[-1,1] + diag 10
    A = gen.random200()
    assert A["n"] == 200 and A["nnz"] == 1200
    x = np.random.default_rng(11).uniform(-1, 1, 200)
    D = gen.to_dense(A)
    # same ascending-column order on both sides -> identical rounding
    np.testing.assert_array_equal(oracle.spmv(A, x), oracle.dense_matvec(D, x))
    # against numpy's own (BLAS) product: equal up to reassociation
    assert _norm_err(oracle.spmv(A, x), D @ x, A, x) <= 1e-14


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (2.5, 0.0), (-1.0, 1.0), (0.5, -3.0), (0.0, 2.0)])
def test_spmv_alpha_beta(alpha, beta):
    A = gen.random200(seed=7)
    rng = np.random.default_rng(3)
    x, y0 = rng.standard_normal(200), rng.standard_normal(200)
    D = gen.to_dense(A)
    ref = alpha * (D @ x) + beta * y0
    got = oracle.spmv(A, x, alpha, beta, y0)
    assert np.max(np.abs(got - ref)) <= 1e-12 * (1 + np.max(np.abs(ref)))


def test_spmv_beta_zero_ignores_y():
    A = gen.random200()
    y0 = np.full(200, np.nan)
    assert np.all(np.isfinite(oracle.spmv(A, np.ones(200), 1.0, 0.0, y0)))


@pytest.mark.parametrize("n", [1, 2, 7, 50, 257])
def test_laplace1d_eigenpairs(n):
    A = gen.laplace1d(n)
    i = np.arange(1, n + 1)
    for k in {1, (n + 1) // 2, n}:
        v = np.sin(i * k * math.pi / (n + 1))
        lam = 2.0 - 2.0 * math.cos(k * math.pi / (n + 1))
        r = oracle.spmv(A, v) - lam * v
        # the sines themselves carry ~eps*argument error (arguments up to k*pi)
        assert np.max(np.abs(r)) <= 64 * 2.2e-16 * (1 + k * math.pi) * np.max(np.abs(v))


@pytest.mark.parametrize("N", [3, 16, 64])
def test_poisson2d_eigenpairs(N):
    A = gen.poisson2d(N)
    assert A["nnz"] == 5 * N * N - 4 * N
    h = math.pi / (N + 1)
    ix = np.arange(1, N + 1)
    for j, k in [(1, 1), (2, N), (N // 2 + 1, 3)]:
        v = np.outer(np.sin(ix * k * h), np.sin(ix * j * h)).ravel()  # x fastest
        lam = 4.0 - 2.0 * math.cos(j * h) - 2.0 * math.cos(k * h)
        r = oracle.spmv(A, v) - lam * v
        assert np.max(np.abs(r)) <= 64 * 2.2e-16 * (1 + N * math.pi) * np.max(np.abs(v))


def test_laplace3d_eigenpair_and_rowsums():
    N = 9
    A = gen.laplace3d(N)
    assert A["nnz"] == 7 * N ** 3 - 6 * N * N
    h = math.pi / (N + 1)
    s = np.sin(np.arange(1, N + 1) * h)
    s2 = np.sin(np.arange(1, N + 1) * 2 * h)
    v = np.einsum("z,y,x->zyx", s, s2, s).ravel()
    lam = 6.0 - 4.0 * math.cos(h) - 2.0 * math.cos(2 * h)
    assert np.max(np.abs(oracle.spmv(A, v) - lam * v)) <= 1e-13
    # A*ones = number of missing neighbours (non-zero only on the boundary)
    g = np.indices((N, N, N))
    missing = sum(((g[a] == 0).astype(int) + (g[a] == N - 1).astype(int)) for a in range(3))
    np.testing.assert_array_equal(oracle.spmv(A, np.ones(N ** 3)), missing.ravel().astype(float))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sym_upper_equals_full(seed):
    U = gen.random_sym_upper(120, per_row=5, seed=seed)
    F = gen.full_from_upper(U)
    x = np.random.default_rng(seed + 10).uniform(-1, 1, 120)
    ys = oracle.spmv(U, x)
    yf = oracle.spmv(F, x)
    assert _norm_err(ys, yf, F, x) <= 1e-14
    # and both against numpy on the dense symmetric matrix
    D = gen.to_dense(U)
    np.testing.assert_array_equal(D, D.T)
    assert _norm_err(ys, D @ x, F, x) <= 1e-14


def test_sym_upper_stencil_equals_full():
    U = gen.laplace3d(12, upper=True)
    F = gen.laplace3d(12)
    assert U["nnz"] == (F["nnz"] + F["n"]) // 2
    x = np.random.default_rng(5).standard_normal(F["n"])
    assert np.max(np.abs(oracle.spmv(U, x) - oracle.spmv(F, x))) <= 1e-13


def test_sym_alpha_beta():
    U = gen.random_sym_upper(40, seed=4)
    D = gen.to_dense(U)
    rng = np.random.default_rng(0)
    x, y0 = rng.standard_normal(40), rng.standard_normal(40)
    got = oracle.spmv(U, x, -2.0, 0.5, y0)
    np.testing.assert_allclose(got, -2.0 * (D @ x) + 0.5 * y0, rtol=0, atol=1e-12)


def test_edge_empty_rows_and_tiny():
    # rows 1 and 3 are empty; row 4 holds all remaining entries
    A = dict(n=5, nnz=6, rowptr=np.array([0, 1, 1, 2, 2, 6], np.int32),
             col=np.array([0, 2, 0, 1, 3, 4], np.int32),
             val=np.array([2.0, -1.0, 1.0, 1.0, 1.0, 1.0]), sym_upper=False)
    x = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    np.testing.assert_array_equal(oracle.spmv(A, x), [2.0, 0.0, -3.0, 0.0, 12.0])
    one = dict(n=1, nnz=1, rowptr=np.array([0, 1], np.int32), col=np.array([0], np.int32),
               val=np.array([3.0]), sym_upper=False)
    np.testing.assert_array_equal(oracle.spmv(one, np.array([2.0])), [6.0])
    zero = dict(n=3, nnz=0, rowptr=np.zeros(4, np.int32), col=np.zeros(0, np.int32),
                val=np.zeros(0), sym_upper=False)
    np.testing.assert_array_equal(oracle.spmv(zero, np.ones(3), 1.0, 2.0, np.ones(3)), [2.0] * 3)


def test_spmv_f32_accumulates_in_single():
    A = gen.poisson2d(8)
    x = np.random.default_rng(2).uniform(-1, 1, A["n"]).astype(np.float32)
    y = oracle.spmv_f32(A, x)
    assert y.dtype == np.float32
    yd = gen.to_dense(A) @ x.astype(np.float64)
    # 5-term rows: at most 5 roundings of relative size 2^-24 each
    assert np.max(np.abs(y - yd)) <= 5 * 2.0 ** -24 * 8 * 1.0


def test_powerlaw_recipe_properties():
    A = gen.powerlaw(n=20000, seed=3)
    rp, col, val = A["rowptr"], A["col"], A["val"]
    L = np.diff(rp) - 1
    assert L.min() >= 1 and L.max() <= 19999
    # arithmetic mean of the lognormal row lengths ~12 (sample tolerance)
    assert 10.0 < L.mean() < 14.0
    for i in [0, 17, 5000, 19999]:
        c = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0) and i in c
        v = val[rp[i]:rp[i + 1]]
        d = v[c == i][0]
        assert d == pytest.approx(2.0 * np.abs(v[c != i]).sum(), rel=1e-12)


def test_openmp_build_matches_the_plain_oracle():
    """The benchmark's all-cores baseline runs the OpenMP build of the same
    source: its row-parallel SpMV keeps each row's summation order (bit for
    bit), and its solvers, whose dot products sum in per-thread pieces, reach
    the same iteration counts on a well-conditioned problem."""
    A = gen.powerlaw(n=20000, seed=3)
    x = np.random.default_rng(1).uniform(-1, 1, A["n"])
    np.testing.assert_array_equal(oracle.spmv(A, x, omp=True), oracle.spmv(A, x))
    P = gen.poisson2d(40)
    b = oracle.spmv(P, np.ones(P["n"]))
    _, i1 = oracle.gmres(P, b, m=30, tol=1e-8)
    _, i2 = oracle.gmres(P, b, m=30, tol=1e-8, omp=True)
    assert abs(i1["iters"] - i2["iters"]) <= 3 and i2["res_true"] <= 1e-8
    assert oracle.lib_omp().orc_num_threads() >= 1
