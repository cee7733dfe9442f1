"""The dependency levels that schedule ILU(0) on the device (Sec. 4.3 runs the
solvers with ILU(0); the factorization and both substitutions go level by
level), host logic only: the library's levels against their definition
written out here, the property every level schedule needs (a row depends only
on rows of lower levels), and a missing diagonal as a breakdown."""
import numpy as np
import pytest

import paper_2405_01599_gb300 as xb
from paper_2405_01599_gb300 import gen


@pytest.fixture(scope="module")
def lib():
    try:
        return xb.lib()
    except ImportError:
        pytest.skip("CUDA library not built")


def definition(A):
    rp, ci, n = A["rowptr"], A["col"], A["n"]
    lev = [0] * n
    for i in range(n):
        lower = [lev[k] for k in ci[rp[i]:rp[i + 1]] if k < i]
        lev[i] = 1 + max(lower) if lower else 0
    ulev = [0] * n
    for i in reversed(range(n)):
        upper = [ulev[k] for k in ci[rp[i]:rp[i + 1]] if k > i]
        ulev[i] = 1 + max(upper) if upper else 0
    return np.array(lev), np.array(ulev)


MATS = {
    "poisson12": lambda: gen.poisson2d(12),
    "convdiff8": lambda: gen.convdiff3d(N=8),
    "random200": lambda: gen.random200(),
    "powerlaw2000": lambda: gen.powerlaw(n=2000, seed=4, cap=200),
    "tridiag": lambda: gen.laplace1d(50),
    "diagonal": lambda: dict(n=5, nnz=5, rowptr=np.arange(6), col=np.arange(5),
                             val=np.ones(5), sym_upper=False),
}


@pytest.mark.parametrize("mname", list(MATS))
def test_levels_match_definition(lib, mname):
    A = MATS[mname]()
    lev, ulev, (nl, nu) = xb.ilu_levels(A["rowptr"], A["col"])
    dl, du = definition(A)
    np.testing.assert_array_equal(lev, dl)
    np.testing.assert_array_equal(ulev, du)
    assert nl == dl.max() + 1 and nu == du.max() + 1
    rp, ci = A["rowptr"], A["col"]
    for i in range(A["n"]):
        for k in ci[rp[i]:rp[i + 1]]:
            if k < i:
                assert lev[k] < lev[i]
            elif k > i:
                assert ulev[k] < ulev[i]


def test_closed_forms(lib):
    # a tridiagonal matrix is a chain: n levels each way
    lev, ulev, (nl, nu) = xb.ilu_levels(gen.laplace1d(50)["rowptr"], gen.laplace1d(50)["col"])
    np.testing.assert_array_equal(lev, np.arange(50))
    np.testing.assert_array_equal(ulev, np.arange(50)[::-1])
    # the N x N 5-point stencil: level of (x, y) is x + y, 2N - 1 levels
    N = 12
    A = gen.poisson2d(N)
    lev, _, (nl, _) = xb.ilu_levels(A["rowptr"], A["col"])
    xy = np.arange(N * N)
    np.testing.assert_array_equal(lev, xy % N + xy // N)
    assert nl == 2 * N - 1


def test_missing_diagonal_is_a_breakdown(lib):
    A = gen.laplace1d(10)
    rp, ci = A["rowptr"].copy(), A["col"].copy()
    # drop row 4's diagonal entry
    q = rp[4] + int(np.nonzero(ci[rp[4]:rp[5]] == 4)[0][0])
    ci = np.delete(ci, q)
    rp = rp.copy()
    rp[5:] -= 1
    with pytest.raises(xb.XbError) as e:
        xb.ilu_levels(rp, ci)
    assert e.value.code == xb.XB_EBREAKDOWN and "row 4" in str(e.value)
