"""The block-CRS structure of the format-conversion AT's BCSR candidate (Sec. 5
names blocked formats as the AT's next step), host logic only: the library's
layout against its definition written out here (block row b = rows [r b,
r b + r); its blocks are the distinct column blocks of those rows, ascending)."""
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


def definition(A, r):
    rp = np.asarray(A["rowptr"], np.int64)
    col = np.asarray(A["col"], np.int64)
    n = A["n"]
    bptr, bcol = [0], []
    for b in range((n + r - 1) // r):
        c = col[rp[b * r]:rp[min(n, b * r + r)]]
        u = np.unique(c // r)
        bcol += list(u)
        bptr.append(len(bcol))
    return np.array(bptr, np.int64), np.array(bcol, np.int64)


MATS = {
    "block3d_4_dof3": lambda: gen.block_stencil3d(4, 3),
    "block3d_3_dof2": lambda: gen.block_stencil3d(3, 2),
    "poisson13": lambda: gen.poisson2d(13),
    "powerlaw500": lambda: gen.powerlaw(n=500, seed=1, cap=100),
    "empty_rows": lambda: gen.random_general(37, np.array([0, 3, 0, 5] * 9 + [1]), seed=2),
    "n1": lambda: dict(n=1, nnz=1, rowptr=np.array([0, 1], np.int32), col=np.array([0], np.int32),
                       val=np.ones(1), sym_upper=False),
}


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("r", [2, 3, 4])
def test_bcsr_layout_matches_definition(lib, name, r):
    A = MATS[name]()
    bptr, bcol = xb.bcsr_layout(A["rowptr"], A["col"], r)
    dp, dc = definition(A, r)
    np.testing.assert_array_equal(bptr, dp)
    np.testing.assert_array_equal(bcol, dc)


def test_bcsr_of_a_node_blocked_matrix_has_no_fill(lib):
    """With the block size equal to the unknowns per node every block of the
    3-dof stencil is dense: r^2 blocks entries equal the non-zeros."""
    A = gen.block_stencil3d(5, 3)
    bptr, bcol = xb.bcsr_layout(A["rowptr"], A["col"], 3)
    assert 9 * bcol.size == A["nnz"]
    _, bcol2 = xb.bcsr_layout(A["rowptr"], A["col"], 2)
    assert 4 * bcol2.size > A["nnz"]  # misaligned blocks carry zero fill
