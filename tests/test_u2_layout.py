"""The nnz-balanced warp tiles of the U2 variant (Sec. 3.2.2, Fig. 3: rows
split so that each worker gets about the same number of non-zeros, no row
split), host logic only: the library's partition against the properties its
kernel relies on and the rule that builds it."""
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


MATS = {
    "poisson13": lambda: gen.poisson2d(13)["rowptr"],
    "laplace3d_9": lambda: gen.laplace3d(9)["rowptr"],
    "powerlaw3000": lambda: gen.powerlaw(n=3000, seed=1, cap=600)["rowptr"],
    "mixed_empty": lambda: gen.random_general(77, np.array([0, 3, 0, 5] * 19 + [1]), seed=2)["rowptr"],
    "long_rows": lambda: gen.random_general(3000, np.array([1, 2, 700, 9, 0, 129, 128, 127, 3, 1000] * 300),
                                            seed=4)["rowptr"],
    "one_row": lambda: np.array([0, 5], np.int32),
    "all_empty": lambda: np.zeros(41, np.int32),
    "n0": lambda: np.zeros(1, np.int32),
}


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("ipt", [4, 8, 16])
def test_u2_tiles_partition_the_rows(lib, name, ipt):
    rp = np.asarray(MATS[name](), np.int64)
    n = rp.size - 1
    L = np.diff(rp)
    W = 32 * ipt
    tiles, longs = xb.u2_layout(rp, ipt)
    # every row exactly once, in order: tiles and long rows interleave by row
    pieces = [(int(t[0]), int(t[1])) for t in tiles] + [(int(r), int(r) + 1) for r in longs]
    pieces.sort()
    cur = 0
    for a, b in pieces:
        assert a == cur and b > a
        cur = b
    assert cur == n
    long_set = set(int(r) for r in longs)
    for r in long_set:  # a long row overflows a window on its own
        assert rp[r + 1] - (rp[r] - rp[r] % ipt) > W
    nonempty_before = np.concatenate([[0], np.cumsum(L > 0)])
    for r0, r1, ne0, kind in tiles:
        A = rp[r0] - rp[r0] % ipt
        assert rp[r1] - A <= W  # the tile's non-zeros fit its aligned window
        mx = L[r0:r1].max()
        assert (kind & 3) == (0 if mx <= ipt else 1)
        if (kind & 3) == 0:
            assert r1 - r0 <= 32
        assert bool(kind & 4) == bool(np.any(L[r0:r1] == 0))
        assert ne0 == nonempty_before[r0]
        # greedy: the next row, unless it starts a long row, could not join
        if r1 < n and r1 not in long_set:
            grow_max = max(mx, L[r1])
            assert rp[r1 + 1] - A > W or (grow_max <= ipt and r1 - r0 == 32)


def test_u2_uniform_short_rows_are_32_row_blocks(lib):
    """On a 7-point stencil every tile is 32 rows, thread per row: the
    nnz-balanced split coincides with the row split (U1), as Fig. 3 shows for
    uniform rows."""
    rp = gen.laplace3d(12)["rowptr"]
    tiles, longs = xb.u2_layout(rp, 8)
    n = rp.size - 1
    assert longs.size == 0
    assert np.all(tiles[:, 0] == 32 * np.arange(tiles.shape[0]))
    assert np.all(tiles[:, 1] == np.minimum(n, 32 * np.arange(1, tiles.shape[0] + 1)))
    assert np.all((tiles[:, 3] & 3) == 0)


def test_u2_layout_rejects_bad_arguments(lib):
    with pytest.raises(xb.XbError):
        xb.u2_layout(np.array([0, 1], np.int32), 0)
    with pytest.raises(xb.XbError):
        xb.u2_layout(np.array([0, 1], np.int32), 32)
