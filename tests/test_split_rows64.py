"""64-bit row offsets: the row blocks a plan over more than 2^31 - 64
non-zeros is cut into (host logic only, no matrix is allocated).  Synthetic
row pointers whose offsets cross 2^31 check the split against its rule:
consecutive blocks, rows never split, each block at most the limit, each
block as long as the limit allows."""
import numpy as np
import pytest

import paper_2405_01599_gb300 as xb

LIMIT = 2 ** 31 - 1 - 64  # the int32 plan limit


@pytest.fixture(scope="module")
def lib():
    try:
        return xb.lib()
    except ImportError:
        pytest.skip("CUDA library not built")


def check_split(rp, limit, st):
    n = rp.size - 1
    assert st[0] == 0 and st[-1] == n
    assert np.all(np.diff(st) > 0)
    for a, b in zip(st[:-1], st[1:]):
        assert rp[b] - rp[a] <= limit                      # fits int32 offsets
        if b < n:
            assert rp[b + 1] - rp[a] > limit               # greedy: the next row would not fit


@pytest.mark.parametrize("lengths", [
    [400_000_000] * 12,                                    # 4.8e9 non-zeros
    [1_000_000_000, 1, 0, 1_147_483_000, 5, 2_000_000_000, 3, 700_000_000, 700_000_000],
    [LIMIT, LIMIT, 1],                                     # rows exactly at the limit
    list(np.random.default_rng(0).integers(0, 90_000_000, size=500)),
])
def test_split_crosses_2_31(lib, lengths):
    rp = np.concatenate([[0], np.cumsum(np.asarray(lengths, np.int64))])
    assert rp[-1] > 2 ** 31
    st = xb.split_rows64(rp, LIMIT)
    check_split(rp, LIMIT, st)
    assert st.size - 1 >= int(np.ceil(rp[-1] / LIMIT))


def test_split_below_the_limit_is_one_block(lib):
    rp = np.concatenate([[0], np.cumsum(np.full(1000, 7, np.int64))])
    np.testing.assert_array_equal(xb.split_rows64(rp, LIMIT), [0, 1000])
    np.testing.assert_array_equal(xb.split_rows64(rp, 700), [0, 100, 200, 300, 400, 500, 600, 700,
                                                             800, 900, 1000])


def test_split_rejects_a_row_over_the_limit(lib):
    rp = np.array([0, 5, 5 + LIMIT + 1, 5 + LIMIT + 2], np.int64)
    with pytest.raises(xb.XbError):
        xb.split_rows64(rp, LIMIT)
    with pytest.raises(xb.XbError):
        xb.split_rows64(np.array([0, 3, 2], np.int64), LIMIT)  # decreasing
    with pytest.raises(xb.XbError):
        xb.split_rows64(np.array([1, 3], np.int64), LIMIT)     # rowptr[0] != 0
