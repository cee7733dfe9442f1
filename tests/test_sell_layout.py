"""The SELL-32-sigma layout of the format-conversion AT (Sec. 5 names CRS to
ELL-type conversions as the AT's next step), host logic only: the library's
layout against its definition written out here (rows sorted by length,
longest first and stable, in windows of sigma rows; slices of 32 slots as
wide as their longest row), and the properties the SELL kernel relies on."""
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


def definition(rowptr, sigma):
    L = np.diff(np.asarray(rowptr, np.int64))
    n = L.size
    order = []
    for w0 in range(0, n, sigma):
        win = list(range(w0, min(n, w0 + sigma)))
        order += sorted(win, key=lambda r: -L[r])  # Python's sort is stable
    slots = 32 * ((n + 31) // 32)
    perm = np.full(slots, -1, np.int64)
    perm[:n] = order
    slen = np.where(perm >= 0, L[np.maximum(perm, 0)], 0)
    widths = slen.reshape(-1, 32).max(axis=1) if slots else np.zeros(0, np.int64)
    off = np.concatenate([[0], np.cumsum(32 * widths)]).astype(np.int64)
    return perm, slen, off, int(off[-1])


MATS = {
    "poisson13": lambda: gen.poisson2d(13)["rowptr"],
    "powerlaw3000": lambda: gen.powerlaw(n=3000, seed=1, cap=300)["rowptr"],
    "mixed_empty": lambda: gen.random_general(77, np.array([0, 3, 0, 5] * 19 + [1]), seed=2)["rowptr"],
    "n1": lambda: np.array([0, 4]),
    "n0": lambda: np.array([0]),
    "ties": lambda: np.concatenate([[0], np.cumsum(np.tile([2, 2, 1, 1, 3], 40))]),
}


@pytest.mark.parametrize("mname", list(MATS))
@pytest.mark.parametrize("sigma", [1, 32, 100, 1024])
def test_layout_matches_definition(lib, mname, sigma):
    rp = MATS[mname]()
    perm, slen, off, total = xb.sell_layout(rp, sigma)
    dp, dl, do, dt = definition(rp, sigma)
    np.testing.assert_array_equal(perm, dp)
    np.testing.assert_array_equal(slen, dl)
    np.testing.assert_array_equal(off, do)
    assert total == dt
    n = len(rp) - 1
    # every row in exactly one slot; a row's entries fit inside its slice
    assert sorted(perm[perm >= 0].tolist()) == list(range(n))
    for q in range(len(off) - 1):
        assert np.all(off[q] + 32 * slen[32 * q:32 * q + 32] <= off[q + 1])
