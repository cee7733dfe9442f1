"""Host-side helpers of bench.py: the algorithmic-bytes formula of one SpMV
(12 nnz + 4 (n + 1) + 16 n for FP64 with int32 indices, plus 8 n when y is
read) and the code regions that keep the recorded DRAM-traffic figure valid
(every marker must still be found, or the figure would silently disappear)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes():
    A = dict(n=10, nnz=37)
    assert bench.alg_bytes(A) == 12 * 37 + 4 * 11 + 16 * 10
    assert bench.alg_bytes(A, beta=True) == 12 * 37 + 4 * 11 + 24 * 10
    assert bench.alg_bytes(A, vb=4) == 8 * 37 + 4 * 11 + 8 * 10


def test_headline_source_regions_are_found():
    h = bench.headline_src_hash()
    assert h is not None and len(h) == 64
    for key, (traffic, digest) in bench.NCU_TRAFFIC.items():
        assert traffic > 0 and len(digest) == 64, key
