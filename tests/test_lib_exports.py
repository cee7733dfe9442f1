"""The CUDA library builds (cross-compiled for sm_103a), loads on a host
without a GPU, and exports every function that include/xabc.h declares.
The host-only entry points (MM ratio, DAFRT judgement) run here too."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "xabc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "for", "while")))


@pytest.fixture(scope="module")
def lib():
    import paper_2405_01599_gb300 as xb
    xb.build()
    return xb.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("spmv_crs", "spmv_sym", "spmv_segscan", "gmres_solve", "bicgstab_solve",
                 "xb_plan_create", "xb_tune_exhaustive"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_entry_points(lib):
    import paper_2405_01599_gb300 as xb
    assert xb.mm_ratio([1.0, 0.5, 0.25, 0.125, 0.0625], 5, 5) == 16.0
    assert xb.mm_ratio([3.0] * 5, 5, 5) == 1.0
    assert xb.dafrt([1.0] * 5, 10.0) == 1
    assert xb.dafrt([1, 0.5, 0.25, 0.125, 0.0625], 10.0) == 0
    o = xb.default_options()
    assert o.tol == 1e-8 and o.m == 30 and o.maxtime_s == 1000.0 and o.dafrt_window == 5
    assert o.dafrt_dm == 5


def test_no_cpu_fallback_without_gpu():
    """On a host without a GPU the product path must fail loudly."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import numpy as np
    import paper_2405_01599_gb300 as xb
    from paper_2405_01599_gb300 import gen
    with pytest.raises(Exception):
        xb.Plan.from_host(gen.poisson2d(4), "cpu")
