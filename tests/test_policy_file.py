"""The numerical policy file of Sec. 2.3.2 ("<keyword> = <value>" lines; POLICY
is TIME / ACCURACY / MEMORY / STABLE with TIME the default; the other
registered keywords CPU, RESIDUAL, MAXMEMORY, MAXTIME, PRECONDITIONER,
SOLVER): the library's reader, host logic only (no device work)."""
import os

import pytest

import paper_2405_01599_gb300 as xb

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "policy")


@pytest.fixture(scope="module")
def lib():
    try:
        return xb.lib()
    except ImportError:
        pytest.skip("CUDA library not built")


def test_policy_values(lib):
    for text, pol in (("POLICY = TIME", xb.POLICY_TIME), ("POLICY=ACCURACY", xb.POLICY_ACCURACY),
                      ("  policy =  memory  ", xb.POLICY_MEMORY), ("Policy = Stable", xb.POLICY_STABLE),
                      ("POLICY = FASTEST", xb.POLICY_TIME)):  # an unregistered value -> TIME
        o, _ = xb.policy_parse(text)
        assert o.policy == pol, text


def test_all_keywords_and_defaults(lib):
    base = xb.default_options()
    o, extra = xb.policy_parse("")
    assert (o.policy, o.tol, o.maxtime_s, o.precond) == (base.policy, base.tol, base.maxtime_s,
                                                         base.precond)
    assert extra == dict(solver=None, max_memory=None, cpu=None)
    text = "\n".join(["# comment", "! Fortran-style comment", "", "RESIDUAL = 1.0D-10",
                      "MAXTIME = 250.5", "PRECONDITIONER = ILU0", "SOLVER = arnoldi",
                      "MAXMEMORY = 512M", "CPU = 8", "SOMETHING_ELSE = 3", "POLICY = MEMORY\r"])
    o, extra = xb.policy_parse(text)
    assert o.tol == 1e-10 and o.maxtime_s == 250.5 and o.precond == xb.PRECOND_ILU0
    assert o.policy == xb.POLICY_MEMORY
    assert extra == dict(solver=xb.SOLVER_ARNOLDI, max_memory=512 * 2.0 ** 20, cpu=8)
    for v, b in (("1024", 1024.0), ("2K", 2048.0), ("16GB", 16 * 2.0 ** 30), ("1.5T", 1.5 * 2.0 ** 40)):
        assert xb.policy_parse(f"MAXMEMORY = {v}")[1]["max_memory"] == b
    for v, s in (("GMRES", xb.SOLVER_GMRES), ("BiCGStab", xb.SOLVER_BICGSTAB),
                 ("LANCZOS", xb.SOLVER_LANCZOS)):
        assert xb.policy_parse(f"SOLVER = {v}")[1]["solver"] == s
    o, _ = xb.policy_parse("PRECONDITIONER = NONE", opt=xb.default_options(precond=1))
    assert o.precond == xb.PRECOND_NONE


def test_bad_lines_are_rejected_with_their_number(lib):
    for text, line in (("POLICY = TIME\nRESIDUAL 1e-8", 2), ("RESIDUAL = abc", 1),
                       ("\n\nMAXTIME = -3", 3), ("SOLVER = CG", 1), ("CPU = 2.5", 1),
                       ("MAXMEMORY = lots", 1), ("PRECONDITIONER = ILUT", 1),
                       ("RESIDUAL = 0", 1)):
        with pytest.raises(xb.XbError) as e:
            xb.policy_parse(text)
        assert f"line {line}" in str(e.value), (text, str(e.value))


def test_read_the_file_by_thread_number(lib):
    o, extra = xb.policy_read(0, GOLDEN)
    assert o.policy == xb.POLICY_ACCURACY and o.tol == 1e-8 and o.maxtime_s == 1000.0
    assert o.precond == xb.PRECOND_ILU0
    assert extra == dict(solver=xb.SOLVER_GMRES, max_memory=16 * 2.0 ** 30, cpu=16)
    with pytest.raises(xb.XbError):
        xb.policy_read(1, GOLDEN)  # no OPENATI_POLICY_INPUT.1


def test_options_from_the_file_feed_the_solvers(lib):
    """The solvers' binding takes the Options the reader filled; keyword
    arguments override single fields of a copy (marshalling only)."""
    o, _ = xb.policy_read(0, GOLDEN)
    m = xb.merge_options(o, dict(m=50))
    assert m.m == 50 and m.policy == xb.POLICY_ACCURACY and m.tol == 1e-8
    assert o.m != 50 or xb.default_options().m == 50  # the original is not modified
    assert xb.merge_options(None, dict(m=7)) == dict(m=7)
    with pytest.raises(KeyError):
        xb.merge_options(o, dict(not_a_field=1))
