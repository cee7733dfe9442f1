"""CPU oracle for the CRS SpMV + restarted Krylov hot path (test infrastructure).

Plain FP64 C (``oracle.c``) reached through ctypes, and the restarted
Arnoldi eigensolver in plain numpy / scipy (``eig.py``).  Only the test suite,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline / reference arm
may import this package; the CUDA library never does, and the two share no
code.  ``build()`` compiles the C source with gcc (no architecture-specific
flags, no fast-math, no FP contraction, so results are identical on x86 and
Arm hosts).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_OUT_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")
_lib = None
_lib_omp = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")


def build(force: bool = False, omp: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so if missing or stale; with omp,
    the OpenMP build _build/liboracle_omp.so used only for the benchmark's
    all-cores CPU baseline (its dot products round differently)."""
    out = _OUT_OMP if omp else _OUT
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fno-fast-math",
                               *(["-fopenmp"] if omp else []),
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def lib_omp():
    """The OpenMP build (benchmark timing only; never for parity)."""
    global _lib_omp
    if _lib_omp is None:
        _lib_omp = _bind(C.CDLL(build(omp=True)))
    return _lib_omp


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(C.CDLL(build()))
    return _lib


def _bind(L):
    """argtypes / restypes of the exported routines."""
    vi, vd, vp = C.c_int, C.c_double, C.c_void_p
    L.orc_spmv.argtypes = [vi, _i32p, _i32p, _f64p, vd, _f64p, vd, _f64p]
    L.orc_spmv_sym.argtypes = [vi, _i32p, _i32p, _f64p, vd, _f64p, vd, _f64p]
    L.orc_spmv_f32.argtypes = [vi, _i32p, _i32p, _f32p, C.c_float, _f32p, C.c_float, _f32p]
    L.orc_dense_matvec.argtypes = [vi, vi, _f64p, _f64p, _f64p]
    L.orc_lu_solve.argtypes = [vi, _f64p, _f64p]
    L.orc_lu_solve.restype = vi
    L.orc_mm_ratio.argtypes = [_f64p, vi, vi]
    L.orc_mm_ratio.restype = vd
    L.orc_dafrt.argtypes = [vi, _f64p, vd]
    L.orc_dafrt.restype = vi
    L.orc_arnoldi.argtypes = [vi, vi, _i32p, _i32p, _f64p, _f64p, vi, _f64p, _f64p]
    L.orc_arnoldi.restype = vi
    L.orc_arnoldi_ortho.argtypes = [vi, vi, _i32p, _i32p, _f64p, _f64p, vi, vi, vi, _f64p,
                                    _f64p]
    L.orc_arnoldi_ortho.restype = vi
    L.orc_gs_qr.argtypes = [vi, vi, _f64p, vi, vi, _f64p, _f64p]
    L.orc_gs_qr.restype = vi
    L.orc_gmres.argtypes = [vi, vi, _i32p, _i32p, _f64p, _f64p, _f64p, vi, vi, vd, vi,
                            vi, vd, vi, vi, vi, vi, vp, _i32p, _f64p, vp, vp, vi]
    L.orc_sym_eig.argtypes = [vi, _f64p, _f64p, _f64p]
    L.orc_lanczos.argtypes = [vi, vi, _i32p, _i32p, _f64p, vi, vi, vi, vd, vd, vi, _f64p,
                              _f64p, vp, _f64p, _i32p]
    L.orc_lanczos.restype = vi
    L.orc_ilu0.argtypes = [vi, _i32p, _i32p, _f64p, _f64p]
    L.orc_ilu0.restype = vi
    L.orc_ilu0_solve.argtypes = [vi, _i32p, _i32p, _f64p, _f64p, _f64p]
    L.orc_gmres.restype = vi
    L.orc_bicgstab.argtypes = [vi, vi, _i32p, _i32p, _f64p, _f64p, _f64p, vd, vi, vp,
                               _i32p, _f64p]
    L.orc_bicgstab.restype = vi
    L.orc_gmres_f32_inner.argtypes = [vi, _i32p, _i32p, _f32p, _f32p, _f32p, vi, vd, vi]
    L.orc_gmres_f32_inner.restype = vi
    L.orc_gmres_ir.argtypes = [vi, _i32p, _i32p, _f64p, _f64p, _f64p, vi, vd, vd, vi, vi,
                               _i32p, _f64p]
    L.orc_gmres_ir.restype = vi
    L.orc_features.argtypes = [vi, _i32p, _i32p, _f64p, vi, _f64p, _f64p]
    L.orc_mlp_forward.argtypes = [_f64p, vi, vi, vi, vi, _f64p, vi, _f64p]
    L.orc_mlp_loss_grad.argtypes = [_f64p, vi, vi, vi, vi, _i32p, _f64p, _i32p, vi, _f64p]
    L.orc_mlp_loss_grad.restype = vd
    L.orc_adam.argtypes = [_f64p, _f64p, _f64p, _f64p, vi, vi, vd, vd, vd, vd]
    L.orc_num_threads.restype = vi
    return L


def _csr(A):
    rp = np.ascontiguousarray(A["rowptr"], dtype=np.int32)
    ci = np.ascontiguousarray(A["col"], dtype=np.int32)
    va = np.ascontiguousarray(A["val"], dtype=np.float64)
    return int(A["n"]), rp, ci, va


def spmv(A, x, alpha=1.0, beta=0.0, y=None, omp=False):
    """y = alpha*A*x + beta*y (general CRS, or upper CRS when A['sym_upper']);
    omp: the OpenMP build's row-parallel loop (benchmark timing only)."""
    n, rp, ci, va = _csr(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(n) if y is None else np.array(y, dtype=np.float64, copy=True)
    L = lib_omp() if omp else lib()
    f = L.orc_spmv_sym if A.get("sym_upper", False) else L.orc_spmv
    f(n, rp, ci, va, float(alpha), x, float(beta), y)
    return y


def spmv_f32(A, x, alpha=1.0, beta=0.0, y=None):
    n, rp, ci, va = _csr(A)
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.zeros(n, np.float32) if y is None else np.array(y, dtype=np.float32, copy=True)
    lib().orc_spmv_f32(n, rp, ci, va.astype(np.float32), np.float32(alpha), x,
                       np.float32(beta), y)
    return y


def dense_matvec(D, x):
    D = np.ascontiguousarray(D, dtype=np.float64)
    y = np.zeros(D.shape[0])
    lib().orc_dense_matvec(D.shape[0], D.shape[1], D, np.ascontiguousarray(x, np.float64), y)
    return y


def lu_solve(D, b):
    D = np.array(D, dtype=np.float64, copy=True, order="C")
    z = np.array(b, dtype=np.float64, copy=True)
    if lib().orc_lu_solve(D.shape[0], D, z) != 0:
        raise np.linalg.LinAlgError("zero pivot")
    return z


def mm_ratio(r, s, t):
    return lib().orc_mm_ratio(np.ascontiguousarray(r, np.float64), int(s), int(t))


def dafrt(samp, theta):
    samp = np.ascontiguousarray(samp, np.float64)
    return lib().orc_dafrt(samp.size, samp, float(theta))


# orthogonalisations (Sec. 3.2.2) and the accuracy policy (Sec. 3.3.2)
MGS, CGS, DGKS, BCGS, AUTO = 0, 1, 2, 3, 4


def arnoldi(A, v0, m, ortho=MGS, bl=4):
    n, rp, ci, va = _csr(A)
    V = np.zeros((m + 1) * n)
    H = np.zeros((m + 1) * m)
    k = lib().orc_arnoldi_ortho(n, 1 if A.get("sym_upper", False) else 0, rp, ci, va,
                                np.ascontiguousarray(v0, np.float64), m, int(ortho), int(bl),
                                V, H)
    return k, V.reshape(m + 1, n), H.reshape(m + 1, m)


def gs_qr(X, ortho=MGS, bl=4):
    """Gram-Schmidt QR of the columns of X (n x k) with the given
    orthogonalisation; returns (Q, R, columns done)."""
    X = np.asarray(X, np.float64)
    n, k = X.shape
    Xc = np.ascontiguousarray(X.T)  # column j contiguous
    Q = np.zeros(n * k)
    R = np.zeros(k * k)
    d = lib().orc_gs_qr(n, k, Xc, int(ortho), int(bl), Q, R)
    return Q.reshape(k, n).T, R.reshape(k, k).T, d


def sym_eig(M):
    """Jacobi eigen-decomposition of a symmetric matrix: (eigenvalues largest
    first, eigenvectors as columns)."""
    M = np.array(M, dtype=np.float64, copy=True)
    m = M.shape[0]
    w = np.zeros(m)
    S = np.zeros(m * m)
    lib().orc_sym_eig(m, np.ascontiguousarray(M).reshape(-1), w, S)
    return w, S.reshape(m, m)


def lanczos(A, nev=10, m=40, tol=1e-10, maxrestart=1000, v0=None, vectors=True, m_max=None,
            theta=10.0):
    """The nev largest eigenvalues of a symmetric A by thick-restart Lanczos;
    returns (evals, evecs (n x nev) or None, info)."""
    n, rp, ci, va = _csr(A)
    v0 = np.ones(n) if v0 is None else np.ascontiguousarray(v0, np.float64)
    ev = np.zeros(nev)
    res = np.zeros(nev)
    vec = np.zeros(n * nev) if vectors else None
    ii = np.zeros(3, np.int32)
    st = lib().orc_lanczos(n, 1 if A.get("sym_upper", False) else 0, rp, ci, va, int(nev),
                           int(m), int(m_max if m_max is not None else m), float(theta),
                           float(tol), int(maxrestart), v0, ev,
                           vec.ctypes.data if vectors else None, res, ii)
    return ev, (vec.reshape(nev, n).T if vectors else None), dict(
        status=st, steps=int(ii[0]), restarts=int(ii[1]), m_final=int(ii[2]), resid=res)


def ilu0(A):
    """ILU(0) factors of a general CRS matrix in its own pattern (values
    aligned with A's col array); returns (lu, status)."""
    n, rp, ci, va = _csr(A)
    lu = np.zeros(max(va.size, 1))
    st = lib().orc_ilu0(n, rp, ci, va, lu)
    return lu[:va.size], st


def ilu0_solve(A, lu, r):
    n, rp, ci, _ = _csr(A)
    z = np.zeros(n)
    lib().orc_ilu0_solve(n, rp, ci, np.ascontiguousarray(lu, np.float64),
                         np.ascontiguousarray(r, np.float64), z)
    return z


def _prec(A, prec):
    if not prec:
        return None, None
    lu, st = ilu0(A)
    if st != 0:
        raise ValueError("ILU(0) breakdown")
    return lu, lu.ctypes.data


def gmres(A, b, x0=None, m=30, m_max=None, tol=1e-8, maxiter=100000,
          dafrt=False, theta=10.0, window=5, dm=5, hist_cap=0, ortho=MGS, fault_check=True,
          ilu=False, omp=False):
    """Restarted GMRES(m), right-preconditioned by ILU(0) when ilu; returns
    (x, info dict).  omp: run the OpenMP build (benchmark timing only)."""
    keep, mptr = _prec(A, ilu)
    n, rp, ci, va = _csr(A)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    ii = np.zeros(5, np.int32)
    dd = np.zeros(2)
    hist = np.zeros(max(hist_cap, 1))
    mh = np.zeros(max(hist_cap, 1), np.int32)
    st = (lib_omp() if omp else lib()).orc_gmres(n, 1 if A.get("sym_upper", False) else 0, rp, ci, va,
                         np.ascontiguousarray(b, np.float64), x, int(m),
                         int(m_max if m_max is not None else m), float(tol), int(maxiter),
                         1 if dafrt else 0, float(theta), int(window), int(dm), int(ortho),
                         1 if fault_check else 0, mptr, ii, dd,
                         hist.ctypes.data if hist_cap else None,
                         mh.ctypes.data if hist_cap else None, int(hist_cap))
    info = dict(status=st, iters=int(ii[0]), restarts=int(ii[1]), m_final=int(ii[2]),
                faults=int(ii[3]), ortho=int(ii[4]), res_implicit=float(dd[0]),
                res_true=float(dd[1]))
    if hist_cap:
        k = min(info["restarts"] + 1, hist_cap)
        info["hist"] = hist[:k].copy()
        info["mhist"] = mh[:k].copy()
    return x, info


def bicgstab(A, b, x0=None, tol=1e-8, maxiter=100000, ilu=False, omp=False):
    """BiCGStab, right-preconditioned by ILU(0) when ilu; omp: the OpenMP
    build (benchmark timing only)."""
    keep, mptr = _prec(A, ilu)
    n, rp, ci, va = _csr(A)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    ii = np.zeros(4, np.int32)
    dd = np.zeros(2)
    st = (lib_omp() if omp else lib()).orc_bicgstab(n, 1 if A.get("sym_upper", False) else 0, rp, ci, va,
                            np.ascontiguousarray(b, np.float64), x, float(tol), int(maxiter),
                            mptr, ii, dd)
    return x, dict(status=st, iters=int(ii[0]), restarts=int(ii[1]), faults=int(ii[3]),
                   res_implicit=float(dd[0]), res_true=float(dd[1]))


def gmres_f32_inner(A, r32, m=30, tol_in=1e-5, maxit=300):
    n, rp, ci, va = _csr(A)
    d = np.zeros(n, np.float32)
    it = lib().orc_gmres_f32_inner(n, rp, ci, va.astype(np.float32),
                                   np.ascontiguousarray(r32, np.float32), d, int(m),
                                   float(tol_in), int(maxit))
    return d, it


def gmres_ir(A, b, x0=None, m=30, tol=1e-8, tol_in=1e-5, maxit_in=300, max_outer=50):
    n, rp, ci, va = _csr(A)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    ii = np.zeros(6, np.int32)
    dd = np.zeros(2)
    st = lib().orc_gmres_ir(n, rp, ci, va, np.ascontiguousarray(b, np.float64), x, int(m),
                            float(tol), float(tol_in), int(maxit_in), int(max_outer), ii, dd)
    return x, dict(status=st, inner_iters=int(ii[0]), outer=int(ii[1]), res_true=float(dd[1]))


def features(A):
    n, rp, ci, va = _csr(A)
    raw = np.zeros(7)
    feat = np.zeros(8)
    lib().orc_features(n, rp, ci, va, 1 if A.get("sym_upper", False) else 0, raw, feat)
    return raw, feat


def mlp_param_count(d_in, h1, h2, heads):
    o = int(sum(heads))
    return h1 * d_in + h1 + h2 * h1 + h2 + o * h2 + o


def mlp_forward(P, dims, X):
    d_in, h1, h2, heads = dims
    o = int(sum(heads))
    X = np.ascontiguousarray(X, np.float64)
    out = np.zeros((X.shape[0], o))
    lib().orc_mlp_forward(np.ascontiguousarray(P, np.float64), d_in, h1, h2, o, X,
                          X.shape[0], out)
    return out


def mlp_loss_grad(P, dims, X, labels):
    d_in, h1, h2, heads = dims
    heads = np.ascontiguousarray(heads, np.int32)
    X = np.ascontiguousarray(X, np.float64)
    labels = np.ascontiguousarray(labels, np.int32)
    g = np.zeros(mlp_param_count(d_in, h1, h2, heads))
    loss = lib().orc_mlp_loss_grad(np.ascontiguousarray(P, np.float64), d_in, h1, h2,
                                   heads.size, heads, X, labels, X.shape[0], g)
    return loss, g


def adam(P, G, M, V, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays P, M, V."""
    lib().orc_adam(P, np.ascontiguousarray(G, np.float64), M, V, P.size, int(t), float(lr),
                   float(b1), float(b2), float(eps))


from .eig import LM as EIG_LM, LR as EIG_LR, arnoldi_eig, wanted_order  # noqa: E402,F401
