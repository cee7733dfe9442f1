"""Python binding of the GB300 CRS SpMV + restarted Krylov library.

Argument marshalling only: every step runs in the CUDA library
(``_build/libxabc.so``, built from ``csrc/`` by ``buildlib.py``).  Torch is used
for device memory and the current stream.  There is no fallback: if the
library is missing or no GPU is present, calls raise.

Names follow the C ABI in ``include/xabc.h`` (spmv_crs, spmv_sym,
spmv_segscan, gmres_solve, bicgstab_solve, xb_tune_exhaustive, ...).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libxabc.so")

XB_OK, XB_EINVAL, XB_ENOMEM, XB_ECUDA, XB_ENOCONV, XB_EBREAKDOWN, XB_ETIMEOUT, XB_EFAULT = \
    0, -1, -2, -3, -4, -5, -6, -7
VAR_AUTO, VAR_ROW, VAR_NNZ, VAR_SEGSCAN, VAR_SYM_ATOMIC, VAR_SYM_TILE, VAR_SELL = -1, 0, 1, 2, 3, 4, 5
VAR_SYM_PART, VAR_SYM_WAGG, VAR_BCSR = 6, 7, 8
VARIANT_NAMES = {0: "row", 1: "nnz", 2: "segscan", 3: "sym_atomic", 4: "sym_tile", 5: "sell",
                 6: "sym_part", 7: "sym_wagg", 8: "bcsr"}
ORTHO_MGS, ORTHO_CGS, ORTHO_DGKS, ORTHO_BCGS, ORTHO_AUTO = 0, 1, 2, 3, 4
POLICY_NONE, POLICY_TIME, POLICY_ACCURACY, POLICY_MEMORY, POLICY_STABLE = 0, 1, 2, 3, 4
PRECOND_NONE, PRECOND_ILU0 = 0, 1
EIG_LR, EIG_LM = 0, 1
SOLVER_GMRES, SOLVER_BICGSTAB, SOLVER_LANCZOS, SOLVER_ARNOLDI = 0, 1, 2, 3
PREC_FP64, PREC_MIXED = 0, 1
TUNER_NONE, TUNER_EXHAUSTIVE, TUNER_MLP = 0, 1, 2


class XbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"xabc error {code}: {msg}")
        self.code = code


class Csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p), ("sym_upper", C.c_int32)]


class Csr64(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p), ("sym_upper", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxiter", C.c_int32), ("maxtime_s", C.c_double),
                ("m", C.c_int32), ("m_max", C.c_int32), ("dafrt", C.c_int32),
                ("dafrt_theta", C.c_double), ("dafrt_window", C.c_int32),
                ("dafrt_dm", C.c_int32), ("ortho", C.c_int32), ("precision", C.c_int32),
                ("tol_inner", C.c_double), ("maxiter_inner", C.c_int32),
                ("max_outer", C.c_int32), ("variant", C.c_int32), ("block", C.c_int32),
                ("ipt", C.c_int32), ("tuner", C.c_int32), ("check_every", C.c_int32),
                ("timing", C.c_int32), ("policy", C.c_int32), ("fault_check", C.c_int32),
                ("precond", C.c_int32), ("ir_fallback", C.c_int32), ("small_n", C.c_int32)]


class Info(C.Structure):
    _fields_ = [(k, C.c_int32) for k in ("status", "iters", "restarts", "m_final", "faults",
                                         "outer", "inner_iters", "fallback", "variant_used",
                                         "block_used", "ipt_used", "spmv_calls",
                                         "ortho_used")] + \
               [(k, C.c_double) for k in ("res_implicit", "res_true", "t_solve_s", "spmv_ms",
                                          "bytes_alg", "mem_bytes")] + \
               [("persistent", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchSys(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("b", C.c_void_p), ("x", C.c_void_p), ("m", C.c_int32),
                ("mode", C.c_int32), ("zero_x", C.c_int32)]


class BatchInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("restarts", C.c_int32),
                ("m", C.c_int32), ("mode", C.c_int32), ("res_true", C.c_double), ("ms", C.c_double)]


class Choice(C.Structure):
    _fields_ = [("variant", C.c_int32), ("block", C.c_int32), ("ipt", C.c_int32),
                ("ms", C.c_float)]


_lib = None


def build(force=False):
    """Compile the CUDA library in-tree (nvcc, sm_103a) if missing or stale."""
    from . import buildlib
    return buildlib.build(force=force)


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} (run build())")
    L = C.CDLL(LIB_PATH)
    vp, i32, f64, f32 = C.c_void_p, C.c_int32, C.c_double, C.c_float
    P = C.POINTER
    sig = {
        "xb_options_default": (None, [P(Options)]),
        "xb_last_error": (C.c_char_p, []),
        "xb_plan_create": (i32, [P(Csr), P(Options), vp, P(vp)]),
        "xb_plan_destroy": (i32, [vp]),
        "xb_plan_create64": (i32, [P(Csr64), P(Options), vp, P(vp)]),
        "xb_split_rows64": (i32, [i32, P(C.c_int64), C.c_int64, P(i32), i32, P(i32)]),
        "xb_plan_set_choice": (i32, [vp, i32, i32, i32]),
        "xb_plan_get_choice": (i32, [vp, P(Choice)]),
        "spmv_crs": (i32, [vp, f64, vp, f64, vp, vp]),
        "spmv_sym": (i32, [vp, f64, vp, f64, vp, vp]),
        "spmv_segscan": (i32, [vp, f64, vp, f64, vp, vp]),
        "xb_spmv": (i32, [vp, i32, i32, i32, f64, vp, f64, vp, vp]),
        "xb_spmv_f32": (i32, [vp, i32, f32, vp, f32, vp, vp]),
        "gmres_solve": (i32, [vp, vp, vp, P(Options), P(Info), vp]),
        "bicgstab_solve": (i32, [vp, vp, vp, P(Options), P(Info), vp]),
        "xb_dot": (i32, [vp, i32, vp, vp, vp, vp]),
        "xb_axpy": (i32, [i32, f64, vp, vp, vp]),
        "xb_mgs": (i32, [vp, i32, i32, vp, C.c_int64, vp, vp, vp]),
        "xb_orth": (i32, [vp, i32, i32, vp, C.c_int64, vp, vp, i32, vp]),
        "xb_lanczos": (i32, [vp, i32, i32, i32, f64, f64, i32, i32, vp, P(f64), vp, P(f64),
                             P(i32), P(f64), vp]),
        "xb_arnoldi": (i32, [vp, i32, i32, i32, f64, f64, i32, i32, i32, i32, vp, P(f64), P(f64),
                             vp, vp, P(f64), P(i32), P(f64), vp]),
        "xb_dense_eig": (i32, [i32, P(f64), i32, P(f64), P(f64), P(f64), P(f64)]),
        "xb_dense_restart_basis": (i32, [i32, P(f64), i32, i32, P(f64), P(i32)]),
        "xb_policy_parse": (i32, [C.c_char_p, P(Options), P(i32), P(f64), P(i32)]),
        "xb_u2_layout": (i32, [i32, P(i32), i32, P(i32), i32, P(i32), P(i32), i32, P(i32)]),
        "xb_bcsr_layout": (i32, [i32, P(i32), P(i32), i32, P(i32), P(i32), C.c_int64,
                                 P(C.c_int64)]),
        "xb_sell_layout": (i32, [i32, P(i32), i32, P(i32), P(i32), P(C.c_int64),
                                 P(C.c_int64)]),
        "xb_ilu_levels": (i32, [i32, P(i32), P(i32), P(i32), P(i32), P(i32)]),
        "xb_policy_read": (i32, [C.c_char_p, i32, P(Options), P(i32), P(f64), P(i32)]),
        "xb_ilu0_setup": (i32, [vp, vp]),
        "xb_ilu0_apply": (i32, [vp, vp, vp, vp]),
        "xb_ilu0_factors": (i32, [vp, vp, vp]),
        "xb_ilu0_config": (i32, [vp, i32, i32]),
        "xb_tune_exhaustive": (i32, [vp, P(Choice), vp]),
        "xb_mm_ratio": (f64, [P(f64), i32, i32]),
        "xb_dafrt": (i32, [i32, P(f64), f64]),
        "xb_features": (i32, [P(Csr), P(f64), P(f32), vp]),
        "xb_tune_sweep": (i32, [vp, P(Choice), i32, P(i32), vp]),
        "xb_tune_mlp": (i32, [vp, P(Csr), vp, P(Choice), P(i32), vp]),
        "xb_mlp_create": (i32, [i32, i32, i32, i32, P(i32), C.c_uint64, P(vp)]),
        "xb_mlp_destroy": (i32, [vp]),
        "xb_mlp_param_count": (C.c_int64, [vp]),
        "xb_mlp_get_params": (i32, [vp, P(f32)]),
        "xb_mlp_set_params": (i32, [vp, P(f32)]),
        "xb_mlp_set_norm": (i32, [vp, P(f32), P(f32)]),
        "xb_mlp_forward": (i32, [vp, vp, i32, vp, vp]),
        "xb_mlp_loss_grad": (i32, [vp, vp, vp, i32, P(f32), vp, vp]),
        "xb_mlp_adam": (i32, [vp, i32, f32, f32, f32, f32, vp]),
        "xb_mlp_train": (i32, [vp, vp, vp, i32, i32, i32, f32, C.c_uint64, P(f32), vp]),
        "xb_mlp_predict": (i32, [vp, vp, i32, P(i32), vp]),
        "xb_mlp_save": (i32, [vp, C.c_char_p]),
        "xb_mlp_load": (i32, [C.c_char_p, P(vp)]),
        "xb_batch_create": (i32, [i32, P(BatchSys), P(Options), vp, P(vp)]),
        "xb_batch_run": (i32, [vp, vp]),
        "xb_batch_results": (i32, [vp, P(BatchInfo), vp]),
        "xb_batch_destroy": (i32, [vp]),
        "xb_batch_solve": (i32, [i32, P(BatchSys), P(Options), P(BatchInfo), vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def last_error():
    return lib().xb_last_error().decode()


def _check(code, ok=(XB_OK,)):
    if code not in ok:
        raise XbError(code, last_error())
    return code


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


def _need(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor (got {t.dtype})")


def dense_restart_basis(A, k, which=EIG_LR):
    """The Arnoldi restart step on a small dense matrix (host logic): an
    orthonormal real basis (n x k') of the invariant subspace of A's k leading
    wanted eigenvalues (k' = k, or k +- 1 to keep a conjugate pair whole)."""
    import numpy as np
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    Q = np.zeros((k + 1) * n)
    ko = C.c_int32()
    P = C.POINTER(C.c_double)
    _check(lib().xb_dense_restart_basis(n, A.ctypes.data_as(P), int(which), int(k),
                                        Q.ctypes.data_as(P), C.byref(ko)))
    return Q[:n * ko.value].reshape(ko.value, n).T


def sell_layout(rowptr, sigma):
    """The SELL-32-sigma layout the SELL variant builds: (perm, slen, off,
    total) as numpy arrays (host logic)."""
    import numpy as np
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    n = rp.size - 1
    slots = 32 * ((n + 31) // 32)
    perm = np.zeros(max(slots, 1), np.int32)
    slen = np.zeros(max(slots, 1), np.int32)
    off = np.zeros((n + 31) // 32 + 1, np.int64)
    tot = C.c_int64()
    f = lambda a, t: a.ctypes.data_as(C.POINTER(t))
    _check(lib().xb_sell_layout(n, f(rp, C.c_int32), int(sigma), f(perm, C.c_int32),
                                f(slen, C.c_int32), f(off, C.c_int64), C.byref(tot)))
    return perm[:slots], slen[:slots], off, tot.value


def u2_layout(rowptr, ipt):
    """The nnz-balanced warp tiles the NNZ (U2) variant builds: (tiles, longs)
    with tiles an (ntiles, 4) int32 array {r0, r1, ne0, kind | 4*has_empty}
    (host logic)."""
    import numpy as np
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    n = rp.size - 1
    nt, nl = C.c_int32(), C.c_int32()
    f = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
    _check(lib().xb_u2_layout(n, f(rp), int(ipt), None, 0, C.byref(nt), None, 0, C.byref(nl)))
    tiles = np.zeros(4 * max(nt.value, 1), np.int32)
    longs = np.zeros(max(nl.value, 1), np.int32)
    _check(lib().xb_u2_layout(n, f(rp), int(ipt), f(tiles), nt.value, C.byref(nt), f(longs),
                              nl.value, C.byref(nl)))
    return tiles[:4 * nt.value].reshape(-1, 4), longs[:nl.value]


def split_rows64(rowptr, max_nnz):
    """The row blocks of a 64-bit row pointer that xb_plan_create64 plans
    separately (host logic): the first row of each block, then n."""
    import numpy as np
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    n = rp.size - 1
    nb = C.c_int32()
    st = np.zeros(n + 2, np.int32)
    _check(lib().xb_split_rows64(n, rp.ctypes.data_as(C.POINTER(C.c_int64)), int(max_nnz),
                                 st.ctypes.data_as(C.POINTER(C.c_int32)), n + 2, C.byref(nb)))
    return st[:nb.value + 1]


def bcsr_layout(rowptr, col, r):
    """The block-CRS structure the BCSR variant builds for r x r blocks:
    (bptr, bcol) as numpy arrays (host logic)."""
    import numpy as np
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    n = rp.size - 1
    f = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
    nb = C.c_int64()
    bptr = np.zeros((n + r - 1) // r + 1, np.int32)
    _check(lib().xb_bcsr_layout(n, f(rp), f(ci), int(r), f(bptr), None, 0, C.byref(nb)))
    bcol = np.zeros(max(nb.value, 1), np.int32)
    _check(lib().xb_bcsr_layout(n, f(rp), f(ci), int(r), f(bptr), f(bcol), nb.value, C.byref(nb)))
    return bptr, bcol[:nb.value]


def ilu_levels(rowptr, col):
    """Dependency levels of the ILU(0) triangles (host logic): (lev, ulev,
    (number of lower levels, number of upper levels))."""
    import numpy as np
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    n = rp.size - 1
    lev = np.zeros(max(n, 1), np.int32)
    ulev = np.zeros(max(n, 1), np.int32)
    nl = np.zeros(2, np.int32)
    f = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
    _check(lib().xb_ilu_levels(n, f(rp), f(ci) if ci.size else None, f(lev), f(ulev), f(nl)))
    return lev[:n], ulev[:n], (int(nl[0]), int(nl[1]))


def merge_options(options, kw):
    """A copy of options (an Options) with the fields in kw replaced, or kw
    itself when options is None (the solvers then start from the defaults)."""
    if options is None:
        return kw
    o = Options.from_buffer_copy(options)
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def default_options(**kw):
    o = Options()
    lib().xb_options_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Plan:
    """A matrix in CRS on the device plus the library's setup data."""

    def __init__(self, rowptr, col, val, sym_upper=False, stream=None):
        """rowptr int32 (xb_plan_create) or int64 (xb_plan_create64: 64-bit row
        offsets, split into row blocks beyond 2^31 - 64 non-zeros)."""
        import torch
        wide = rowptr.dtype == torch.int64
        _need(rowptr, torch.int64 if wide else torch.int32, "rowptr")
        _need(col, torch.int32, "col")
        _need(val, torch.float64, "val")
        self.n = rowptr.numel() - 1
        self.nnz = col.numel()
        self.sym_upper = bool(sym_upper)
        self._keep = (rowptr, col, val)
        h = C.c_void_p()
        if wide:
            self._csr = Csr64(self.n, self.nnz, _ptr(rowptr), _ptr(col), _ptr(val), int(sym_upper))
            _check(lib().xb_plan_create64(C.byref(self._csr), None, _stream(stream), C.byref(h)))
        else:
            self._csr = Csr(self.n, self.nnz, _ptr(rowptr), _ptr(col), _ptr(val), int(sym_upper))
            _check(lib().xb_plan_create(C.byref(self._csr), None, _stream(stream), C.byref(h)))
        self._h = h

    @classmethod
    def from_host(cls, A, device="cuda"):
        import torch
        return cls(torch.as_tensor(A["rowptr"], dtype=torch.int32, device=device),
                   torch.as_tensor(A["col"], dtype=torch.int32, device=device),
                   torch.as_tensor(A["val"], dtype=torch.float64, device=device),
                   sym_upper=A.get("sym_upper", False))

    def close(self):
        if getattr(self, "_h", None):
            lib().xb_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- SpMV ----
    def _vec(self, x, y):
        import torch
        _need(x, torch.float64, "x")
        _need(y, torch.float64, "y")
        if x.numel() != self.n or y.numel() != self.n:
            raise ValueError("vector length != n")

    def spmv_crs(self, x, y, alpha=1.0, beta=0.0, stream=None):
        self._vec(x, y)
        _check(lib().spmv_crs(self._h, alpha, _ptr(x), beta, _ptr(y), _stream(stream)))
        return y

    def spmv_sym(self, x, y, alpha=1.0, beta=0.0, stream=None):
        self._vec(x, y)
        _check(lib().spmv_sym(self._h, alpha, _ptr(x), beta, _ptr(y), _stream(stream)))
        return y

    def spmv_segscan(self, x, y, alpha=1.0, beta=0.0, stream=None):
        self._vec(x, y)
        _check(lib().spmv_segscan(self._h, alpha, _ptr(x), beta, _ptr(y), _stream(stream)))
        return y

    def spmv(self, x, y, alpha=1.0, beta=0.0, variant=VAR_AUTO, block=0, ipt=0, stream=None):
        self._vec(x, y)
        _check(lib().xb_spmv(self._h, variant, block, ipt, alpha, _ptr(x), beta, _ptr(y),
                             _stream(stream)))
        return y

    def spmv_f32(self, x, y, alpha=1.0, beta=0.0, variant=VAR_AUTO, stream=None):
        import torch
        _need(x, torch.float32, "x")
        _need(y, torch.float32, "y")
        _check(lib().xb_spmv_f32(self._h, variant, alpha, _ptr(x), beta, _ptr(y), _stream(stream)))
        return y

    # ---- solvers ----
    def _solve(self, fn, b, x, opts, stream):
        import torch
        _need(b, torch.float64, "b")
        _need(x, torch.float64, "x")
        o = opts if isinstance(opts, Options) else default_options(**(opts or {}))
        info = Info()
        code = fn(self._h, _ptr(b), _ptr(x), C.byref(o), C.byref(info), _stream(stream))
        d = info.as_dict()
        d["status"] = code
        d["error"] = last_error() if code != XB_OK else ""
        if code in (XB_EINVAL, XB_ENOMEM, XB_ECUDA):
            raise XbError(code, d["error"])
        return d

    def gmres(self, b, x, stream=None, options=None, **opts):
        """GMRES(m); options: an Options (e.g. from policy_read), opts override fields."""
        return self._solve(lib().gmres_solve, b, x, merge_options(options, opts), stream)

    def bicgstab(self, b, x, stream=None, options=None, **opts):
        return self._solve(lib().bicgstab_solve, b, x, merge_options(options, opts), stream)

    # ---- tuning ----
    def tune(self, stream=None):
        c = Choice()
        _check(lib().xb_tune_exhaustive(self._h, C.byref(c), _stream(stream)))
        return dict(variant=c.variant, block=c.block, ipt=c.ipt, ms=c.ms)

    def set_choice(self, variant, block=256, ipt=8):
        _check(lib().xb_plan_set_choice(self._h, variant, block, ipt))

    def choice(self):
        c = Choice()
        _check(lib().xb_plan_get_choice(self._h, C.byref(c)))
        return dict(variant=c.variant, block=c.block, ipt=c.ipt, ms=c.ms)

    def sweep(self, stream=None):
        """Every SpMV candidate with its best time (list of dicts)."""
        cap = 64
        arr = (Choice * cap)()
        cnt = C.c_int32()
        _check(lib().xb_tune_sweep(self._h, arr, cap, C.byref(cnt), _stream(stream)))
        return [dict(variant=arr[i].variant, block=arr[i].block, ipt=arr[i].ipt, ms=arr[i].ms)
                for i in range(min(cnt.value, cap))]

    def tune_mlp(self, model, stream=None):
        """Learned tuning: returns (choice dict, predicted restart length m)."""
        c = Choice()
        m = C.c_int32()
        _check(lib().xb_tune_mlp(self._h, C.byref(self._csr), model._h, C.byref(c), C.byref(m),
                                 _stream(stream)))
        return dict(variant=c.variant, block=c.block, ipt=c.ipt), m.value

    # ---- vector ops ----
    def dot(self, x, y, stream=None):
        import torch
        out = torch.empty(1, dtype=torch.float64, device=x.device)
        _check(lib().xb_dot(self._h, x.numel(), _ptr(x), _ptr(y), _ptr(out), _stream(stream)))
        return out

    def mgs(self, V, w, stream=None):
        """One MGS sweep of w against the k rows of V; returns h (k+1)."""
        import torch
        k, ld = V.shape
        h = torch.empty(k + 1, dtype=torch.float64, device=V.device)
        _check(lib().xb_mgs(self._h, w.numel(), k, _ptr(V), ld, _ptr(w), _ptr(h),
                            _stream(stream)))
        return h

    def lanczos(self, nev=10, m=40, tol=1e-8, maxrestart=1000, v0=None, vectors=True,
                m_max=None, theta=10.0, policy=POLICY_NONE, stream=None):
        """The nev largest eigenvalues (thick-restart Lanczos), under an optional
        numerical computation policy; returns (evals, evecs n x nev or None,
        info dict)."""
        import numpy as np
        import torch
        dev = self._keep[2].device
        if v0 is not None:
            _need(v0, torch.float64, "v0")
        ev = (C.c_double * nev)()
        rs = (C.c_double * nev)()
        cnt = (C.c_int32 * 5)()
        sts = (C.c_double * 2)()
        vec = torch.empty((nev, self.n), dtype=torch.float64, device=dev) if vectors else None
        code = lib().xb_lanczos(self._h, nev, m, m if m_max is None else m_max, theta, tol,
                                maxrestart, int(policy), _ptr(v0) if v0 is not None
                                else None, ev, _ptr(vec) if vectors else None, rs, cnt, sts,
                                _stream(stream))
        if code in (XB_EINVAL, XB_ENOMEM, XB_ECUDA):
            raise XbError(code, last_error())
        info = dict(status=code, steps=cnt[0], restarts=cnt[1], m_final=cnt[2],
                    ortho_used=cnt[3], outer=cnt[4], mem_bytes=sts[0], true_resid=sts[1],
                    resid=np.array(rs[:]))
        return np.array(ev[:]), (vec.T if vectors else None), info

    def arnoldi(self, nev=10, m=20, tol=1e-8, maxrestart=1000, v0=None, vectors=True,
                m_max=None, theta=10.0, which=EIG_LR, ortho=ORTHO_DGKS, policy=POLICY_NONE,
                stream=None):
        """nev eigenvalues of a general A at the wanted end (EIG_LR: largest
        real part, EIG_LM: largest modulus) by restarted Arnoldi, under an
        optional numerical computation policy; returns (evals complex numpy
        (nev), evecs complex n x nev or None, info dict)."""
        import numpy as np
        import torch
        dev = self._keep[2].device
        if v0 is not None:
            _need(v0, torch.float64, "v0")
        er = (C.c_double * nev)()
        ei = (C.c_double * nev)()
        rs = (C.c_double * nev)()
        cnt = (C.c_int32 * 5)()
        sts = (C.c_double * 2)()
        vr = torch.empty((nev, self.n), dtype=torch.float64, device=dev) if vectors else None
        vi = torch.empty((nev, self.n), dtype=torch.float64, device=dev) if vectors else None
        code = lib().xb_arnoldi(self._h, nev, m, m if m_max is None else m_max, theta, tol,
                                maxrestart, int(which), int(ortho), int(policy),
                                _ptr(v0) if v0 is not None else None, er, ei,
                                _ptr(vr) if vectors else None, _ptr(vi) if vectors else None,
                                rs, cnt, sts, _stream(stream))
        if code in (XB_EINVAL, XB_ENOMEM, XB_ECUDA):
            raise XbError(code, last_error())
        info = dict(status=code, steps=cnt[0], restarts=cnt[1], m_final=cnt[2],
                    ortho_used=cnt[3], outer=cnt[4], mem_bytes=sts[0], true_resid=sts[1],
                    resid=np.array(rs[:]))
        ev = np.array(er[:]) + 1j * np.array(ei[:])
        vec = torch.complex(vr, vi).T if vectors else None
        return ev, vec, info

    def ilu0_setup(self, stream=None):
        _check(lib().xb_ilu0_setup(self._h, _stream(stream)))

    def ilu0_apply(self, r, z, stream=None):
        """z = (L U)^{-1} r with the plan's ILU(0) factors."""
        self._vec(r, z)
        _check(lib().xb_ilu0_apply(self._h, _ptr(r), _ptr(z), _stream(stream)))
        return z

    def ilu0_config(self, mode=-1, barrier_polls=0):
        """ILU(0) substitution path (-1 automatic, 0 graph, 1 persistent) and
        the persistent path's barrier poll limit (0 = default)."""
        _check(lib().xb_ilu0_config(self._h, int(mode), int(barrier_polls)))

    def ilu0_factors(self, stream=None):
        import torch
        lu = torch.empty(self.nnz, dtype=torch.float64, device=self._keep[2].device)
        _check(lib().xb_ilu0_factors(self._h, _ptr(lu), _stream(stream)))
        return lu

    def orth(self, V, w, ortho, stream=None):
        """Orthogonalise w against the k rows of V with ORTHO_MGS / CGS / DGKS /
        BCGS; returns h (k projection coefficients, then ||w||)."""
        import torch
        k, ld = V.shape
        h = torch.empty(k + 1, dtype=torch.float64, device=V.device)
        _check(lib().xb_orth(self._h, w.numel(), k, _ptr(V), ld, _ptr(w), _ptr(h), int(ortho),
                             _stream(stream)))
        return h


def axpy(a, x, y, stream=None):
    _check(lib().xb_axpy(x.numel(), a, _ptr(x), _ptr(y), _stream(stream)))
    return y


def features(rowptr, col, val, sym_upper=False, stream=None):
    import numpy as np
    csr = Csr(rowptr.numel() - 1, col.numel(), _ptr(rowptr), _ptr(col), _ptr(val), int(sym_upper))
    raw = (C.c_double * 7)()
    feat = (C.c_float * 8)()
    _check(lib().xb_features(C.byref(csr), raw, feat, _stream(stream)))
    return np.array(raw[:]), np.array(feat[:], dtype=np.float32)


def dense_eig(A, which=EIG_LR, vectors=True):
    """Eigenvalues (wanted order, conjugate pairs adjacent) and unit
    eigenvectors (columns) of a small dense general matrix: the host step of
    the Arnoldi eigensolver."""
    import numpy as np
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    P = C.POINTER(C.c_double)
    f = lambda a: a.ctypes.data_as(P)
    wr, wi = np.zeros(n), np.zeros(n)
    vr, vi = (np.zeros((n, n)), np.zeros((n, n))) if vectors else (None, None)
    _check(lib().xb_dense_eig(n, f(A), int(which), f(wr), f(wi), f(vr) if vectors else None,
                              f(vi) if vectors else None))
    return wr + 1j * wi, ((vr + 1j * vi).T if vectors else None)


def _policy_result(code, o, sv, mm, cpu):
    _check(code)
    extra = dict(solver=sv.value if sv.value >= 0 else None,
                 max_memory=mm.value if mm.value >= 0 else None,
                 cpu=cpu.value if cpu.value >= 0 else None)
    return o, extra


def policy_parse(text, opt=None):
    """Numerical policy file contents (Sec. 2.3.2) -> (Options updated from
    opt or the defaults, dict(solver, max_memory, cpu) with None for absent
    keywords)."""
    o = opt if opt is not None else default_options()
    sv, mm, cpu = C.c_int32(-1), C.c_double(-1.0), C.c_int32(-1)
    return _policy_result(lib().xb_policy_parse(text.encode(), C.byref(o), C.byref(sv),
                                                C.byref(mm), C.byref(cpu)), o, sv, mm, cpu)


def policy_read(thread_id=0, directory=None, opt=None):
    """Read OPENATI_POLICY_INPUT.<thread_id> (from directory, default the
    current one) as policy_parse does."""
    o = opt if opt is not None else default_options()
    sv, mm, cpu = C.c_int32(-1), C.c_double(-1.0), C.c_int32(-1)
    d = directory.encode() if directory else None
    return _policy_result(lib().xb_policy_read(d, int(thread_id), C.byref(o), C.byref(sv),
                                               C.byref(mm), C.byref(cpu)), o, sv, mm, cpu)


def mm_ratio(r, s, t):
    arr = (C.c_double * len(r))(*r)
    return lib().xb_mm_ratio(arr, s, t)


def dafrt(samp, theta):
    arr = (C.c_double * len(samp))(*samp)
    return lib().xb_dafrt(len(samp), arr, theta)


TUNER_HEADS = (5, 4, 5, 6)          # variant, CTA size, items per thread, restart m
TUNER_BLOCKS = (64, 128, 256, 512)
TUNER_IPTS = (1, 4, 8, 16, 32)
TUNER_RESTARTS = (10, 20, 30, 50, 80, 120)


class Mlp:
    """The learned tuner's MLP; every forward/backward/update step runs in the
    library's CUDA kernels."""

    def __init__(self, d_in=8, h1=64, h2=64, heads=TUNER_HEADS, seed=0, _handle=None):
        if _handle is not None:
            self._h = _handle
        else:
            hs = (C.c_int32 * len(heads))(*heads)
            h = C.c_void_p()
            _check(lib().xb_mlp_create(d_in, h1, h2, len(heads), hs, seed, C.byref(h)))
            self._h = h
        self.dims = (d_in, h1, h2, tuple(heads))

    @classmethod
    def load(cls, path):
        h = C.c_void_p()
        _check(lib().xb_mlp_load(path.encode(), C.byref(h)))
        import struct
        with open(path, "rb") as f:
            f.read(8)
            d_in, h1, h2, nh = struct.unpack("4i", f.read(16))
            heads = struct.unpack("8i", f.read(32))[:nh]
        obj = cls.__new__(cls)
        obj._h = h
        obj.dims = (d_in, h1, h2, tuple(heads))
        return obj

    def close(self):
        if getattr(self, "_h", None):
            lib().xb_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def param_count(self):
        return int(lib().xb_mlp_param_count(self._h))

    def get_params(self):
        import numpy as np
        P = np.zeros(self.param_count(), np.float32)
        _check(lib().xb_mlp_get_params(self._h, P.ctypes.data_as(C.POINTER(C.c_float))))
        return P

    def set_params(self, P):
        import numpy as np
        P = np.ascontiguousarray(P, np.float32)
        _check(lib().xb_mlp_set_params(self._h, P.ctypes.data_as(C.POINTER(C.c_float))))

    def set_norm(self, mu, sd):
        import numpy as np
        mu = np.ascontiguousarray(mu, np.float32)
        sd = np.ascontiguousarray(sd, np.float32)
        _check(lib().xb_mlp_set_norm(self._h, mu.ctypes.data_as(C.POINTER(C.c_float)),
                                     sd.ctypes.data_as(C.POINTER(C.c_float))))

    def forward(self, X, stream=None):
        import torch
        _need(X, torch.float32, "X")
        out = torch.empty((X.shape[0], sum(self.dims[3])), dtype=torch.float32, device=X.device)
        _check(lib().xb_mlp_forward(self._h, _ptr(X), X.shape[0], _ptr(out), _stream(stream)))
        return out

    def loss_grad(self, X, labels, stream=None):
        import torch
        _need(X, torch.float32, "X")
        _need(labels, torch.int32, "labels")
        g = torch.empty(self.param_count(), dtype=torch.float32, device=X.device)
        loss = C.c_float()
        _check(lib().xb_mlp_loss_grad(self._h, _ptr(X), _ptr(labels), X.shape[0], C.byref(loss),
                                      _ptr(g), _stream(stream)))
        return loss.value, g

    def adam(self, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=None):
        _check(lib().xb_mlp_adam(self._h, t, lr, b1, b2, eps, _stream(stream)))

    def train(self, X, labels, epochs=200, batch=256, lr=3e-3, seed=0, stream=None):
        import torch
        _need(X, torch.float32, "X")
        _need(labels, torch.int32, "labels")
        loss = C.c_float()
        _check(lib().xb_mlp_train(self._h, _ptr(X), _ptr(labels), X.shape[0], epochs, batch, lr,
                                  seed, C.byref(loss), _stream(stream)))
        return loss.value

    def predict(self, X, stream=None):
        import numpy as np
        import torch
        _need(X, torch.float32, "X")
        out = np.zeros((X.shape[0], len(self.dims[3])), np.int32)
        _check(lib().xb_mlp_predict(self._h, _ptr(X), X.shape[0],
                                    out.ctypes.data_as(C.POINTER(C.c_int32)), _stream(stream)))
        return out

    def save(self, path):
        _check(lib().xb_mlp_save(self._h, path.encode()))


class Batch:
    """Many independent systems solved by GMRES(m) in one persistent,
    graph-captured launch (xb_batch_*).  systems: list of dicts with device
    tensors rowptr, col, val, b, x and ints m, mode (0 thread/row, 1 warp/row).
    """

    def __init__(self, systems, stream=None, zero_x=True, **opts):
        import torch
        self._keep = []
        arr = (BatchSys * max(1, len(systems)))()
        for i, q in enumerate(systems):
            for k in ("rowptr", "col"):
                _need(q[k], torch.int32, k)
            for k in ("val", "b", "x"):
                _need(q[k], torch.float64, k)
            arr[i] = BatchSys(q["rowptr"].numel() - 1, q["col"].numel(), _ptr(q["rowptr"]),
                              _ptr(q["col"]), _ptr(q["val"]), _ptr(q["b"]), _ptr(q["x"]),
                              int(q.get("m", 30)), int(q.get("mode", 0)), int(zero_x))
            self._keep.append(q)
        self.count = len(systems)
        o = default_options(**opts)
        h = C.c_void_p()
        _check(lib().xb_batch_create(self.count, arr, C.byref(o), _stream(stream), C.byref(h)))
        self._h = h

    def run(self, stream=None):
        _check(lib().xb_batch_run(self._h, _stream(stream)))

    def results(self, stream=None):
        infos = (BatchInfo * max(1, self.count))()
        lib().xb_batch_results(self._h, infos, _stream(stream))
        return [{k: getattr(infos[i], k) for k, _ in BatchInfo._fields_} for i in range(self.count)]

    def close(self):
        if getattr(self, "_h", None):
            lib().xb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
