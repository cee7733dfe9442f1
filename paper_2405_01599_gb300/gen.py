"""Seeded synthetic matrix generators (input recipes only).

These build the CRS inputs that both the CUDA library and the CPU oracle are
run on.  They contain none of the solver's or the SpMV's arithmetic: only the
construction of matrices from their recipes (stencil coefficients, random
patterns and values).  The right-hand side "b = A * ones" of the paper's
solver experiments (Sec. 4.3) is NOT formed here; callers compute it with the
oracle (tests) or the library (benchmark).

A matrix is a dict: n, nnz, rowptr (int32, n+1), col (int32), val (float64),
sym_upper (bool: only the upper triangle, diagonal included, is stored).
Columns are 0-based and strictly ascending within each row.
"""
from __future__ import annotations

import math

import numpy as np


def _mat(n, rowptr, col, val, sym_upper=False, **extra):
    d = dict(n=int(n), nnz=int(rowptr[-1]), rowptr=np.ascontiguousarray(rowptr, np.int32),
             col=np.ascontiguousarray(col, np.int32),
             val=np.ascontiguousarray(val, np.float64), sym_upper=bool(sym_upper))
    d.update(extra)
    return d


def _stencil(dims, coeffs, upper=False):
    """Grid stencil on a box with zero Dirichlet boundary.

    dims: grid sides (x fastest).  coeffs: dict offset-tuple -> coefficient;
    the offset (0,..,0) is the diagonal.  Rows/columns are grid points in
    lexicographic order x + Nx*y + Nx*Ny*z.  Neighbours outside the box are
    dropped.  upper=True keeps only entries with column >= row.
    """
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    idx = np.arange(n, dtype=np.int64)
    coord = [(idx // strides[a]) % dims[a] for a in range(len(dims))]
    offs = []
    for off, c in coeffs.items():
        lin = sum(o * s for o, s in zip(off, strides))
        offs.append((lin, off, c))
    offs.sort(key=lambda t: t[0])  # ascending column offset = sorted CRS rows
    if upper:
        offs = [t for t in offs if t[0] >= 0]
    k = len(offs)
    cols = np.empty((n, k), np.int64)
    vals = np.empty((n, k), np.float64)
    mask = np.ones((n, k), bool)
    for j, (lin, off, c) in enumerate(offs):
        ok = np.ones(n, bool)
        for a, o in enumerate(off):
            if o:
                ok &= (coord[a] + o >= 0) & (coord[a] + o < dims[a])
        mask[:, j] = ok
        cols[:, j] = idx + lin
        vals[:, j] = c
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return n, rowptr, cols[mask], vals[mask]


def laplace1d(n):
    """tridiag(-1, 2, -1), n x n."""
    n_, rp, c, v = _stencil((n,), {(0,): 2.0, (-1,): -1.0, (1,): -1.0})
    return _mat(n_, rp, c, v, kind="laplace1d", side=n)


def poisson2d(N, upper=False):
    """2D 5-point Poisson on an N x N grid: diagonal 4, neighbours -1."""
    co = {(0, 0): 4.0, (-1, 0): -1.0, (1, 0): -1.0, (0, -1): -1.0, (0, 1): -1.0}
    n, rp, c, v = _stencil((N, N), co, upper)
    return _mat(n, rp, c, v, upper, kind="poisson2d", side=N)


def poisson2d_dense_rows(N, count=4, length=3000, seed=0):
    """2D 5-point Poisson on an N x N grid with `count` rows (seeded choice)
    widened to about `length` entries: each added entry (a distinct random
    column) holds -1 / length, and those rows' diagonal grows by 1, so the
    matrix stays diagonally dominant.  Skewed rows on a well-conditioned
    system (for the long-row paths of the SpMV kernels)."""
    A = poisson2d(N)
    n = A["n"]
    rng = np.random.default_rng(seed)
    wide = set(int(r) for r in rng.choice(n, size=min(count, n), replace=False))
    rp, ci, va = A["rowptr"], A["col"], A["val"]
    rows_c, rows_v = [], []
    for r in range(n):
        c = ci[rp[r]:rp[r + 1]].astype(np.int64)
        v = va[rp[r]:rp[r + 1]].copy()
        if r in wide:
            extra = np.setdiff1d(rng.choice(n, size=min(length, n), replace=False), c)
            v = np.where(c == r, v + 1.0, v)
            c = np.concatenate([c, extra])
            v = np.concatenate([v, np.full(extra.size, -1.0 / length)])
            o = np.argsort(c, kind="stable")
            c, v = c[o], v[o]
        rows_c.append(c)
        rows_v.append(v)
    rowptr = np.zeros(n + 1, np.int64)
    rowptr[1:] = np.cumsum([len(c) for c in rows_c])
    return _mat(n, rowptr, np.concatenate(rows_c), np.concatenate(rows_v),
                kind="poisson2d_dense_rows", side=N)


def laplace3d(N, upper=False):
    """3D 7-point Laplacian on an N^3 grid: diagonal 6, neighbours -1."""
    co = {(0, 0, 0): 6.0}
    for a in range(3):
        for s in (-1, 1):
            o = [0, 0, 0]
            o[a] = s
            co[tuple(o)] = -1.0
    n, rp, c, v = _stencil((N, N, N), co, upper)
    return _mat(n, rp, c, v, upper, kind="laplace3d", side=N)


def stencil27(N):
    """3D 27-point stencil on an N^3 grid (the FEM-like class of 10-30
    non-zeros per row): diagonal 26, every neighbour in the 3 x 3 x 3 box -1."""
    co = {}
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                co[(dx, dy, dz)] = 26.0 if (dx, dy, dz) == (0, 0, 0) else -1.0
    n, rp, c, v = _stencil((N, N, N), co)
    return _mat(n, rp, c, v, kind="stencil27", side=N)


def convdiff3d(N=256, pe=10.0, dims=None):
    """3D convection-diffusion -Lap(u) + Pe*(u_x + u_y + u_z) on (0,1)^3.

    Zero Dirichlet boundary, h = 1/(N+1), first-order upwind for the positive
    velocity (Pe, Pe, Pe), scaled by h^2: diagonal 6 + 3*Pe*h, the -x/-y/-z
    neighbours -(1 + Pe*h), the +x/+y/+z neighbours -1.  Nonsymmetric.
    dims = (Nx, Ny, Nz) gives a box grid with the same stencil (h from N).
    """
    h = 1.0 / (N + 1)
    ph = pe * h
    co = {(0, 0, 0): 6.0 + 3.0 * ph}
    for a in range(3):
        o = [0, 0, 0]
        o[a] = -1
        co[tuple(o)] = -(1.0 + ph)
        o[a] = 1
        co[tuple(o)] = -1.0
    n, rp, c, v = _stencil(tuple(dims) if dims is not None else (N, N, N), co)
    return _mat(n, rp, c, v, kind="convdiff3d", side=N, pe=pe)


def block_stencil3d(N, dof=3, seed=0):
    """A 7-point 3D grid (N^3 nodes) with `dof` unknowns per node and a dense
    dof x dof coupling block for every stencil neighbour pair: the pattern of
    vector-valued PDEs such as 3D elasticity (3 displacements per node).  Node
    (i, j, k) is index (i * N + j) * N + k; its unknowns are consecutive rows.
    Off-diagonal blocks U[-1, 0]; the diagonal block U[-1, 1] off its diagonal
    and 1 + the row's absolute sum on it (strictly diagonally dominant)."""
    rng = np.random.default_rng(seed)
    nodes = N ** 3
    n = nodes * dof
    idx = np.arange(nodes, dtype=np.int64)
    i, j, k = idx // (N * N), (idx // N) % N, idx % N
    nb = [idx]
    ok = [np.ones(nodes, bool)]
    for d, (di, dj, dk) in enumerate(((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1))):
        ii, jj, kk = i + di, j + dj, k + dk
        ok.append((ii >= 0) & (ii < N) & (jj >= 0) & (jj < N) & (kk >= 0) & (kk < N))
        nb.append(np.clip(ii, 0, N - 1) * N * N + np.clip(jj, 0, N - 1) * N + np.clip(kk, 0, N - 1))
    nb = np.stack(nb, axis=1)   # nodes x 7 (0: the node itself)
    ok = np.stack(ok, axis=1)
    order = np.argsort(np.where(ok, nb, np.iinfo(np.int64).max), axis=1, kind="stable")
    nbs = np.take_along_axis(nb, order, axis=1)
    oks = np.take_along_axis(ok, order, axis=1)
    deg = oks.sum(axis=1)
    # every row of a node has the node's neighbours' unknowns, ascending
    cols = (nbs[:, None, :, None] * dof + np.arange(dof)[None, None, None, :])  # node, -, t, b
    cols = np.broadcast_to(cols, (nodes, dof, 7, dof))
    mask = np.broadcast_to(oks[:, None, :, None], cols.shape)
    same = np.broadcast_to((nbs == idx[:, None])[:, None, :, None], cols.shape)
    v = np.where(same, rng.uniform(-1, 1, cols.shape), rng.uniform(-1, 0, cols.shape))
    rows = idx[:, None] * dof + np.arange(dof)[None, :]                         # node, a
    diag = cols == rows[:, :, None, None]
    v = np.where(diag | ~mask, 0.0, v)
    v = np.where(diag, 1.0 + np.abs(v).sum(axis=(2, 3), keepdims=True), v)
    col = cols[mask]
    val = v[mask]
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.repeat(deg * dof, dof), out=rowptr[1:])
    return _mat(n, rowptr, col, val, kind="block_stencil3d", side=N, dof=dof)


def quasi_triangular(n=400, per_row=4, seed=0, pair_frac=0.5, top=10.0, ratio=0.995,
                     signed=False, off=1.0):
    """Block upper-triangular n x n with a spectrum known by construction.

    Diagonal blocks, top to bottom: 1 x 1 blocks [a] and 2 x 2 blocks
    [[a, b], [-b, a]] (a block is 2 x 2 with probability pair_frac) with
    eigenvalues a +- ib.  The a values are top * ratio**j, j = 0, 1, ...
    (times a random sign if signed), assigned to the blocks in random order;
    b is U[0.5, 2].  Right of each row's block: per_row distinct columns with
    values off * U[-1, 1].  The blocks are kept in "blocks" as (a, b) pairs
    (b = 0 for a 1 x 1 block).
    """
    rng = np.random.default_rng(seed)
    sizes = []
    i = 0
    while i < n:
        two = i + 1 < n and rng.random() < pair_frac
        sizes.append(2 if two else 1)
        i += sizes[-1]
    nb = len(sizes)
    a_vals = top * ratio ** np.arange(nb, dtype=np.float64)
    if signed:
        a_vals *= rng.choice([-1.0, 1.0], size=nb)
    a_vals = rng.permutation(a_vals)
    blocks = [(float(a), float(rng.uniform(0.5, 2.0)) if sz == 2 else 0.0)
              for a, sz in zip(a_vals, sizes)]
    rows_c, rows_v = [], []
    i0 = 0
    for (a, b), size in zip(blocks, sizes):
        for r in range(size):
            c = [i0, i0 + 1] if size == 2 else [i0]
            v = ([a, b] if r == 0 else [-b, a]) if size == 2 else [a]
            right = n - (i0 + size)
            if right > 0:
                cc = i0 + size + np.sort(rng.choice(right, size=min(per_row, right),
                                                    replace=False))
                c = c + cc.tolist()
                v = v + (off * rng.uniform(-1.0, 1.0, size=len(cc))).tolist()
            rows_c.append(np.array(c, np.int64))
            rows_v.append(np.array(v, np.float64))
        i0 += size
    rowptr = np.zeros(n + 1, np.int64)
    rowptr[1:] = np.cumsum([len(c) for c in rows_c])
    return _mat(n, rowptr, np.concatenate(rows_c), np.concatenate(rows_v),
                kind="quasi_triangular", blocks=blocks)


def toeplitz3(n, sub, diag, sup):
    """Tridiagonal Toeplitz tridiag(sub, diag, sup), n x n (nonsymmetric for
    sub != sup)."""
    n_, rp, c, v = _stencil((n,), {(0,): float(diag), (-1,): float(sub), (1,): float(sup)})
    return _mat(n_, rp, c, v, kind="toeplitz3", side=n)


def random200(n=200, per_row=5, diag=10.0, seed=1):
    """n x n random sparse: per row `per_row` distinct off-diagonal columns
    drawn uniformly without replacement from {0..n-1} minus the row, values
    U[-1, 1], plus the diagonal `diag`."""
    rng = np.random.default_rng(seed)
    rows_c, rows_v = [], []
    for i in range(n):
        choices = np.delete(np.arange(n), i)
        c = np.sort(rng.choice(choices, size=per_row, replace=False))
        v = rng.uniform(-1.0, 1.0, size=per_row)
        c = np.append(c, i)
        v = np.append(v, diag)
        o = np.argsort(c, kind="stable")
        rows_c.append(c[o])
        rows_v.append(v[o])
    rowptr = np.zeros(n + 1, np.int64)
    rowptr[1:] = np.cumsum([len(c) for c in rows_c])
    return _mat(n, rowptr, np.concatenate(rows_c), np.concatenate(rows_v), kind="random200")


def _distinct_cols(rng, n, L):
    """Per row i, L[i] distinct columns from {0..n-1} minus {i}, sorted.
    Returns (rows, cols) int64 arrays grouped by row, columns ascending.
    Rows asking for more than half of the n-1 candidates are drawn as a
    random subset directly; the rest by rejection of duplicates."""
    L = np.asarray(L, np.int64)
    dense = np.flatnonzero(L > (n - 1) // 2)
    if dense.size:
        Ls = L.copy()
        Ls[dense] = 0
        rows, cols = _distinct_cols(rng, n, Ls)
        parts_r, parts_c = [rows], [cols]
        for i in dense:
            c = np.sort(rng.choice(n - 1, size=int(L[i]), replace=False))
            c += (c >= i)
            parts_r.append(np.full(c.size, i, np.int64))
            parts_c.append(c)
        r = np.concatenate(parts_r)
        c = np.concatenate(parts_c)
        o = np.lexsort((c, r))
        return r[o], c[o]
    rows = np.repeat(np.arange(n, dtype=np.int64), L)
    c = rng.integers(0, n - 1, size=rows.size, dtype=np.int64)
    c += (c >= rows)
    keys = rows * n + c
    keys.sort()
    while True:
        dup = np.flatnonzero(keys[1:] == keys[:-1]) + 1
        if dup.size == 0:
            break
        r = keys[dup] // n
        cc = rng.integers(0, n - 1, size=dup.size, dtype=np.int64)
        cc += (cc >= r)
        keys[dup] = r * n + cc
        keys.sort()
    return keys // n, keys % n


def powerlaw(n=4_000_000, mean=12.0, sigma=1.5, cap=20000, seed=3, mu_is_log_mean=False):
    """Nonsymmetric power-law matrix ("very unbalanced" rows, Sec. 4.4.1.3).

    Off-diagonal count per row L = min(cap, max(1, round(lognormal(mu, sigma))))
    with the ARITHMETIC mean `mean` (mu = ln(mean) - sigma^2/2; set
    mu_is_log_mean for mu = ln(mean)); columns uniform without replacement
    excluding the row; values U[-1, 1]; diagonal 2 * sum_j |a_ij| (1 if the row
    has no off-diagonal), which makes A strictly diagonally dominant.
    """
    rng = np.random.default_rng(seed)
    mu = math.log(mean) if mu_is_log_mean else math.log(mean) - sigma * sigma / 2.0
    L = np.rint(rng.lognormal(mu, sigma, size=n))
    L = np.clip(L, 1, max(1, min(cap, n - 1))).astype(np.int64)
    if n == 1:
        L[:] = 0
    rows, cols = _distinct_cols(rng, n, L)
    offval = rng.uniform(-1.0, 1.0, size=cols.size)
    keys = rows * n + cols
    diag_keys = np.arange(n, dtype=np.int64) * (n + 1)
    pos = np.searchsorted(keys, diag_keys)
    absum = np.bincount(rows, weights=np.abs(offval), minlength=n)
    dval = np.where(absum > 0, 2.0 * absum, 1.0)
    col = np.insert(cols, pos, np.arange(n, dtype=np.int64))
    val = np.insert(offval, pos, dval)
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(L + 1, out=rowptr[1:])
    return _mat(n, rowptr, col, val, kind="powerlaw", seed=seed)


def random_sym_upper(n, per_row=4, seed=0, diag_shift=1.0):
    """Random symmetric matrix stored as upper triangle: per row up to
    `per_row` distinct columns > i (uniform), values U[-1, 1], diagonal
    diag_shift + 2 * (sum of |off-diagonals| in the full row)."""
    rng = np.random.default_rng(seed)
    ent = []
    for i in range(n):
        k = min(per_row, n - 1 - i)
        if k > 0:
            c = np.sort(rng.choice(np.arange(i + 1, n), size=k, replace=False))
            for j in c:
                ent.append((i, int(j), float(rng.uniform(-1.0, 1.0))))
    absum = np.zeros(n)
    for i, j, v in ent:
        absum[i] += abs(v)
        absum[j] += abs(v)
    ent += [(i, i, diag_shift + 2.0 * absum[i]) for i in range(n)]
    ent.sort()
    rows = np.array([e[0] for e in ent], np.int64)
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return _mat(n, rowptr, [e[1] for e in ent], [e[2] for e in ent], True, kind="randsym")


def random_general(n, lengths, seed=0, diag=None):
    """General CRS with prescribed off-diagonal row lengths `lengths` (array of
    n ints, each <= n-1), uniform distinct columns, values U[-1, 1].  With
    diag=None no diagonal is added; otherwise the diagonal is
    diag + 2*sum|off|.  Used for adversarial row-length shapes."""
    rng = np.random.default_rng(seed)
    L = np.asarray(lengths, np.int64)
    rows, cols = _distinct_cols(rng, n, L) if n > 1 else (np.zeros(0, np.int64),) * 2
    val = rng.uniform(-1.0, 1.0, size=cols.size)
    rowptr = np.zeros(n + 1, np.int64)
    if diag is None:
        np.cumsum(L, out=rowptr[1:])
        return _mat(n, rowptr, cols, val, kind="randgen")
    keys = rows * n + cols
    pos = np.searchsorted(keys, np.arange(n, dtype=np.int64) * (n + 1))
    absum = np.bincount(rows, weights=np.abs(val), minlength=n)
    col = np.insert(cols, pos, np.arange(n, dtype=np.int64))
    val = np.insert(val, pos, diag + 2.0 * absum)
    np.cumsum(L + 1, out=rowptr[1:])
    return _mat(n, rowptr, col, val, kind="randgen")


def full_from_upper(U):
    """Full-storage CRS of U + U^T - diag(U) for an upper-stored matrix
    (pure index/value bookkeeping: every stored (i, j, u) with j != i is
    mirrored to (j, i, u))."""
    n = U["n"]
    rp = U["rowptr"].astype(np.int64)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    cols = U["col"].astype(np.int64)
    vals = U["val"]
    off = cols != rows
    R = np.concatenate([rows, cols[off]])
    Cc = np.concatenate([cols, rows[off]])
    V = np.concatenate([vals, vals[off]])
    o = np.lexsort((Cc, R))
    R, Cc, V = R[o], Cc[o], V[o]
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(R, minlength=n), out=rowptr[1:])
    return _mat(n, rowptr, Cc, V, kind=U.get("kind", "") + "_full")


def to_dense(A):
    """Dense n x n array of a (general or upper-stored) CRS matrix."""
    n = A["n"]
    D = np.zeros((n, n))
    rp = A["rowptr"]
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            D[i, A["col"][k]] = A["val"][k]
            if A["sym_upper"] and A["col"][k] != i:
                D[A["col"][k], i] = A["val"][k]
    return D


def batch_specs(count=512, nmin=1000, nmax=200_000, seed=5):
    """Specs of a batch of uneven systems: n log-uniform on [nmin, nmax]; kind
    k mod 3 = 0: 2D 5-point (side round(sqrt n)), 1: 3D 7-point (side
    round(cbrt n)), 2: power-law recipe with that n (seed derived from k)."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=count))
    specs = []
    for k in range(count):
        n = int(round(ns[k]))
        kind = k % 3
        if kind == 0:
            specs.append(("poisson2d", max(2, int(round(math.sqrt(n))))))
        elif kind == 1:
            specs.append(("laplace3d", max(2, int(round(n ** (1.0 / 3.0))))))
        else:
            specs.append(("powerlaw", n, seed * 100003 + k))
    return specs


def from_spec(spec):
    if spec[0] == "poisson2d":
        return poisson2d(spec[1])
    if spec[0] == "laplace3d":
        return laplace3d(spec[1])
    if spec[0] == "powerlaw":
        return powerlaw(n=spec[1], seed=spec[2])
    raise ValueError(spec)
