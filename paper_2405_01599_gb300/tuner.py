"""Learned tuner: training data from the library's own tuning sweeps, training
with the library's MLP kernels, and evaluation against the exhaustive tuner.

Data: for each generated matrix (seeded recipes spanning the shapes of the
solver workloads: 2D/3D stencils, convection-diffusion, power-law rows with
varied mean/spread, fixed-length random rows, symmetric upper storage; n
log-uniform on [1e3, 2e5]) the library's exhaustive sweep times every SpMV
candidate (variant x CTA size x items per thread; Sec. 3.1: each at most 4
times after a warm-up, minimum kept) and GMRES(m) is timed for each restart
length m in {10, 20, 30, 50, 80, 120} (b = A*ones, x0 = 0, tol 1e-8, capped
time; unconverged runs are extrapolated from their residual reduction).
Labels: the fastest SpMV candidate and the fastest m.  Features: the
library's xb_features (8 floats).

Run on a GPU:  python -m paper_2405_01599_gb300.tuner --make-data 750 --seed 100 --out D.npz
               python -m paper_2405_01599_gb300.tuner --train D.npz --model M.bin
               python -m paper_2405_01599_gb300.tuner --evaluate M.bin --make-data 60 --seed 900
After an SpMV kernel changes, re-time the saved sweeps (the GMRES(m) timings
are kept) and retrain:
               python -m paper_2405_01599_gb300.tuner --resweep D1.npz D2.npz ...
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import time

import numpy as np

from . import gen

GENERAL_CANDS = ([(0, b, 1) for b in (64, 128, 256, 512)] +
                 [(1, b, i) for b in (128, 256, 512) for i in (4, 8, 16)] +
                 [(2, b, i) for b in (128, 256) for i in (4, 8, 16, 32)])
SYM_CANDS = ([(3, b, 1) for b in (128, 256, 512)] +
             [(4, b, i) for b in (128, 256, 512) for i in (4, 8, 16)])
ALL_CANDS = GENERAL_CANDS + SYM_CANDS
RESTARTS = (10, 20, 30, 50, 80, 120)
BLOCKS = (64, 128, 256, 512)
IPTS = (1, 4, 8, 16, 32)
DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
MODEL_PATH = os.path.join(DATA_DIR, "mlp_tuner.bin")
SMALL_CAP_S = 0.1        # per-solve time cap of the GMRES(m) timings


def random_spec(rng, large=False):
    """One matrix recipe, n log-uniform on [1e3, 2e5] (large: [2e5, 5e6] for
    the random kinds, up to 256^3 for the stencils)."""
    if large:
        n = int(math.exp(rng.uniform(math.log(2e5), math.log(5e6))))
    else:
        n = int(math.exp(rng.uniform(math.log(1e3), math.log(2e5))))
    kind = rng.choice(["poisson2d", "laplace3d", "convdiff3d", "powerlaw", "fixedrows",
                       "poisson2d_sym", "laplace3d_sym", "randsym"],
                      p=[0.14, 0.12, 0.12, 0.26, 0.12, 0.08, 0.08, 0.08])
    seed = int(rng.integers(1 << 30))
    if kind in ("poisson2d", "poisson2d_sym"):
        return (kind, max(4, int(round(math.sqrt(n)))))
    if kind in ("laplace3d", "laplace3d_sym", "convdiff3d"):
        side = max(3, int(round(n ** (1 / 3))))
        if large:
            side = int(rng.integers(60, 257))
        return (kind, side)
    if kind == "powerlaw":
        return (kind, n, float(rng.uniform(4, 40)), float(rng.uniform(0.3, 2.0)), seed)
    if kind == "fixedrows":
        return (kind, n, int(rng.integers(2, 64)), seed)
    return (kind, n, int(rng.integers(2, 12)), seed)


def make(spec):
    k = spec[0]
    if k == "poisson2d":
        return gen.poisson2d(spec[1])
    if k == "poisson2d_sym":
        return gen.poisson2d(spec[1], upper=True)
    if k == "laplace3d":
        return gen.laplace3d(spec[1])
    if k == "laplace3d_sym":
        return gen.laplace3d(spec[1], upper=True)
    if k == "convdiff3d":
        return gen.convdiff3d(N=spec[1])
    if k == "powerlaw":
        return gen.powerlaw(n=spec[1], mean=spec[2], sigma=spec[3], seed=spec[4])
    if k == "fixedrows":
        n, L, seed = spec[1], spec[2], spec[3]
        return gen.random_general(n, np.full(n, min(L, n - 1)), seed=seed, diag=1.0)
    if k == "randsym":
        n, per, seed = spec[1], spec[2], spec[3]
        return _randsym_fast(n, per, seed)
    raise ValueError(spec)


def _randsym_fast(n, per, seed):
    """Random symmetric matrix in upper storage (vectorised): per row `per`
    random columns above the diagonal, values U[-1,1], diagonal 1 + 2*|row|."""
    rng = np.random.default_rng(seed)
    L = np.minimum(per, n - 1 - np.arange(n))
    rows = np.repeat(np.arange(n, dtype=np.int64), L)
    span = (n - 1 - rows)
    cols = rows + 1 + (rng.integers(0, 1 << 62, size=rows.size) % np.maximum(span, 1))
    keys = np.unique(rows * n + cols)
    rows, cols = keys // n, keys % n
    vals = rng.uniform(-1, 1, size=rows.size)
    absum = np.bincount(rows, np.abs(vals), minlength=n) + np.bincount(cols, np.abs(vals), minlength=n)
    R = np.concatenate([rows, np.arange(n)])
    Cc = np.concatenate([cols, np.arange(n)])
    V = np.concatenate([vals, 1.0 + 2.0 * absum])
    o = np.lexsort((Cc, R))
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(R, minlength=n), out=rowptr[1:])
    return gen._mat(n, rowptr, Cc[o], V[o], True, kind="randsym")


def record(xb, torch, dev, A, gmres_cap_s=SMALL_CAP_S, gmres_maxiter=1500):
    """Sweep one matrix: features, every SpMV candidate's time, GMRES(m) times."""
    plan = xb.Plan.from_host(A, dev)
    t = [torch.as_tensor(A[k], device=dev) for k in ("rowptr", "col", "val")]
    raw, feat = xb.features(t[0], t[1], t[2], A["sym_upper"])
    t0 = time.perf_counter()
    sw = plan.sweep()
    t_sweep = time.perf_counter() - t0
    times = np.full(len(ALL_CANDS), np.nan)
    for c in sw:
        key = (c["variant"], c["block"], c["ipt"])
        if key in ALL_CANDS:
            times[ALL_CANDS.index(key)] = c["ms"]
    best = ALL_CANDS[int(np.nanargmin(times))]
    plan.set_choice(*best)
    n = A["n"]
    b = torch.empty(n, dtype=torch.float64, device=dev)
    plan.spmv(torch.ones(n, dtype=torch.float64, device=dev), b)
    mt = np.full(len(RESTARTS), np.inf)
    conv = np.zeros(len(RESTARTS), bool)
    for k, m in enumerate(RESTARTS):
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        info = plan.gmres(b, x, m=m, tol=1e-8, maxiter=gmres_maxiter, maxtime_s=gmres_cap_s,
                          check_every=10)
        ts = info["t_solve_s"]
        res = info["res_true"]
        if info["status"] == 0:
            mt[k] = ts
            conv[k] = True
        elif 0.0 < res < 1.0:
            mt[k] = ts * math.log(1e-8) / math.log(res)
    return dict(raw=raw, feat=feat, times=times, mtimes=mt, mconv=conv, t_sweep=t_sweep, best=best)


def make_data(count, seed, dev="cuda", log_every=50, large=False):
    import torch

    import paper_2405_01599_gb300 as xb
    xb.build()
    rng = np.random.default_rng(seed)
    recs, specs = [], []
    t0 = time.perf_counter()
    for i in range(count):
        spec = random_spec(rng, large)
        A = make(spec)
        if large:  # cap each GMRES(m) timing; unconverged runs are extrapolated
            recs.append(record(xb, torch, torch.device(dev), A, gmres_cap_s=0.6, gmres_maxiter=600))
        else:
            recs.append(record(xb, torch, torch.device(dev), A))
        specs.append(repr(spec))
        if log_every and (i + 1) % log_every == 0:
            print(f"[tuner data] {i + 1}/{count} matrices, {time.perf_counter() - t0:.0f}s", flush=True)
    return dict(feat=np.stack([r["feat"] for r in recs]).astype(np.float32),
                raw=np.stack([r["raw"] for r in recs]),
                times=np.stack([r["times"] for r in recs]),
                mtimes=np.stack([r["mtimes"] for r in recs]),
                mconv=np.stack([r["mconv"] for r in recs]),
                t_sweep=np.array([r["t_sweep"] for r in recs]),
                specs=np.array(specs))


def resweep(D, dev="cuda", log_every=100):
    """Re-time every SpMV candidate of a saved dataset with the current
    kernels (the matrices are regenerated from their recorded recipes); the
    GMRES(m) timings are kept.  Returns a new dataset."""
    import ast

    import torch

    import paper_2405_01599_gb300 as xb
    xb.build()
    out = {k: np.array(v, copy=True) for k, v in D.items()}
    t0 = time.perf_counter()
    for s, spec in enumerate(D["specs"]):
        # recipes were saved as repr() of tuples whose strings may print as np.str_('...')
        A = make(ast.literal_eval(re.sub(r"np\.\w+\(([^()]*)\)", r"\1", str(spec))))
        plan = xb.Plan.from_host(A, torch.device(dev))
        t1 = time.perf_counter()
        sw = plan.sweep()
        out["t_sweep"][s] = time.perf_counter() - t1
        times = np.full(len(ALL_CANDS), np.nan)
        for c in sw:
            key = (c["variant"], c["block"], c["ipt"])
            if key in ALL_CANDS:
                times[ALL_CANDS.index(key)] = c["ms"]
        out["times"][s] = times
        del plan
        if log_every and (s + 1) % log_every == 0:
            print(f"[tuner resweep] {s + 1}/{len(D['specs'])} matrices, "
                  f"{time.perf_counter() - t0:.0f}s", flush=True)
    return out


def remeasure_m(D, cap_s=4.0, kinds=("poisson2d", "laplace3d", "convdiff3d", "fixedrows",
                                      "poisson2d_sym", "laplace3d_sym", "randsym"),
                dev="cuda", log_every=10):
    """Re-time GMRES(m) for every m of the saved records of the given kinds
    with a per-solve cap of cap_s (SpMV choice: the record's fastest
    candidate), marking which runs converged; other records are kept.
    Returns a new dataset with an "m_full" flag per record (1 = re-timed, its
    converged runs are labels whatever the matrix size)."""
    import ast

    import torch

    import paper_2405_01599_gb300 as xb
    xb.build()
    out = {k: np.array(v, copy=True) for k, v in D.items()}
    if "mconv" not in out:  # older sweeps: a run converged when it beat the 0.6 s cap
        out["mconv"] = np.isfinite(out["mtimes"]) & (out["mtimes"] < 0.6)
    out["m_full"] = np.zeros(len(D["specs"]), np.int32)
    t0 = time.perf_counter()
    done = 0
    for s, spec in enumerate(D["specs"]):
        sp = ast.literal_eval(re.sub(r"np\.\w+\(([^()]*)\)", r"\1", str(spec)))
        if sp[0] not in kinds:
            continue
        A = make(sp)
        plan = xb.Plan.from_host(A, torch.device(dev))
        t = D["times"][s]
        plan.set_choice(*ALL_CANDS[int(np.nanargmin(t))])
        n = A["n"]
        b = torch.empty(n, dtype=torch.float64, device=dev)
        plan.spmv(torch.ones(n, dtype=torch.float64, device=dev), b)
        for k, m in enumerate(RESTARTS):
            x = torch.zeros(n, dtype=torch.float64, device=dev)
            info = plan.gmres(b, x, m=m, tol=1e-8, maxiter=1_000_000, maxtime_s=cap_s,
                              check_every=10)
            conv = info["status"] == 0
            out["mconv"][s, k] = conv
            out["mtimes"][s, k] = info["t_solve_s"] if conv else np.inf
        out["m_full"][s] = 1
        del plan
        done += 1
        if log_every and done % log_every == 0:
            print(f"[tuner m] {done} matrices re-timed, {time.perf_counter() - t0:.0f}s", flush=True)
    return out


M_LABEL_MAX_N = 200_000  # above this the m timings are capped extrapolations


def labels_of(D):
    """Head labels: (variant, CTA-size class, ipt class, m class).  The m label
    is -1 (left out of the loss) for matrices larger than M_LABEL_MAX_N: their
    GMRES(m) timings were cut short, and extrapolating a capped run favours
    small m, whose restarted iteration stalls later."""
    N = D["feat"].shape[0]
    lab = np.zeros((N, 4), np.int32)
    for s in range(N):
        v, b, i = ALL_CANDS[int(np.nanargmin(D["times"][s]))]
        lab[s] = (v, BLOCKS.index(b), IPTS.index(i), m_label(D, s))
    return lab


def m_label(D, s):
    """Fastest restart length among the runs that converged within the cap
    (capped runs are extrapolations, which favour small m); -1 when none did
    or the matrix is above M_LABEL_MAX_N."""
    full = "m_full" in D and D["m_full"][s]
    if D["raw"][s][0] > M_LABEL_MAX_N and not full:
        return -1
    mt = D["mtimes"][s]
    conv = D["mconv"][s] if "mconv" in D else (mt < SMALL_CAP_S)
    if not conv.any():
        return -1
    return int(np.argmin(np.where(conv, mt, np.inf)))


def n_records(D):
    return int(np.isfinite(D["times"]).sum() + np.isfinite(D["mtimes"]).sum())


def train_model(D, epochs=400, batch=128, lr=3e-3, seed=0, dev="cuda"):
    import torch

    import paper_2405_01599_gb300 as xb
    X = D["feat"].astype(np.float32)
    mu = X.mean(axis=0)
    sd = X.std(axis=0)
    sd[sd < 1e-3] = 1.0
    model = xb.Mlp(seed=seed)
    model.set_norm(mu, sd)
    Xt = torch.tensor(X, device=dev)
    Lt = torch.tensor(labels_of(D), device=dev)
    loss = model.train(Xt, Lt, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return model, loss


def evaluate(model, D, dev="cuda"):
    """Regret of the learned choice vs the exhaustive optimum and gain over the
    fixed default (no tuning), per matrix, for SpMV time and GMRES time."""
    import torch
    X = torch.tensor(D["feat"].astype(np.float32), device=dev)
    pred = model.predict(X)
    lab = labels_of(D)
    out = dict(spmv_regret=[], spmv_gain_vs_default=[], m_regret=[], m_gain_vs_default=[],
               variant_acc=float(np.mean(pred[:, 0] == lab[:, 0])))
    # variants whose best launch shape is within 5% of the optimum are ties:
    # picking any of them costs at most 5%
    near = []
    for s in range(len(pred)):
        t = D["times"][s]
        best_v = {}
        for k, c in enumerate(ALL_CANDS):
            if np.isfinite(t[k]):
                best_v[c[0]] = min(best_v.get(c[0], np.inf), t[k])
        near.append(best_v.get(int(pred[s, 0]), np.inf) <= 1.05 * np.nanmin(t))
    out["variant_acc_within_5pct"] = float(np.mean(near))
    for s in range(len(pred)):
        t = D["times"][s]
        sym = bool(D["raw"][s][6]) and np.isnan(t[:len(GENERAL_CANDS)]).all()
        # the library's choice logic: masked arg-max, nearest supported shape
        v = int(pred[s, 0])
        ok_v = (3, 4) if sym else (0, 1, 2)
        if v not in ok_v:
            v = ok_v[0]
        cands = [k for k, c in enumerate(ALL_CANDS) if c[0] == v and np.isfinite(t[k])]
        want_b, want_i = BLOCKS[pred[s, 1]], IPTS[pred[s, 2]]
        k = min(cands, key=lambda q: (ALL_CANDS[q][1] != want_b) + (ALL_CANDS[q][2] != want_i))
        t_ml = t[k]
        t_best = np.nanmin(t)
        dflt = (4, 256, 8) if sym else ((2, 256, 8) if D["raw"][s][4] > 64 and D["raw"][s][4] > 16 * D["raw"][s][2] else (1, 256, 8))
        t_def = t[ALL_CANDS.index(dflt)]
        out["spmv_regret"].append(float(t_ml / t_best))
        out["spmv_gain_vs_default"].append(float(t_def / t_ml))
        if m_label(D, s) >= 0:
            mt = D["mtimes"][s]
            m_ml = mt[pred[s, 3]]
            out["m_regret"].append(float(m_ml / mt[m_label(D, s)]))
            out["m_gain_vs_default"].append(float(mt[RESTARTS.index(30)] / m_ml))
    summ = {k: (float(np.exp(np.mean(np.log(v)))) if isinstance(v, list) and v else v)
            for k, v in out.items()}
    return summ, out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--make-data", type=int, default=0)
    ap.add_argument("--large", action="store_true", help="matrices with n in [2e5, 5e6]")
    ap.add_argument("--seed", type=int, default=100)
    ap.add_argument("--out", default=None)
    ap.add_argument("--train", nargs="*", default=None, help="dataset(s) to concatenate")
    ap.add_argument("--model", default=None)
    ap.add_argument("--evaluate", default=None)
    ap.add_argument("--evaluate-data", default=None,
                    help="saved held-out sweep (.npz) for --evaluate instead of --make-data")
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--resweep", nargs="*", default=None,
                    help="re-time the SpMV candidates of saved datasets in place")
    ap.add_argument("--remeasure-m", nargs="*", default=None,
                    help="re-time GMRES(m) of saved large-matrix records (4 s cap) in place")
    a = ap.parse_args()
    D = None
    for f in a.resweep or ():
        R = resweep(dict(np.load(f)))
        np.savez_compressed(f, **R)
        print(f"[tuner resweep] {f}: {len(R['feat'])} matrices re-timed")
    for f in a.remeasure_m or ():
        R = remeasure_m(dict(np.load(f)))
        np.savez_compressed(f, **R)
        print(f"[tuner m] {f}: {int(R['m_full'].sum())} records re-timed")
    if a.make_data:
        D = make_data(a.make_data, a.seed, large=a.large)
        print(f"[tuner data] {n_records(D)} timing records from {len(D['feat'])} matrices")
        if a.out:
            np.savez_compressed(a.out, **D)
    if a.train:
        parts = [dict(np.load(f)) for f in a.train]
        for p_ in parts:
            if "mconv" not in p_:
                p_["mconv"] = p_["mtimes"] < (SMALL_CAP_S if p_["raw"][:, 0].max() <= M_LABEL_MAX_N
                                              else 0.6)
        for p_ in parts:
            if "m_full" not in p_:
                p_["m_full"] = np.zeros(len(p_["feat"]), np.int32)
        Dt = {k: np.concatenate([p_[k] for p_ in parts]) for k in parts[0]}
        print(f"[tuner train] {n_records(Dt)} timing records from {len(Dt['feat'])} matrices")
        model, loss = train_model(Dt, epochs=a.epochs)
        print(f"[tuner train] {len(Dt['feat'])} samples, final loss {loss:.4f}")
        if a.model:
            model.save(a.model)
        summ, _ = evaluate(model, Dt)
        print("[tuner train-set]", json.dumps(summ))
    if a.evaluate:
        import paper_2405_01599_gb300 as xb
        model = xb.Mlp.load(a.evaluate)
        if D is None and a.evaluate_data:
            D = dict(np.load(a.evaluate_data))
        if D is None:
            raise SystemExit("--evaluate needs --make-data (held-out matrices)")
        summ, _ = evaluate(model, D)
        print("[tuner held-out]", json.dumps(summ))


if __name__ == "__main__":
    main()
