#!/usr/bin/env python
"""Benchmark of the CRS SpMV + Krylov hot path on GB300.

Headline (one JSON line on rank 0): achieved HBM GB/s of the auto-tuned FP64
SpMV y = A x on the power-law matrix of the unbalanced-rows workload
(n = 4,000,000, lognormal row lengths with arithmetic mean 12, sigma 1.5, cap
20,000, uniform random columns, diagonal 2 * row |sum|; ~52M non-zeros,
~0.70 GB of algorithmic traffic per SpMV, so every step streams more than
the 129 MB L2).  GB/s counts algorithmic bytes: 12 B per non-zero (value +
column index), rowptr once, x once, y once.

--impl reference times the CPU oracle's SpMV on the same matrix with the same
metric: its OpenMP build, the rows split statically over all host cores (the
paper's row decomposition U1 on the CPU).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMV HBM GB/s vs peak; GMRES time-to-1e-8, tuned/mixed vs plain FP64"
WORKLOAD = ("power-law CRS n=4,000,000 (lognormal rows mean 12 sigma 1.5 cap 20k, "
            "uniform columns, diagonal 2x row |sum|), FP64, y = A x")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=4_000_000)
    ap.add_argument("--no-extras", action="store_true", help="skip per-variant/sym/solver lines")
    ap.add_argument("--no-solvers", action="store_true",
                    help="skip the GMRES time-to-1e-8 comparison (256^3 convection-diffusion)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 512-system batch (config 5)")
    ap.add_argument("--batch-rule-arms", action="store_true",
                    help="batch: also the arms with the restart-frequency rule (Eq. 1)")
    ap.add_argument("--variant", default=None,
                    choices=["row", "nnz", "segscan", "sym-atomic", "sym-tile", "sell"],
                    help="fixed SpMV variant instead of the exhaustive tuner")
    ap.add_argument("--block", type=int, default=256)
    ap.add_argument("--ipt", type=int, default=8)
    ap.add_argument("--profile-only", action="store_true",
                    help="only warm-up + timed steps (for ncu captures); prints a short line")
    ap.add_argument("--matrix", default="c3",
                    choices=["c3", "c2-upper", "c2-full", "c4", "c4-160", "c2-box"],
                    help="profile-only: power-law n (c3), 128^3 Laplacian upper/full (c2), "
                         "256^3 (c4) or 160^3 (c4-160) convection-diffusion, 120 x 128 x 136 "
                         "convection-diffusion box (c2-box)")
    ap.add_argument("--gmres-steps", type=int, default=0,
                    help="profile-only: run this many GMRES(30) Arnoldi steps instead of SpMVs")
    ap.add_argument("--eig-restarts", type=int, default=0,
                    help="profile-only: run this many restarts of Arnoldi (nev 10, m 40)")
    ap.add_argument("--ortho", default="mgs", choices=["mgs", "cgs", "dgks", "bcgs"],
                    help="profile-only GMRES / Arnoldi: orthogonalisation")
    ap.add_argument("--ilu", action="store_true",
                    help="profile-only GMRES: ILU(0) right preconditioning")
    ap.add_argument("--mixed", action="store_true",
                    help="profile-only GMRES: FP32 inner solve in FP64 refinement (one outer "
                         "step of --gmres-steps inner steps)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
         "utilization.gpu")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        def rd():
            for line in self.proc.stdout:
                self.rows.append([c.strip() for c in line.split(",")])
        self.t = threading.Thread(target=rd, daemon=True)
        self.t.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, busy, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for k, nm in enumerate(names):
                    if r[4 + k].lower().startswith("active"):
                        reasons.add(nm)
                if float(r[8]) >= 50:
                    busy.append(float(r[0]))
            except Exception:
                continue
        use = busy if busy else sm
        return {"sm_mhz": float(np.median(use)) if use else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "samples_under_load": len(busy),
                "reasons": sorted(reasons)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, pg, dev=None):
    """The slowest rank's time: replicas run concurrently, so the job takes as
    long as its slowest rank (pg: torch.distributed or None)."""
    if pg is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=dev if dev is not None else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws, bytes_per_step, ms_per_step):
    """Whole-job GB/s: every one of the ws ranks moved bytes_per_step per step."""
    return ws * bytes_per_step / (ms_per_step * 1e-3) / 1e9


def make_c3(n):
    from paper_2405_01599_gb300 import gen
    return gen.powerlaw(n=n, seed=3)


def alg_bytes(A, vb=8, beta=False):
    n, nnz = A["n"], A["nnz"]
    return (vb + 4) * nnz + 4 * (n + 1) + 2 * vb * n + (vb * n if beta else 0)


# DRAM bytes (read + write) of one headline SpMV launch (k_bss) from an ncu capture,
# keyed by (variant, block, ipt, n, nnz) and valid only while the code that launch
# ran is unchanged: the sha256 of the segmented-scan kernels, their launcher and the
# row-store helper (csrc/spmv.cu) and of the plan builders of their row-end bitmask,
# warp start rows and BSS data format copy (csrc/plan.cu; not the host-side
# clean-up of unused copies), as cut out by HEADLINE_SRC below.  The
# capture and its command are summarised in profiles/.
NCU_TRAFFIC = {
    ("segscan", 128, 8, 4_000_000, 52_238_581):
        (707.47e6, "a24e7aa087f91861d8c824d106efd10128028785ec457e2eb9cb5686caf38a48"),
}
HEADLINE_SRC = [
    ("spmv.cu", "__device__ __forceinline__ void store_row(", "// U1: one thread per row"),
    ("spmv.cu", "// U3 (BSS) with the plan's row-end bitmask", "// S1-like baseline"),
    ("spmv.cu", "int launch_seg(", "int launch_sym("),
    ("plan.cu", "__global__ void k_seg_rows(", "void bss_trim("),
    ("plan.cu", "const SegPart *get_segs(", "__global__ void k_to_f32("),
]


def headline_src_hash():
    import hashlib
    parts = []
    for fname, start, end in HEADLINE_SRC:
        with open(os.path.join(ROOT, "paper_2405_01599_gb300", "csrc", fname)) as f:
            src = f.read()
        i = src.find(start)
        j = src.find(end, i + 1) if i >= 0 else -1
        if i < 0 or j < 0:
            return None
        parts.append(src[i:j])
    return hashlib.sha256("\0".join(parts).encode()).hexdigest()


def ncu_traffic(choice_name, block, ipt, n, nnz):
    ent = NCU_TRAFFIC.get((choice_name, block, ipt, n, nnz))
    if ent is None or headline_src_hash() != ent[1]:
        return None
    return ent[0]


def host_cpu():
    """The host's CPU model, vendor and logical core count (lscpu, else
    /proc/cpuinfo)."""
    info = {"model": None, "vendor": None, "nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            key, _, val = line.partition(":")
            if key.strip() == "Model name" and info["model"] is None:
                info["model"] = val.strip()
            elif key.strip() == "Vendor ID" and info["vendor"] is None:
                info["vendor"] = val.strip()
    except Exception:
        pass
    if info["model"] is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        info["model"] = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return info


def cpu_oracle_rate(A, budget_s=10.0, max_nnz=None, omp=False):
    """Time the oracle's SpMV on a row block (one core, or the OpenMP build's
    row-parallel loop over every host core); median of the runs."""
    import oracle
    rp = A["rowptr"]
    n = A["n"]
    if max_nnz is not None and A["nnz"] > max_nnz:
        r1 = int(np.searchsorted(rp, max_nnz, side="right")) - 1
        r1 = max(1, r1)
    else:
        r1 = n
    sub = dict(n=r1, nnz=int(rp[r1]), rowptr=np.ascontiguousarray(rp[: r1 + 1]),
               col=A["col"], val=A["val"], sym_upper=False)
    x = np.random.default_rng(0).uniform(-1, 1, n)
    y = np.zeros(r1)
    L = oracle.lib_omp() if omp else oracle.lib()
    times = []
    t_end = time.perf_counter() + budget_s
    while True:
        t0 = time.perf_counter()
        L.orc_spmv(r1, sub["rowptr"], A["col"], A["val"], 1.0, x, 0.0, y)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() > t_end or len(times) >= 50:
            break
    t = float(np.median(times))
    return alg_bytes(sub) / t / 1e9, t, sub, len(times), L.orc_num_threads()


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    A = make_c3(args.n)
    L = oracle.lib_omp()
    n = A["n"]
    x = np.random.default_rng(0).uniform(-1, 1, n)
    y = np.zeros(n)
    # one step: the oracle's SpMV over the whole matrix, rows split over all host
    # cores (the OpenMP build of the plain loops)
    for _ in range(args.warmup):
        L.orc_spmv(n, A["rowptr"], A["col"], A["val"], 1.0, x, 0.0, y)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        L.orc_spmv(n, A["rowptr"], A["col"], A["val"], 1.0, x, 0.0, y)
    el = time.perf_counter() - t0
    val = alg_bytes(A) * args.steps / el / 1e9
    threads = L.orc_num_threads()
    sample = (f"the whole n=4M power-law SpMV per step ({A['nnz']} non-zeros), rows split "
              f"statically over {threads} OpenMP threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": val, "unit": "GB/s", "cores": threads, "kind": "oracle",
                         "sample": sample, "cpu": host_cpu()},
        "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    ws, rank, local = dist_init()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    import torch
    import paper_2405_01599_gb300 as xb
    xb.build()
    xb.lib()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    stream = torch.cuda.current_stream()

    if args.profile_only and args.matrix != "c3":
        from paper_2405_01599_gb300 import gen
        A = {"c2-upper": lambda: gen.laplace3d(128, upper=True), "c2-full": lambda: gen.laplace3d(128),
             "c4": lambda: gen.convdiff3d(N=256),
             "c4-160": lambda: gen.convdiff3d(N=160),
             "c2-box": lambda: gen.convdiff3d(128, pe=10.0, dims=(120, 128, 136))}[args.matrix]()
    else:
        A = make_c3(args.n)
    n, nnz = A["n"], A["nnz"]
    plan = xb.Plan.from_host(A, dev)
    if args.variant:
        v = {"row": xb.VAR_ROW, "nnz": xb.VAR_NNZ, "segscan": xb.VAR_SEGSCAN, "sell": xb.VAR_SELL,
             "sym-atomic": xb.VAR_SYM_ATOMIC, "sym-tile": xb.VAR_SYM_TILE}[args.variant]
        plan.set_choice(v, args.block, args.ipt)
        choice = plan.choice()
    else:
        choice = plan.tune()
    if args.profile_only and args.eig_restarts:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, _, ainfo = plan.arnoldi(nev=10, m=40, tol=1e-30, maxrestart=args.eig_restarts,
                                    vectors=False,
                                    ortho=["mgs", "cgs", "dgks", "bcgs"].index(args.ortho))
        el = time.perf_counter() - t0
        if rank == 0:
            print(json.dumps({"profile_only": True, "matrix": args.matrix,
                              "arnoldi_steps": ainfo["steps"], "restarts": ainfo["restarts"],
                              "s": el, "choice": choice}))
        return
    if args.profile_only and args.gmres_steps:
        bvec = torch.empty(n, dtype=torch.float64, device=dev)
        plan.spmv(torch.ones(n, dtype=torch.float64, device=dev), bvec)
        xg = torch.zeros(n, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        extra = dict(precision=xb.PREC_MIXED, tol_inner=1e-30, maxiter_inner=args.gmres_steps,
                     max_outer=1) if args.mixed else {}
        if args.ilu:
            plan.ilu0_setup()
            extra["precond"] = xb.PRECOND_ILU0
        info = plan.gmres(bvec, xg, m=30, tol=1e-30, maxiter=args.gmres_steps, check_every=10,
                          ortho=["mgs", "cgs", "dgks", "bcgs"].index(args.ortho), **extra)
        el = time.perf_counter() - t0
        if rank == 0:
            print(json.dumps({"profile_only": True, "matrix": args.matrix,
                              "gmres_steps": info["iters"] or info["inner_iters"],
                              "s": el, "GBs_solve": info["bytes_alg"] / el / 1e9, "choice": choice}))
        return
    x = torch.tensor(np.random.default_rng(0).uniform(-1, 1, n), device=dev)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    bytes_step = alg_bytes(A)
    launches_per_spmv = 2 if choice["variant"] == xb.VAR_SEGSCAN else 1

    for _ in range(max(3, args.warmup)):
        plan.spmv(x, y)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    clocks = Clocks(local)
    clocks.start()
    # untimed load phase (~1 s of the same SpMV) so the clock samples see the GPU busy
    # right before and during the timed steps
    t_load = time.perf_counter() + (0.0 if args.profile_only else 1.0)
    while time.perf_counter() < t_load:
        for _ in range(50):
            plan.spmv(x, y)
        torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        ev[2 * k].record(stream)
        plan.spmv(x, y)
        ev[2 * k + 1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clk = clocks.stop()
    total_ms = t0.elapsed_time(t1)
    per_launch = [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(args.steps)]
    avg_launch_ms = float(np.mean(per_launch))
    total_ms = max_over_ranks(total_ms, pg, dev)
    ms_step = total_ms / args.steps
    value = job_rate(ws, bytes_step, ms_step)
    if args.profile_only:
        if rank == 0:
            print(json.dumps({"profile_only": True, "n": n, "nnz": nnz, "choice": choice,
                              "ms_per_step": ms_step, "GBs": value}))
        if pg:
            pg.destroy_process_group()
        return

    # end to end through the C ABI with host buffers: every step copies its x from
    # pinned host memory, runs the SpMV and copies its y back.  Steps are
    # pipelined the way an application streaming independent inputs would run
    # them: H2D of step k, SpMV of step k-1 and D2H of step k-2 overlap on three
    # streams (double-buffered device vectors, ordered by events).
    xh = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(2)]
    for h in xh:
        h.copy_(x.cpu())
    yh = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(2)]
    xd = [torch.empty_like(x) for _ in range(2)]
    yd = [torch.empty_like(y) for _ in range(2)]
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()

    def e2e_run(k_steps):
        ev = lambda: torch.cuda.Event(enable_timing=False)
        h2d = [ev() for _ in range(k_steps)]
        cmp = [ev() for _ in range(k_steps)]
        d2h = [ev() for _ in range(k_steps)]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s_in)
        s_cmp.wait_event(e0)
        s_out.wait_event(e0)
        for k in range(k_steps):
            b = k % 2
            with torch.cuda.stream(s_in):
                if k >= 2:
                    s_in.wait_event(cmp[k - 2])   # xd[b] read by the SpMV of step k-2
                xd[b].copy_(xh[b], non_blocking=True)
                h2d[k].record(s_in)
            s_cmp.wait_event(h2d[k])
            if k >= 2:
                s_cmp.wait_event(d2h[k - 2])      # yd[b] copied out by step k-2
            plan.spmv(xd[b], yd[b], stream=s_cmp)
            cmp[k].record(s_cmp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(cmp[k])
                yh[b].copy_(yd[b], non_blocking=True)
                d2h[k].record(s_out)
        s_out.wait_event(d2h[-1])
        e1.record(s_out)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    e2e_run(3)
    e2e_ms = max_over_ranks(e2e_run(args.steps), pg, dev) / args.steps
    e2e_val = job_rate(ws, bytes_step, e2e_ms)
    e2e_check = float((yd[(args.steps - 1) % 2] - y).abs().max().item())  # same x, same y

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    peak, peak_kind = peaks()
    achieved = bytes_step / (avg_launch_ms * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "nnz": nnz,
                   "spmv_choice": {"variant": xb.VARIANT_NAMES[choice["variant"]],
                                   "block": choice["block"], "ipt": choice["ipt"]},
                   "alg_bytes_per_step": bytes_step,
                   "l2": "inputs larger than L2 (0.70 GB streamed per step > 129 MB)",
                   "clocks_window": "1 s untimed load phase of the same SpMV, then the timed steps",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": ncu_traffic(xb.VARIANT_NAMES[choice["variant"]], choice["block"],
                                            choice["ipt"], n, nnz),
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "kernel": "spmv (" + xb.VARIANT_NAMES[choice["variant"]] + ")"},
        "e2e": {"value": e2e_val, "unit": "GB/s", "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * n, "ms_per_step": e2e_ms,
                "pipelined": "H2D / SpMV / D2H of consecutive steps overlap on 3 streams",
                "max_abs_diff_vs_device_run": e2e_check},
        "gpu_launches": launches_per_spmv * args.steps,
        "clocks": clk,
    }
    if ws == 1:
        gbs, t, sub, reps, thr = cpu_oracle_rate(A, budget_s=6.0, omp=True)
        g1, t1, _, reps1, _ = cpu_oracle_rate(A, budget_s=6.0)
        out["cpu_baseline"] = {
            "value": gbs, "unit": "GB/s", "cores": thr, "kind": "oracle",
            "sample": f"the whole n=4M SpMV, rows split over {thr} OpenMP threads "
                      f"(the oracle's OpenMP build), median of {reps} runs",
            "single_core": {"value": g1, "unit": "GB/s", "cores": 1,
                            "sample": f"the whole n=4M SpMV, plain oracle, median of {reps1} runs"},
            "cpu": host_cpu()}
    if not args.no_extras:
        args.sm_mhz = clk.get("sm_mhz")
        out["extras"] = extras(xb, torch, dev, plan, A, x, y, args)
    print(json.dumps(out))
    if pg:
        pg.destroy_process_group()


def _time_spmv(torch, fn, reps=20):
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def extras(xb, torch, dev, plan, A, x, y, args):
    from paper_2405_01599_gb300 import gen
    import oracle
    res = {}
    b3 = alg_bytes(A)
    var = {}
    for name, v, blk, ipt in [("row_U1", 0, 256, 1), ("nnz_U2", 1, 128, 8),
                              ("nnz_U2_b256", 1, 256, 8), ("segscan_U3", 2, 128, 8),
                              ("segscan_U3_b256", 2, 256, 8), ("segscan_U3_i16", 2, 128, 16)]:
        ms = _time_spmv(torch, lambda: plan.spmv(x, y, variant=v, block=blk, ipt=ipt))
        var[name] = {"ms": ms, "GBs": b3 / ms / 1e6}
    var["ratios"] = {"segscan_U3_vs_row_U1": var["row_U1"]["ms"] / var["segscan_U3"]["ms"],
                     "nnz_U2_vs_row_U1": var["row_U1"]["ms"] / var["nnz_U2"]["ms"],
                     "paper_T2K_16_threads": "U3/U1 4.62x on trans4 (Sec. 4.4.1.3), "
                                             "U2/U1 2.8x on epb3 (Sec. 4.4.1.2)"}
    res["c3_variants"] = var
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (args.sm_mhz or 2070.0)
    fp64_peak = 2.0 * nsm * mhz * 1e6  # FP64 FMA lanes per second: 2 per clock per SM
    # config 2: 3D 7-point Laplacian 128^3, symmetric upper storage vs full
    U = gen.laplace3d(128, upper=True)
    F = gen.laplace3d(128)
    pu = xb.Plan.from_host(U, dev)
    pf = xb.Plan.from_host(F, dev)
    cu = pu.tune()
    cf = pf.tune()
    n2 = U["n"]
    x2 = torch.ones(n2, dtype=torch.float64, device=dev)
    y2 = torch.empty_like(x2)
    reps = 200
    ms_sym = _time_spmv(torch, lambda: pu.spmv(x2, y2), reps)
    ms_full = _time_spmv(torch, lambda: pf.spmv(x2, y2), reps)
    ms_sym_atomic = _time_spmv(torch, lambda: pu.spmv(x2, y2, variant=3, block=256, ipt=1), reps)
    bs = 12 * U["nnz"] + 4 * (n2 + 1) + 16 * n2
    bf = alg_bytes(F)
    flops = 2 * F["nnz"]
    # FP64 pipe operations per SpMV: symmetric (alpha = 1) = one FMA per stored
    # entry for the row sum plus one multiply per stored off-diagonal for its
    # transpose term; full storage = one FMA per entry.  Equal counts.
    ops_sym = 2 * U["nnz"] - n2
    ops_full = F["nnz"]
    fp = lambda ops, ms: {"ops": ops, "achieved_G": ops / ms / 1e6, "peak_G": fp64_peak / 1e9,
                          "frac": ops / (ms * 1e-3) / fp64_peak}
    res["c2_sym_vs_full"] = {
        "sym_tuned": {"choice": cu, "ms": ms_sym, "GBs": bs / ms_sym / 1e6, "GFLOPs": flops / ms_sym / 1e6,
                      "fp64": fp(ops_sym, ms_sym)},
        "sym_atomic_S1": {"ms": ms_sym_atomic, "GBs": bs / ms_sym_atomic / 1e6,
                          "fp64": fp(ops_sym, ms_sym_atomic)},
        "full_tuned": {"choice": cf, "ms": ms_full, "GBs": bf / ms_full / 1e6, "GFLOPs": flops / ms_full / 1e6,
                       "fp64": fp(ops_full, ms_full)},
        "200_spmv_ms": {"sym": 200 * ms_sym, "full": 200 * ms_full},
        "sym_speedup_vs_full": ms_full / ms_sym,
        "fp64_peak_note": f"2 FMA lanes/clk/SM x {nsm} SMs x {mhz:.0f} MHz (sampled SM clock)",
    }
    # format-conversion AT (Sec. 5): a 27-point stencil (128^3, 56M nnz), where
    # the tuner converts to SELL-32-sigma; every general variant's throughput
    try:
        S27 = gen.stencil27(128)
        p27 = xb.Plan.from_host(S27, dev)
        c27 = p27.tune()
        x27 = torch.ones(S27["n"], dtype=torch.float64, device=dev)
        y27 = torch.empty_like(x27)
        b27 = alg_bytes(S27)
        t27 = {}
        for lab, (v, b, i) in {"row": (xb.VAR_ROW, 256, 1), "nnz": (xb.VAR_NNZ, 256, 8),
                               "segscan": (xb.VAR_SEGSCAN, 256, 8),
                               "sell_s32": (xb.VAR_SELL, 128, 1),
                               "sell_s1024": (xb.VAR_SELL, 128, 32)}.items():
            ms = _time_spmv(torch, lambda: p27.spmv(x27, y27, variant=v, block=b, ipt=i), 50)
            t27[lab] = {"ms": ms, "GBs": b27 / ms / 1e6}
        res["stencil27_128_spmv"] = {"tuned": {"variant": xb.VARIANT_NAMES[c27["variant"]],
                                               "block": c27["block"], "ipt": c27["ipt"]},
                                     "variants": t27}
        del p27, S27, x27, y27
    except xb.XbError as e:
        res["stencil27_128_spmv"] = {"error": str(e)}
    # format-conversion AT with blocks: a 3D 7-point grid with 3 unknowns per
    # node and dense 3 x 3 coupling blocks (elasticity-like; 80^3 nodes, n =
    # 1.5M, 32M non-zeros), where the tuner may convert to BCSR
    try:
        B3 = gen.block_stencil3d(80, 3)
        pb = xb.Plan.from_host(B3, dev)
        cb = pb.tune()
        xb3 = torch.ones(B3["n"], dtype=torch.float64, device=dev)
        yb3 = torch.empty_like(xb3)
        bb = alg_bytes(B3)
        tb = {}
        for lab, (v, b, i) in {"row": (xb.VAR_ROW, 128, 1), "nnz": (xb.VAR_NNZ, 128, 8),
                               "segscan": (xb.VAR_SEGSCAN, 128, 8), "sell_s32": (xb.VAR_SELL, 128, 1),
                               "bcsr_2x2": (xb.VAR_BCSR, 128, 2), "bcsr_3x3": (xb.VAR_BCSR, 128, 3),
                               "bcsr_4x4": (xb.VAR_BCSR, 128, 4)}.items():
            try:
                ms = _time_spmv(torch, lambda: pb.spmv(xb3, yb3, variant=v, block=b, ipt=i), 50)
                tb[lab] = {"ms": ms, "GBs_crs_bytes": bb / ms / 1e6}
            except xb.XbError as e:
                tb[lab] = {"rejected": str(e)}
        res["block3d_dof3_80_spmv"] = {
            "n": B3["n"], "nnz": B3["nnz"],
            "tuned": {"variant": xb.VARIANT_NAMES[cb["variant"]], "block": cb["block"], "ipt": cb["ipt"]},
            "variants": tb,
            "note": "GB/s over the CRS algorithmic bytes (12 B per non-zero); a 3x3 BCSR copy reads "
                    "8 B per non-zero plus one column index per 9"}
        del pb, B3, xb3, yb3
    except xb.XbError as e:
        res["block3d_dof3_80_spmv"] = {"error": str(e)}
    # restarted Lanczos (OpenATI_EIGENSOLVE): the 10 largest eigenvalues of the
    # 128^3 Laplacian (upper storage), as the paper asks for 10 eigenpairs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = 1.0 / 129.0
    top = 6.0 + 6.0 * np.cos(np.pi * h)  # closed-form largest eigenvalue
    for label, kw in (("c2_lanczos_nev10_m40", {}), ("c2_lanczos_nev10_m20_rule", dict(m_max=120))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, _, linfo = pu.lanczos(nev=10, m=40 if not kw else 20, tol=1e-8, vectors=False, **kw)
        torch.cuda.synchronize()
        res[label] = {"s": time.perf_counter() - t0, "status": linfo["status"],
                      "steps": linfo["steps"], "restarts": linfo["restarts"],
                      "m_final": linfo["m_final"],
                      "max_resid_rel": float(np.max(linfo["resid"] / np.abs(ev))),
                      "lambda_max": float(ev[0]),
                      "lambda_max_err_vs_closed_form": float(abs(ev[0] - top))}
    # restarted Arnoldi (OpenATI_EIGENSOLVE, unsymmetric): the 10 eigenvalues of
    # largest real part of a 120 x 128 x 136 convection-diffusion box (n = 2.09M,
    # distinct side lengths so that no eigenvalue is multiple), BCGS as in the
    # paper's restart experiment; fixed m = 40 against m = 20 with the rule
    CB = gen.convdiff3d(128, pe=10.0, dims=(120, 128, 136))
    pc = xb.Plan.from_host(CB, dev)
    pc.tune()
    ph = 10.0 / 129.0
    lam_top = sum(2.0 + ph + 2.0 * np.sqrt(1.0 + ph) * np.cos(np.pi / (side + 1.0))
                  for side in (120, 128, 136))  # closed form: real spectrum, sum over the axes
    for label, kw in (("c2_arnoldi_convdiff_box_nev10_m40_bcgs", dict(m=40)),
                      ("c2_arnoldi_convdiff_box_nev10_m20_rule_bcgs", dict(m=20, m_max=120))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, _, ainfo = pc.arnoldi(nev=10, tol=1e-8, vectors=False, ortho=xb.ORTHO_BCGS, **kw)
        torch.cuda.synchronize()
        res[label] = {"s": time.perf_counter() - t0, "status": ainfo["status"],
                      "steps": ainfo["steps"], "restarts": ainfo["restarts"],
                      "m_final": ainfo["m_final"],
                      "max_resid_rel": float(np.max(ainfo["resid"] / np.abs(ev))),
                      "lambda_max": float(ev[0].real),
                      "lambda_max_err_vs_closed_form": float(abs(ev[0] - lam_top)),
                      "max_abs_imag": float(np.max(np.abs(ev.imag)))}
    # the numerical computation policies on the same eigenproblem (the paper's
    # Fig. 9-11: time, memory and accuracy of Arnoldi under each policy)
    pol = {}
    for name, code in (("TIME", xb.POLICY_TIME), ("MEMORY", xb.POLICY_MEMORY),
                       ("ACCURACY", xb.POLICY_ACCURACY), ("STABLE", xb.POLICY_STABLE)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, _, ainfo = pc.arnoldi(nev=10, m=40, tol=1e-8, vectors=False, policy=code,
                                  maxrestart=3000)
        torch.cuda.synchronize()
        pol[name] = {"s": time.perf_counter() - t0, "status": ainfo["status"],
                     "steps": ainfo["steps"], "restarts": ainfo["restarts"],
                     "m_final": ainfo["m_final"], "ortho_used": ainfo["ortho_used"],
                     "outer": ainfo["outer"], "mem_GB": ainfo["mem_bytes"] / 1e9,
                     "true_resid_max": ainfo["true_resid"],
                     "lambda_max_err_vs_closed_form": float(abs(ev[0] - lam_top))}
    res["c2_arnoldi_convdiff_box_policies"] = pol
    del pc, CB
    # FP64 roof of the block Gram-Schmidt pass kernel: one BCGS orthogonalisation
    # of a vector against 32 basis rows at the 256^3 size (n = 16.8M) through the
    # library's xb_orth; FMA lanes = n (2k + 1) (k dots, k updates, the norm)
    ng = 256 ** 3
    kk = 32
    # random unit rows of length 16.8M are orthogonal to ~1/sqrt(n) = 2.4e-4:
    # orthonormal enough for a timing
    Vb = torch.randn(kk, ng, dtype=torch.float64, device=dev)
    Vb /= Vb.norm(dim=1, keepdim=True)
    w0 = torch.randn(ng, dtype=torch.float64, device=dev)
    wk = torch.empty_like(w0)
    ms_o = {}
    for nm, code in (("bcgs", xb.ORTHO_BCGS), ("cgs", xb.ORTHO_CGS), ("mgs", xb.ORTHO_MGS)):
        def one():
            wk.copy_(w0)
            plan.orth(Vb, wk, code)
        for _ in range(2):
            one()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ec0, ec1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record()
        for _ in range(reps):
            one()
        e1.record()
        ec0.record()
        for _ in range(reps):
            wk.copy_(w0)
        ec1.record()
        torch.cuda.synchronize()
        ms = (e0.elapsed_time(e1) - ec0.elapsed_time(ec1)) / reps
        ops = ng * (2 * kk + 1)
        ms_o[nm] = {"ms": ms, "fp64": fp(ops, ms)}
    res["orth_fp64_roof_n16.8M_k32"] = ms_o
    del Vb, w0, wk
    # config 1: 64x64 Poisson GMRES(30) to 1e-8, b = A*ones, x0 = 0
    P = gen.poisson2d(64)
    pp = xb.Plan.from_host(P, dev)
    bp_h = oracle.spmv(P, np.ones(P["n"]))
    bp = torch.tensor(bp_h, device=dev)
    t_c1 = time.perf_counter()
    xo, io = oracle.gmres(P, bp_h, m=30, tol=1e-8)
    t_c1 = time.perf_counter() - t_c1
    cpu = {"c1_gmres30": {"s": t_c1, "iters": io["iters"], "cores": 1,
                          "kind": "plain oracle, run to convergence"}}
    res["cpu_oracle"] = cpu
    # the library's default path for a system this small is one persistent
    # launch from one cluster's shared memory (persistent = 2); the batched
    # kernel's single-system path (persistent = 1, XB_RESIDENT_CL=0) and the
    # multi-launch path (small_n = 0; host checks every check_every Arnoldi
    # steps) are timed beside it
    for label, kw, env in (("c1_gmres30_persistent", {}, None),
                           ("c1_gmres30_persistent_bcgs", dict(ortho=xb.ORTHO_BCGS), None),
                           ("c1_gmres30_batched_kernel", {}, "0"),
                           ("c1_gmres30_multilaunch_check1", dict(small_n=0, check_every=1), None),
                           ("c1_gmres30_multilaunch_check8", dict(small_n=0, check_every=8), None)):
        old_env = os.environ.pop("XB_RESIDENT_CL", None)
        if env is not None:
            os.environ["XB_RESIDENT_CL"] = env
        try:
            xs = torch.zeros(P["n"], dtype=torch.float64, device=dev)
            pp.gmres(bp, xs, m=30, tol=1e-8, **kw)  # warm-up (workspace, module load)
            best = None
            for _ in range(3):
                xs.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                info = pp.gmres(bp, xs, m=30, tol=1e-8, **kw)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                best = dt if best is None else min(best, dt)
        finally:
            os.environ.pop("XB_RESIDENT_CL", None)
            if old_env is not None:
                os.environ["XB_RESIDENT_CL"] = old_env
        res[label] = {"s": best, "iters": info["iters"], "oracle_iters": io["iters"],
                      "persistent": info["persistent"], "ortho": info["ortho_used"],
                      "res_true": info["res_true"], "status": info["status"],
                      "us_per_step": 1e6 * best / max(1, info["iters"])}
    xs = torch.zeros(P["n"], dtype=torch.float64, device=dev)
    info = pp.gmres(bp, xs, m=30, tol=1e-8, precision=xb.PREC_MIXED, check_every=8)
    res["c1_gmres30_mixed"] = {"iters_inner": info["inner_iters"], "outer": info["outer"],
                               "res_true": info["res_true"],
                               "err_vs_fp64_oracle": float(np.max(np.abs(xs.cpu().numpy() - xo)) /
                                                           np.max(np.abs(xo)))}
    if not args.no_solvers:
        res.update(solvers(xb, torch, dev, plan, A, args, cpu))
    if not args.no_batch:
        res["c5_batch"] = batch(xb, torch, dev, args, cpu)
    return res


def solvers(xb, torch, dev, plan3, A3, args, cpu):
    """Time to true ||b - A x|| / ||b|| <= 1e-8 (b = A*ones, x0 = 0); the CPU
    oracle's time for the same solves (OpenMP build, all host cores) where it
    finishes in seconds, else per-iteration times scaled to the GPU's
    iteration counts (labelled extrapolated)."""
    import oracle
    from paper_2405_01599_gb300 import gen, tuner
    out = {}
    # config 3: BiCGStab on the power-law matrix (tuned SpMV)
    n3 = A3["n"]
    b3 = torch.empty(n3, dtype=torch.float64, device=dev)
    plan3.spmv(torch.ones(n3, dtype=torch.float64, device=dev), b3)
    x3 = torch.zeros(n3, dtype=torch.float64, device=dev)
    t0 = time.perf_counter()
    info = plan3.bicgstab(b3, x3, tol=1e-8, maxtime_s=120.0, check_every=4)
    out["c3_bicgstab"] = {"s": time.perf_counter() - t0, "iters": info["iters"],
                          "res_true": info["res_true"], "status": info["status"],
                          "spmv_calls": info["spmv_calls"]}
    # the same solve right-preconditioned by ILU(0), as the paper runs its
    # solvers (Sec. 4.3); setup (levels + factorization) timed separately
    x3.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan3.ilu0_setup()
    torch.cuda.synchronize()
    t_ilu = time.perf_counter() - t0
    t0 = time.perf_counter()
    info = plan3.bicgstab(b3, x3, tol=1e-8, maxtime_s=120.0, check_every=1,
                          precond=xb.PRECOND_ILU0)
    torch.cuda.synchronize()
    out["c3_bicgstab_ilu0"] = {"s": time.perf_counter() - t0, "setup_s": t_ilu,
                               "iters": info["iters"], "res_true": info["res_true"],
                               "status": info["status"]}
    # CPU oracle, BiCGStab on the same matrix: a bounded number of iterations
    # of the OpenMP build, per-iteration time x the GPU's iteration count
    b3h = oracle.spmv(A3, np.ones(n3), omp=True)
    k, el = 2, 0.0
    while True:
        t0 = time.perf_counter()
        _, ci = oracle.bicgstab(A3, b3h, tol=1e-30, maxiter=k, omp=True)
        el = time.perf_counter() - t0
        if el > 4.0 or k >= 256:
            break
        k *= 4
    per_it = el / max(1, ci["iters"])
    cpu["c3_bicgstab"] = {"per_iteration_s": per_it, "iterations_timed": ci["iters"],
                          "s_extrapolated": per_it * out["c3_bicgstab"]["iters"],
                          "gpu_iters": out["c3_bicgstab"]["iters"],
                          "cores": oracle.lib_omp().orc_num_threads(),
                          "kind": "extrapolated: OpenMP oracle per-iteration time x GPU iterations"}
    # config 4: 256^3 convection-diffusion, Peclet 10, upwind
    A = gen.convdiff3d(N=256, pe=10.0)
    n = A["n"]
    model = xb.Mlp.load(tuner.MODEL_PATH)
    ones = torch.ones(n, dtype=torch.float64, device=dev)

    def run(label, plan, **kw):
        b = torch.empty(n, dtype=torch.float64, device=dev)
        plan.spmv(ones, b)
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = plan.gmres(b, x, tol=1e-8, maxtime_s=300.0, check_every=10, timing=1, **kw)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        err = float((x - ones).abs().max().item())
        mixed = kw.get("precision") == xb.PREC_MIXED
        timed = info["inner_iters"] + info["outer"] if mixed else info["spmv_calls"]
        out[label] = {"s": el, "status": info["status"], "iters": info["iters"] or info["inner_iters"],
                      "outer": info["outer"], "inner_iters": info["inner_iters"],
                      "fallback": info["fallback"], "fp64_iters_after_fallback": info["iters"] if mixed else None,
                      "res_true": info["res_true"],
                      "err_vs_exact_solution": err, "spmv_calls": info["spmv_calls"],
                      "GBs_solve": info["bytes_alg"] / el / 1e9,
                      "spmv_ms_avg": info["spmv_ms"] / max(1, timed),
                      "spmv_timed": "FP32 inner SpMVs" if mixed else "every SpMV",
                      "variant": xb.VARIANT_NAMES.get(info["variant_used"], "?"),
                      "ortho_used": ["mgs", "cgs", "dgks", "bcgs"][info["ortho_used"]],
                      "block": info["block_used"], "ipt": info["ipt_used"], **kw}

    p_plain = xb.Plan.from_host(A, dev)           # no tuning: the plan's default variant
    run("c4_plain_fp64_m30", p_plain, m=30)
    p_ex = xb.Plan.from_host(A, dev)
    t0 = time.perf_counter()
    p_ex.tune()
    t_ex = time.perf_counter() - t0
    run("c4_exhaustive_fp64_m30", p_ex, m=30)
    out["c4_exhaustive_fp64_m30"]["tune_s"] = t_ex
    # the accuracy policy (Sec. 3.3.2) picks the orthogonalisation: BCGS at tol 1e-8
    run("c4_exhaustive_fp64_m30_policy", p_ex, m=30, ortho=xb.ORTHO_AUTO)
    p_ml = xb.Plan.from_host(A, dev)
    t0 = time.perf_counter()
    ch, m = p_ml.tune_mlp(model)
    t_ml = time.perf_counter() - t0
    run("c4_mlp_fp64", p_ml, m=m, ortho=xb.ORTHO_AUTO)
    run("c4_mlp_mixed", p_ml, m=m, precision=xb.PREC_MIXED, tol_inner=1e-4, maxiter_inner=2000,
        ortho=xb.ORTHO_AUTO)
    out["c4_mlp_mixed"]["tune_s"] = t_ml
    out["c4_mlp_fp64"]["tune_s"] = t_ml
    # ILU(0)-preconditioned FP64 GMRES (the paper's setting): 6x fewer iterations,
    # but each substitution walks the 3N-2 = 766 wavefront levels of the stencil
    t0 = time.perf_counter()
    p_ex.ilu0_setup()
    torch.cuda.synchronize()
    t_ilu4 = time.perf_counter() - t0
    run("c4_exhaustive_fp64_m30_ilu0", p_ex, m=30, ortho=xb.ORTHO_AUTO, precond=xb.PRECOND_ILU0)
    out["c4_exhaustive_fp64_m30_ilu0"]["setup_s"] = t_ilu4
    # ILU(0)-preconditioned BiCGStab (FP64): the fastest FP64 solve of this problem
    b4 = torch.empty(n, dtype=torch.float64, device=dev)
    p_ex.spmv(ones, b4)
    x4 = torch.zeros(n, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = p_ex.bicgstab(b4, x4, tol=1e-8, maxtime_s=120.0, check_every=1,
                         precond=xb.PRECOND_ILU0)
    torch.cuda.synchronize()
    out["c4_exhaustive_bicgstab_ilu0"] = {"s": time.perf_counter() - t0, "iters": info["iters"],
                                          "res_true": info["res_true"], "status": info["status"],
                                          "setup_s": t_ilu4}
    # CPU oracle: one GMRES(30) cycle (30 Arnoldi steps with MGS) of the OpenMP
    # build, x the cycles the untuned FP64 GPU solve needed
    b4h = b4.cpu().numpy()
    t0 = time.perf_counter()
    _, c4i = oracle.gmres(A, b4h, m=30, tol=1e-30, maxiter=30, omp=True)
    t_cyc = time.perf_counter() - t0
    cyc = out["c4_plain_fp64_m30"]["iters"] / 30.0
    cpu["c4_gmres30"] = {"cycle_s": t_cyc, "steps_timed": c4i["iters"], "gpu_cycles": cyc,
                         "s_extrapolated": t_cyc * cyc, "cores": oracle.lib_omp().orc_num_threads(),
                         "kind": "extrapolated: one OpenMP oracle GMRES(30) cycle x the GPU's cycles"}
    del b4h
    # numerical computation policies (Sec. 2.3.2, 3.3) on the 128^3 problem: time,
    # memory and accuracy of each
    A2 = gen.convdiff3d(N=128, pe=10.0)
    n2 = A2["n"]
    ones2 = torch.ones(n2, dtype=torch.float64, device=dev)
    pol = {}
    for name, code in (("time", xb.POLICY_TIME), ("accuracy", xb.POLICY_ACCURACY),
                       ("memory", xb.POLICY_MEMORY), ("stable", xb.POLICY_STABLE)):
        pp = xb.Plan.from_host(A2, dev)
        b2 = torch.empty(n2, dtype=torch.float64, device=dev)
        pp.spmv(ones2, b2)
        x2 = torch.zeros(n2, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = pp.gmres(b2, x2, tol=1e-8, maxtime_s=120.0, check_every=10, policy=code)
        torch.cuda.synchronize()
        pol[name] = {"s": time.perf_counter() - t0, "status": info["status"],
                     "iters": info["iters"], "m_final": info["m_final"],
                     "res_true": info["res_true"], "mem_GB": info["mem_bytes"] / 1e9,
                     "variant": xb.VARIANT_NAMES.get(info["variant_used"], "?"),
                     "ortho_used": ["mgs", "cgs", "dgks", "bcgs"][info["ortho_used"]]}
    out["c4_128_policies"] = pol
    base = out["c4_plain_fp64_m30"]["s"]
    out["c4_speedup_vs_plain_fp64"] = {k: base / out[k]["s"] for k in
                                       ("c4_exhaustive_fp64_m30", "c4_exhaustive_fp64_m30_policy",
                                        "c4_mlp_fp64", "c4_mlp_mixed")}
    fp64_runs = ("c4_plain_fp64_m30", "c4_exhaustive_fp64_m30", "c4_exhaustive_fp64_m30_policy",
                 "c4_mlp_fp64", "c4_exhaustive_fp64_m30_ilu0", "c4_exhaustive_bicgstab_ilu0")
    ok64 = [k for k in fp64_runs if out[k]["status"] == 0]
    fastest = min(ok64, key=lambda k: out[k]["s"]) if ok64 else None
    mx = out["c4_mlp_mixed"]["s"]
    out["c4_mixed_speedup"] = {
        "vs_plain_fp64_untuned": base / mx,
        "vs_exhaustive_fp64_mgs": out["c4_exhaustive_fp64_m30"]["s"] / mx,
        "vs_exhaustive_fp64_policy": out["c4_exhaustive_fp64_m30_policy"]["s"] / mx,
        "vs_mlp_fp64_same_m_and_ortho": out["c4_mlp_fp64"]["s"] / mx,
        "vs_fastest_fp64": (out[fastest]["s"] / mx) if fastest else None,
        "fastest_fp64": fastest,
        "mixed_fallback": out["c4_mlp_mixed"]["fallback"]}
    return out


def batch(xb, torch, dev, args, cpu):
    """512 uneven systems in one persistent graph-captured launch: untuned
    default vs the exhaustive run-time tuner (each system's SpMV candidates
    timed, Sec. 3.1; m fixed at 30) vs the learned tuner (SpMV choice and m).
    Throughput of a launch: algorithmic bytes and flops summed over the
    systems' Arnoldi steps (one SpMV plus the MGS passes of the step at the
    cycle's mean basis size) over the launch time."""
    import oracle
    from paper_2405_01599_gb300 import gen, tuner
    specs = gen.batch_specs(512, seed=5)
    model = xb.Mlp.load(tuner.MODEL_PATH)
    systems, plans, shapes = [], [], []
    t_ml = t_ex = 0.0
    # the batched kernel's two in-CTA SpMV forms: thread per row (the U1
    # counterpart) and warp-sized row blocks with warp- and CTA-wide long rows
    # (the counterpart of the nnz-balanced U2 and U3); a tuned system takes
    # the form of the family its tuner chose
    mode_of = lambda v: 1 if v in (xb.VAR_NNZ, xb.VAR_SEGSCAN) else 0
    for sp in specs:
        A = gen.from_spec(sp)
        pl = xb.Plan.from_host(A, dev)
        n = A["n"]
        b = torch.empty(n, dtype=torch.float64, device=dev)
        pl.spmv(torch.ones(n, dtype=torch.float64, device=dev), b)
        t0 = time.perf_counter()
        ch, m = pl.tune_mlp(model)
        t_ml += time.perf_counter() - t0
        t0 = time.perf_counter()
        ce = pl.tune()
        t_ex += time.perf_counter() - t0
        systems.append(dict(rowptr=pl._keep[0], col=pl._keep[1], val=pl._keep[2], b=b,
                            x=torch.zeros(n, dtype=torch.float64, device=dev),
                            m_ml=m, mode_ml=mode_of(ch["variant"]), mode_ex=mode_of(ce["variant"])))
        plans.append(pl)
        shapes.append((n, A["nnz"]))
    # per-system cap: the power-law systems of this mix stagnate without a
    # preconditioner; the cap bounds their share of the launch
    opts = dict(tol=1e-8, maxiter=3000, maxtime_s=60.0)

    def run(ms, modes, **kw):
        for q, m, md in zip(systems, ms, modes):
            q["m"], q["mode"] = int(m), int(md)
        bt = xb.Batch(systems, **opts, **kw)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bt.run()
        e1.record()
        r = bt.results()
        bt.close()
        return e0.elapsed_time(e1), r

    N = len(systems)

    def thru(r, t_ms):
        by = fl = 0.0
        for (n, nnz), q in zip(shapes, r):
            jm = (q["m"] + 1) / 2.0  # mean basis size of a cycle's step
            steps = q["iters"]
            by += steps * ((12 * nnz + 4 * (n + 1) + 16 * n) + (4 * jm + 5) * 8 * n)
            fl += steps * (2 * nnz + 4 * n * (jm + 1))
        return {"GBs": by / (t_ms * 1e-3) / 1e9, "GFLOPs": fl / (t_ms * 1e-3) / 1e9,
                "alg_GB": by / 1e9, "arnoldi_steps": int(sum(q["iters"] for q in r))}

    # MGS in every arm: inside the batched kernel (one SM per small system,
    # latency-bound) BCGS measured no faster than MGS
    t_def, r_def = run([30] * N, [0] * N)
    t_exh, r_exh = run([30] * N, [q["mode_ex"] for q in systems])
    t_mlp, r_mlp = run([q["m_ml"] for q in systems], [q["mode_ml"] for q in systems])
    ok = lambda r: int(sum(1 for q in r if q["status"] == 0))
    # systems every arm solved: their summed per-system device times compare the
    # tuners on work that finished (systems that hit the cap all ran 3000 steps)
    both = [k for k in range(N) if r_def[k]["status"] == 0 and r_exh[k]["status"] == 0
            and r_mlp[k]["status"] == 0]
    cs = lambda r: float(sum(r[k]["ms"] for k in both))
    # CPU oracle on a seeded sample of the same systems (one core, GMRES(30),
    # the same 3000-step cap), scaled by the summed row counts to all 512
    rng = np.random.default_rng(55)
    order = rng.permutation(N)
    t_cpu, n_cpu, solved, done = 0.0, 0, 0, []
    for k in order:
        if t_cpu > 15.0:
            break
        A = gen.from_spec(specs[k])
        bh = oracle.spmv(A, np.ones(A["n"]))
        t0 = time.perf_counter()
        _, oi = oracle.gmres(A, bh, m=30, tol=1e-8, maxiter=3000)
        t_cpu += time.perf_counter() - t0
        n_cpu += A["n"]
        solved += oi["status"] == 0
        done.append(int(k))
    sum_n = int(sum(q["b"].numel() for q in systems))
    cpu["c5_batch"] = {"systems_timed": len(done), "s_timed": t_cpu, "converged_timed": int(solved),
                       "s_extrapolated": t_cpu * sum_n / max(n_cpu, 1), "cores": 1,
                       "kind": "extrapolated: plain oracle GMRES(30) on a seeded sample, "
                               "scaled by summed rows to all 512 systems"}
    res = {"systems": N, "sum_n": sum_n,
            "launch_ms": {"default": t_def, "exhaustive": t_exh, "learned": t_mlp},
            "throughput": {"default": thru(r_def, t_def), "exhaustive": thru(r_exh, t_exh),
                           "learned": thru(r_mlp, t_mlp)},
            "learned_tune_s": t_ml, "exhaustive_tune_s": t_ex,
            "converged": {"default": ok(r_def), "exhaustive": ok(r_exh), "learned": ok(r_mlp)},
            "solved_by_all": len(both),
            "solved_by_all_sum_ms": {"default": cs(r_def), "exhaustive": cs(r_exh),
                                     "learned": cs(r_mlp)},
            "learned_speedup_on_solved_by_all": {"vs_default": cs(r_def) / max(cs(r_mlp), 1e-9),
                                                 "vs_exhaustive": cs(r_exh) / max(cs(r_mlp), 1e-9)},
            "launch_speedup_learned": {"vs_default": t_def / t_mlp, "vs_exhaustive": t_exh / t_mlp},
            "max_system_ms": {"default": max(q["ms"] for q in r_def),
                              "exhaustive": max(q["ms"] for q in r_exh),
                              "learned": max(q["ms"] for q in r_mlp)}}
    # tuning included: each arm's tuning time plus its launch
    res["launch_plus_tune_s"] = {"default": t_def * 1e-3, "exhaustive": t_ex + t_exh * 1e-3,
                                 "learned": t_ml + t_mlp * 1e-3}
    res["launch_plus_tune_speedup_learned"] = {
        "vs_exhaustive": (t_ex + t_exh * 1e-3) / (t_ml + t_mlp * 1e-3),
        "vs_default": (t_def * 1e-3) / (t_ml + t_mlp * 1e-3)}
    # per-system regret of the learned choice against the exhaustive one on
    # the systems both solve (device time of the system's solve)
    ratios = np.array([r_mlp[i]["ms"] / max(r_exh[i]["ms"], 1e-9) for i in both])
    if ratios.size:
        res["learned_regret_vs_exhaustive_per_system"] = {
            "systems": int(ratios.size), "geomean": float(np.exp(np.mean(np.log(ratios)))),
            "median": float(np.median(ratios)), "p90": float(np.percentile(ratios, 90)),
            "faster_or_equal": int(np.sum(ratios <= 1.0))}
    if args.batch_rule_arms:
        # the paper's full run-time AT: SpMV choice before execution plus the
        # restart-frequency rule during it (m starts at 30, grows by 5 up to 128),
        # and the learned choices as the starting point of the same rule
        t_exr, r_exr = run([30] * N, [q["mode_ex"] for q in systems], dafrt=1, m_max=128,
                           dafrt_theta=10.0)
        t_mlr, r_mlr = run([q["m_ml"] for q in systems], [q["mode_ml"] for q in systems],
                           dafrt=1, m_max=128, dafrt_theta=10.0)
        res["exhaustive_with_restart_rule"] = {"launch_ms": t_exr, "converged": ok(r_exr),
                                               "solved_by_all_sum_ms": cs(r_exr)}
        res["learned_with_restart_rule"] = {"launch_ms": t_mlr, "converged": ok(r_mlr),
                                            "solved_by_all_sum_ms": cs(r_mlr)}
    return res


if __name__ == "__main__":
    main()
