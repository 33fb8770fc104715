"""Benchmark: time to a 1e-10 relative residual of the CG-accelerated block Cimmino solve
(setup + solve) and HBM GB/s per CG iteration, FP64 vs FP32+refinement, on one GB300.

Workload (default, --config 3): a random sparse nonsymmetric system, n = 2^20, 8
off-diagonal entries per row at uniform columns with N(0,1) values, diagonal = 1.2 x the
row's absolute sum (seed 3), f = A x_true with x_true ~ U[-1, 1]; K = 512 blocks of
exactly 2048 rows from the graph partition of the row inner-product graph (Section 2),
computed once before the timed region.  A step = one full pass of the hot path: row
scaling + permutation, A^T, C = A A^T, Gram blocks, batched Cholesky, then Algorithm 2 to
||f - A x|| <= 1e-10 ||f||, with A and f already resident in HBM.  `value` is the FP64
time to solution; FP32 factors + FP64 refinement are timed beside it on the same blocks.

Further legs (each timed with CUDA events, clocks sampled): contiguous blocks of the same
workload, the 64^3 convection-diffusion system against the stored oracle solution, and the
128^3 system with 16 right-hand sides (one full FP32+refine solve, FP64 per iteration over
a fixed window).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own copy of the workload (replicas only: the
solve does not shard); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-10 rel. residual & HBM GB/s per CG iter; FP32+refine vs FP64 on GB300"
TOL = 1e-10
FP64_PEAK_TFLOPS = 1.25  # GB300 FP64 rate (nominal, 152 SMs at 2070 MHz)
# DRAM bytes per launch from one ncu capture of the current kernels (dram__bytes_read.sum +
# dram__bytes_write.sum); None where the kernel changed since its capture
TRAFFIC = {"k_proj_fp64_convdiff3d_64": 659753728, "k_proj_fp32_convdiff3d_64": 726496512,
           "k_proj_fp64_random_dd_n1048576_k8_K512": 3138300000,
           "k_proj_fp32_random_dd_n1048576_k8_K512": 3357500000,
           "k_cholesky_fp64_random_dd_n1048576_k8_K512": 5032485376}
GOLDEN = os.path.join(ROOT, "tests", "golden")
# projection configurations measured by the library's autotuner during the warm-up steps
# and reused (from this file) by every later setup of the run
TUNE_CACHE = os.path.join(tempfile.gettempdir(), f"cimmino_tune_{os.getpid()}.txt")


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling (SM clock, throttle reasons) during a timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None
        self.path = os.path.join(tempfile.gettempdir(),
                                 f"cimmino_clocks_{os.getpid()}_{index}_{id(self)}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [t.strip() for t in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "power_w_median": statistics.median(pw) if pw else None, "samples": len(rows)}


def max_over_ranks(value, device=None):
    """The largest value over all ranks of the default process group (every rank gets it);
    the value itself in a single process.  Replicas report the slowest rank's time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def algorithmic_bytes(n, nnz, factor_bytes, refine_mean, nnz_gram):
    """Minimum bytes one CG iteration must move (1 right-hand side).

    projection: one solve pass streams pass_bytes ~ 2 x factor_bytes (N tiles and
      inv(L_II) for the forward solve, their transposed copies for the backward solve),
      times (1 + refinement steps); each refinement step also reads the exact Gram blocks
      (12 B per entry); u read, y written.
    u = A p with the residual of x: CSR (12 B/entry + 8 B/row), p and x gathered, f_s and d
      read, u written.
    psi = A^T y with p^T psi: transpose (12 B/entry + 8 B/column), y gathered, p read, psi
      written.
    x, r update (4 read, 2 written) and p update (2 read, 1 written).
    """
    proj = (1 + refine_mean) * 2 * factor_bytes + refine_mean * 12 * nnz_gram + 16 * n
    spmv = 12 * nnz + 8 * n + 16 * n + 16 * n + 8 * n
    spmv_t = 12 * nnz + 8 * n + 8 * n + 8 * n + 8 * n
    upd = 6 * 8 * n + 3 * 8 * n
    return {"proj": proj, "iteration": proj + spmv + spmv_t + upd}


# ------------------------------------------------------------------ workloads and partitions

DEFAULT_PARTITION = {1: "contiguous", 2: "contiguous", 3: "graph", 5: "contiguous"}


EXACT_BALANCE = (3, 5)  # blocks of exactly 2048 rows; the 64^3 system allows 5% imbalance


def partition_of(w, partition, config, use_gpu=True):
    """Blocks of the workload: its contiguous blocks, or the graph partition of its row
    inner-product graph (Section 2) with the same K.  Caps: exact balance (n / K rows) for
    the random and 128^3 workloads, 5% imbalance otherwise."""
    import paper_1710_07769_gb300 as g
    K = len(w.block_ptr) - 1
    n = w.A.n
    if partition == "contiguous":
        return w.perm, w.block_ptr, {"partition": "contiguous", "cap": int(np.diff(w.block_ptr).max())}
    cap = n // K if config in EXACT_BALANCE and n % K == 0 else int(math.floor(1.05 * n / K))
    t0 = time.perf_counter()
    if use_gpu:
        C = g.aat(w.A)
    else:
        import oracle
        C = oracle.aat_plain(w.A)
    t_aat = time.perf_counter() - t0
    t0 = time.perf_counter()
    perm, bp, cut = g.partition_rip(n, C, K, cap=cap, seed=0)
    t_part = time.perf_counter() - t0
    return perm, bp, {"partition": "graph", "cap": cap, "aat_s": round(t_aat, 3),
                      "partition_s": round(t_part, 2), "cutsize": round(cut, 2),
                      "block_rows_min": int(np.diff(bp).min()),
                      "block_rows_max": int(np.diff(bp).max())}


def config_dict(w, part, layout, args):
    return {"workload": w.name, "n": int(w.A.n), "nnz": int(w.A.nnz),
            "K": int(len(w.block_ptr) - 1), "partition": part["partition"], "cap": part["cap"],
            "layout": layout, "tol": TOL, "precision": "fp64 (value); fp32_refine beside",
            "x0": "zero", "l2": "flushed (512 MB write) before every timed step",
            "parallelism": "replicas" if args.gpus > 1 else "single"}


# ------------------------------------------------------------------ our arm

class DevCSR:
    pass


def to_device(A, dev):
    import torch
    d = DevCSR()
    d.n = A.n
    d.row_ptr = torch.from_numpy(A.row_ptr).to(dev)
    d.col_idx = torch.from_numpy(A.col_idx).to(dev)
    d.val = torch.from_numpy(A.val).to(dev)
    return d


class Runner:
    """Timed steps of one workload and partition on the library's stream."""

    def __init__(self, w, perm, bp, layout, dev, stream, flush):
        import torch
        self.w, self.perm, self.bp, self.layout = w, perm, bp, layout
        self.dev, self.stream, self.flush = dev, stream, flush
        self.dA = to_device(w.A, dev)
        self.dF = torch.from_numpy(np.ascontiguousarray(w.F[0])).to(dev)
        self.dX = torch.empty_like(self.dF)
        torch.cuda.synchronize()

    def step(self, precision, **kw):
        import torch

        import paper_1710_07769_gb300 as g
        with torch.cuda.stream(self.stream):
            s = g.Solver(self.dA, self.bp, perm=self.perm, precision=precision,
                         layout=self.layout, tune=True, tune_cache=TUNE_CACHE, **kw)
            x, st, code = s.solve(self.dF, tol=TOL, X=self.dX)
        return s, st[0], code

    def timed(self, precision, k, warm, **kw):
        """warm untimed steps, then k steps each bracketed by CUDA events on the stream (L2
        flushed by a 512 MB write before each).  Returns (ms list, last (solver, stats, code))."""
        import torch
        for _ in range(warm):
            s, st, code = self.step(precision, **kw)
            s.close()
        times, last = [], None
        for _ in range(k):
            with torch.cuda.stream(self.stream):
                self.flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(self.stream)
            s, st, code = self.step(precision, **kw)
            with torch.cuda.stream(self.stream):
                e1.record(self.stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            if last is not None:
                last[0].close()
            last = (s, st, code)
        return times, last

    def x_host(self):
        import torch
        torch.cuda.synchronize()
        return self.dX.cpu().numpy().copy()

    def proj_live(self, precision):
        """Average device time of the projection launches inside the CG loop of one more
        solve (CUDA events on the library's stream around every projection launch,
        iterations launched eagerly), and the isolated back-to-back figure beside it."""
        s, st, code = self.step(precision, time_proj=True)
        ms, nl = s.proj_timing()
        kt = s.time_kernels(reps=10)
        s.close()
        kt["proj_ms_isolated"] = kt["proj_ms"]
        kt["proj_ms"] = ms / max(1, nl)
        kt["proj_launches_timed"] = nl
        return kt


def rel_err(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def leg_summary(r, st, times, kt, x, n, nnz, nblk):
    launches = st["iters"] + 1
    refine_mean = st["refine_steps_total"] / max(1, nblk * (launches + 1))
    b = algorithmic_bytes(n, nnz, st["pass_bytes"] / 2, refine_mean, st["nnz_gram"])
    it_ms = st["t_solve_ms"] / max(1, launches)
    out = {"time_to_solution_ms": round(sum(times) / len(times), 3), "steps": len(times),
           "iters": st["iters"], "rel_res": st["rel_res"], "backward_err": st["backward_err"],
           "setup_ms": round(st["t_setup_ms"], 3), "factor_ms": round(st["t_factor_ms"], 3),
           "cholesky_ms": round(st["t_chol_ms"], 3), "solve_ms": round(st["t_solve_ms"], 3),
           "per_iter_ms": round(it_ms, 4),
           "hbm_gbps_per_iter": round(b["iteration"] / (it_ms * 1e-3) / 1e9, 1),
           "refine_steps_mean": round(refine_mean, 4), "fallbacks": st["fallbacks"],
           "factor_bytes": st["factor_bytes"], "pass_bytes": st["pass_bytes"],
           "factor_gflop": round(st["factor_flops"] / 1e9, 3),
           "cholesky_tflops": round(st["factor_flops"] / (st["t_chol_ms"] * 1e-3) / 1e12, 4),
           "cholesky_split_blocks": st["chol_split_blocks"],
           "kernel_launches": st["kernel_launches"],
           "proj_config": {"ring_slots": st["proj_slots"], "ctas_per_sm": st["proj_ctas_per_sm"],
                           "tuned": st["proj_tuned"]},
           "x_err_vs_true": rel_err(x, r.w.x_true[0])}
    if kt is not None:
        out.update({"proj_ms": round(kt["proj_ms"], 5),
                    "proj_ms_isolated": round(kt["proj_ms_isolated"], 5),
                    "proj_launches_timed": kt["proj_launches_timed"],
                    "proj_bytes": round(b["proj"]),
                    "proj_gbps": round(b["proj"] / (kt["proj_ms"] * 1e-3) / 1e9, 1)})
    return out


def leg_config2(dev, stream, flush, layout, local):
    """The 64^3 convection-diffusion system, contiguous blocks: one warm-up and two timed
    solves per precision; x against the stored oracle solution (tests/golden, written from
    the oracle only) at its sample rows.  Then the graph partition of its row inner-product
    graph (K = 128, 5% imbalance, computed before the timed region): one warm-up and one
    timed solve per precision."""
    import inputs
    w = inputs.workload(2)
    gold = json.load(open(os.path.join(GOLDEN, "config2_oracle.json")))
    r = Runner(w, w.perm, w.block_ptr, layout, dev, stream, flush)
    out = {"workload": w.name, "partition": "contiguous", "oracle_iters": gold["iters"]}
    with Clocks(local) as ck:
        for precision in ("fp64", "fp32_refine"):
            times, (s, st, code) = r.timed(precision, 2, 1)
            x = r.x_host()
            s.close()
            idx = np.asarray(gold["x_sample_idx"])
            d = leg_summary(r, st, times, None, x, w.A.n, w.A.nnz, len(w.block_ptr) - 1)
            d["status"] = code
            d["x_err_vs_oracle_max"] = float(np.abs(x[idx] - np.asarray(gold["x_sample"])).max()
                                             / gold["x_max_abs"])
            out[precision] = d
        perm, bp, part = partition_of(w, "graph", 2)
        rg = Runner(w, perm, bp, layout, dev, stream, flush)
        gp = {"partition_info": part}
        for precision in ("fp64", "fp32_refine"):
            times, (s, st, code) = rg.timed(precision, 1, 1)
            x = rg.x_host()
            s.close()
            d = leg_summary(rg, st, times, None, x, w.A.n, w.A.nnz, len(bp) - 1)
            d["status"] = code
            gp[precision] = d
        out["graph_partition"] = gp
    out["clocks"] = ck.summary()
    return out


def leg_config4(dev, stream, flush, layout, local):
    """64 independent 3D convection-diffusion systems (64x64xnz grids, about 5.7 M rows, blocks
    of 256 to 2048 rows) in one context: one launch per stage over every system's blocks.
    Time to 1e-10 for all 64 systems, setup included (inputs resident on the device, right-hand
    sides and solutions through host memory), one run per precision."""
    import torch

    import inputs
    import paper_1710_07769_gb300 as g
    systems = inputs.batch_workload(nsys=64, seed=4)
    dAs = [to_device(w.A, dev) for w in systems]
    bps = [w.block_ptr for w in systems]
    Fs = [w.F[0] for w in systems]
    torch.cuda.synchronize()
    out = {"workload": "batch64_convdiff3d_64x64xnz", "nsys": len(systems),
           "n_total": int(sum(w.A.n for w in systems)),
           "blocks": int(sum(len(b) - 1 for b in bps))}
    with Clocks(local) as ck:
        for precision in ("fp32_refine", "fp64"):
            with torch.cuda.stream(stream):
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                bs = g.BatchSolver(dAs, bps, precision=precision, layout=layout)
                X, st, code = bs.solve(Fs, tol=TOL)
                torch.cuda.synchronize()
                t = (time.perf_counter() - t0) * 1e3
            bs.close()
            its = [q["iters"] for q in st]
            out[precision] = {
                "time_to_solution_ms": round(t, 1), "status": code,
                "iters_min": min(its), "iters_max": max(its),
                "rel_res_max": max(q["rel_res"] for q in st),
                "setup_ms": round(st[0]["t_setup_ms"], 3),
                "factor_ms": round(st[0]["t_factor_ms"], 3),
                "solve_ms": round(st[0]["t_solve_ms"], 3),
                "x_err_vs_true_max": max(rel_err(X[q], systems[q].x_true[0])
                                         for q in range(len(systems)))}
    out["clocks"] = ck.summary()
    del dAs
    return out


def leg_config5(dev, stream, flush, layout, local, window=64):
    """The 128^3 system with 16 right-hand sides sharing the factors (contiguous blocks of
    2048 rows): one full FP32+refine solve of all 16 lanes, and FP64 per CG iteration over a
    fixed window of `window` iterations (its full solve would take minutes)."""
    import torch

    import inputs
    import paper_1710_07769_gb300 as g
    w = inputs.workload(5)
    dA = to_device(w.A, dev)
    dF = torch.from_numpy(np.ascontiguousarray(w.F)).to(dev)
    dX = torch.empty_like(dF)
    torch.cuda.synchronize()
    out = {"workload": w.name, "partition": "contiguous", "nrhs": int(w.F.shape[0])}
    with Clocks(local) as ck:
        with torch.cuda.stream(stream):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s = g.Solver(dA, w.block_ptr, perm=w.perm, precision="fp32_refine", layout=layout)
            X, st, code = s.solve(dF, tol=TOL, X=dX)
            e1.record(stream)
        e1.synchronize()
        t32 = e0.elapsed_time(e1)
        s.close()
        Xh = dX.cpu().numpy()
        its = [q["iters"] for q in st]
        out["fp32_refine"] = {
            "time_to_solution_ms": round(t32, 3), "status": code,
            "iters_min": min(its), "iters_max": max(its),
            "rel_res_max": max(q["rel_res"] for q in st),
            "setup_ms": round(st[0]["t_setup_ms"], 3), "factor_ms": round(st[0]["t_factor_ms"], 3),
            "solve_ms": round(st[0]["t_solve_ms"], 3),
            "per_iter_ms": round(st[0]["t_solve_ms"] / (max(its) + 1), 4),
            "x_err_vs_true_max": max(rel_err(Xh[k], w.x_true[k]) for k in range(len(its)))}
        with torch.cuda.stream(stream):
            s = g.Solver(dA, w.block_ptr, perm=w.perm, precision="fp64", layout=layout,
                         max_iter=window)
            X, st, code = s.solve(dF, tol=TOL, X=dX)
        s.close()
        out["fp64_window"] = {"iters": window, "status": code,
                              "setup_ms": round(st[0]["t_setup_ms"], 3),
                              "factor_ms": round(st[0]["t_factor_ms"], 3),
                              "per_iter_ms": round(st[0]["t_solve_ms"] / (window + 1), 4)}
        # the same FP32+refine iterations with the 16 lanes' triangular solves on the tensor
        # cores (opts.multi_rhs = 2), over the FP64 leg's window
        with torch.cuda.stream(stream):
            s = g.Solver(dA, w.block_ptr, perm=w.perm, precision="fp32_refine", layout=layout,
                         max_iter=window, multi_rhs=2)
            X, st, code = s.solve(dF, tol=TOL, X=dX)
        s.close()
        nproj = (window + 1) * (len(w.block_ptr) - 1) * int(w.F.shape[0])
        out["fp32_refine_tensor_cores_window"] = {
            "iters": window, "mr_tc_blocks": st[0]["mr_tc_blocks"],
            "per_iter_ms": round(st[0]["t_solve_ms"] / (window + 1), 4),
            "refine_steps_per_inner_solve": round(st[0]["refine_steps_total"] / nproj, 3)}
    out["clocks"] = ck.summary()
    del dA, dF, dX
    return out


def run_ours(args, rank, local):
    import torch

    import inputs
    import paper_1710_07769_gb300 as g

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    w = inputs.workload(args.config)
    partition = args.partition or DEFAULT_PARTITION.get(args.config, "contiguous")
    perm, bp, part = partition_of(w, partition, args.config)
    nblk = len(bp) - 1
    r = Runner(w, perm, bp, args.layout, dev, stream, flush)

    if args.gpus > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    t_wall0 = time.time()
    with clocks:
        t64, (s64, st64, code64) = r.timed("fp64", args.steps, args.warmup)
    torch.cuda.synchronize()
    wall = time.time() - t_wall0
    x64 = r.x_host()
    ms_step = sum(t64) / len(t64)
    if args.gpus > 1:
        ms_step = max_over_ranks(ms_step, dev)
        torch.distributed.barrier()
    s64.close()
    kt64 = r.proj_live("fp64")
    # FP32 + refinement on the same blocks (at least 3 timed steps, same rules)
    clocks32 = Clocks(local)
    with clocks32:
        t32, (s32, st32, code32) = r.timed("fp32_refine", max(3, min(args.steps, 5)), 1)
    x32 = r.x_host()
    s32.close()
    kt32 = r.proj_live("fp32_refine")
    # FP32 with the relaxed inner tolerance refine_tol / relres_t (an inexact-Krylov variant:
    # same stopping test, a few more iterations, fewer second factor passes)
    tr, (sr, str_, coder) = r.timed("fp32_refine", 2, 1, refine_relax=True)
    xr = r.x_host()
    sr.close()
    if rank != 0:
        return None, (None, None, None)

    r64 = leg_summary(r, st64, t64, kt64, x64, w.A.n, w.A.nnz, nblk)
    r32 = leg_summary(r, st32, t32, kt32, x32, w.A.n, w.A.nnz, nblk)
    r32["x_err_vs_fp64"] = rel_err(x32, x64)
    r32["clocks"] = clocks32.summary()
    rrx = {"time_to_solution_ms": round(sum(tr) / len(tr), 3), "iters": str_["iters"],
           "rel_res": str_["rel_res"], "status": coder, "solve_ms": round(str_["t_solve_ms"], 3),
           "refine_steps_total": str_["refine_steps_total"],
           "inner_solves": nblk * (str_["iters"] + 1), "x_err_vs_true": rel_err(xr, w.x_true[0]),
           "x_err_vs_fp64": rel_err(xr, x64)}

    # e2e: host CSR and host f / x through the C ABI, copies inside the timed region
    e2e_t = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        se = g.Solver(w.A, bp, perm=perm, precision="fp64", layout=args.layout, tune=True,
                      tune_cache=TUNE_CACHE)
        xe, ste, ce = se.solve(w.F[0], tol=TOL)
        e2e_t.append((time.perf_counter() - t0) * 1e3)
        se.close()
    h2d = w.A.row_ptr.nbytes + w.A.col_idx.nbytes + w.A.val.nbytes + w.F[0].nbytes
    d2h = xe.nbytes

    # the other partition of the same workload (one warm-up and one timed solve each)
    other = None
    if not args.no_other:
        op = "contiguous" if part["partition"] == "graph" else "graph"
        if op == "contiguous" or args.config in (2, 3):
            operm, obp, opart = partition_of(w, op, args.config)
            ro = Runner(w, operm, obp, args.layout, dev, stream, flush)
            other = dict(opart)
            for precision in ("fp64", "fp32_refine"):
                tt, (so, sto, codeo) = ro.timed(precision, 1, 1)
                so.close()
                other[precision] = {"time_to_solution_ms": round(tt[0], 3), "iters": sto["iters"],
                                    "status": codeo, "factor_ms": round(sto["t_factor_ms"], 3),
                                    "cholesky_ms": round(sto["t_chol_ms"], 3),
                                    "solve_ms": round(sto["t_solve_ms"], 3),
                                    "factor_bytes": sto["factor_bytes"]}
            del ro
    cfg2 = None if args.no_cfg2 or args.config == 2 else leg_config2(dev, stream, flush,
                                                                      args.layout, local)
    cfg5 = None if args.no_cfg5 or args.config == 5 else leg_config5(dev, stream, flush,
                                                                      args.layout, local)
    cfg4 = None if args.no_cfg4 else leg_config4(dev, stream, flush, args.layout, local)

    pk = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "fallback" not in pk else "fallback"
    # the FP64 ALU roofline: this GPU's FMA rate measured by the library's probe kernel
    try:
        fp64_peak, fp64_src = g.fp64_peak(), "measured (FP64 FMA probe on every SM)"
    except Exception:
        fp64_peak, fp64_src = FP64_PEAK_TFLOPS, "nominal FP64 rate (152 SMs at 2070 MHz)"
    # the kernel that dominates the FP64 step: the batched Cholesky or the projections
    chol64 = {"bound": "alu",
              "kernel": "k_cholesky (FP64 tile Cholesky, one CTA per SM on a packed block list)",
              "achieved": r64["cholesky_tflops"], "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
              "frac": round(r64["cholesky_tflops"] / fp64_peak, 4),
              "traffic": TRAFFIC.get("k_cholesky_fp64_" + w.name),
              "flops_per_launch": st64["factor_flops"], "ms_per_launch": r64["cholesky_ms"],
              "peak_source": fp64_src, "nominal_peak": FP64_PEAK_TFLOPS}
    flops64 = st64["pass_bytes"] / 4.0  # 2 flops per streamed 8-byte factor element, one pass
    tf64 = flops64 / (kt64["proj_ms"] * 1e-3) / 1e12
    proj64 = {"bound": "alu", "kernel": "k_proj (FP64 tile solves)", "achieved": round(tf64, 4),
              "peak": round(fp64_peak, 4), "unit": "TFLOP/s", "frac": round(tf64 / fp64_peak, 4),
              "traffic": TRAFFIC.get("k_proj_fp64_" + w.name),
              "ms_per_launch": r64["proj_ms"], "peak_source": fp64_src,
              "hbm_view": {"achieved_gbs": r64["proj_gbps"], "frac": round(r64["proj_gbps"] / hbm, 4)}}
    proj32 = {"bound": "hbm", "kernel": "k_proj (FP32 tile solves + FP64 refinement)",
              "achieved": r32["proj_gbps"], "peak": hbm, "unit": "GB/s",
              "frac": round(r32["proj_gbps"] / hbm, 4),
              "traffic": TRAFFIC.get("k_proj_fp32_" + w.name), "ms_per_launch": r32["proj_ms"],
              "peak_source": peak_src}
    chol_share = r64["cholesky_ms"] / r64["time_to_solution_ms"]
    proj_share = r64["proj_ms"] * (r64["iters"] + 1) / r64["time_to_solution_ms"]
    roof = dict(chol64 if chol_share >= proj_share else proj64)
    roof["share_of_step"] = round(max(chol_share, proj_share), 4)
    cfg = config_dict(w, part, args.layout, args)
    out = {
        "metric": METRIC, "value": round(ms_step, 3), "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg, "partition_info": part,
        "fp64": r64, "fp32_refine": r32, "fp32_refine_relaxed": rrx,
        "fp32_vs_fp64_time_ratio": round(r32["time_to_solution_ms"] / r64["time_to_solution_ms"], 4),
        "other_partition": other, "convdiff3d_64": cfg2, "convdiff3d_128_16rhs": cfg5,
        "batch64": cfg4,
        "roofline": roof,
        "roofline_kernels": {"cholesky_fp64": chol64, "proj_fp64": proj64, "proj_fp32": proj32,
                             "cholesky_tc_fp32": {
                                 "bound": "tensor", "kernel": "k_cholesky_tc (3xTF32 tcgen05)",
                                 "useful_tflops": r32["cholesky_tflops"],
                                 "ms_per_launch": r32["cholesky_ms"],
                                 "note": "useful FP32 flops; the tensor pipe issues 3x as "
                                         "TF32 (3xTF32 split)"}},
        "e2e": {"value": round(min(e2e_t), 3), "unit": "ms", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(st64["kernel_launches"]) * args.steps,
        "clocks": clocks.summary(),
        "wall_s": round(wall, 3),
    }
    return out, (w, perm, bp)


# ------------------------------------------------------------------ the oracle on the host cores

def oracle_sample(w, perm, bp, cores, steps, warmup, iters):
    """The FP64 oracle as it stands, on the host cores, in bounded samples of the workload.

    Once (not part of a step): the oracle's setup without factors (scaling, permutation,
    C = A A^T; OpenMP over rows / columns where the oracle has it).  Each step: the
    oracle's Cholesky of `cores` consecutive Gram blocks (one block per thread, OpenMP over
    blocks, i.e. one wave of the full factorisation) and one inner solve of each of those
    blocks (one wave of a projection's solves), blocks rotating from step to step.  The
    full oracle time to solution is estimated from these as
      setup + ceil(K / cores) * factor wave + iters * ceil(K / cores) * solve wave,
    the sparse products of an iteration being small beside the dense block solves."""
    import oracle
    K = len(bp) - 1
    S = max(1, min(cores, K))
    t0 = time.perf_counter()
    o = oracle.Oracle(w.A, bp, perm=perm, factor=False, nthreads=cores)
    t_setup = time.perf_counter() - t0
    u = np.random.default_rng(0).standard_normal(w.A.n)
    step_ms, fac_s, sol_s = [], [], []
    for i in range(warmup + steps):
        b0 = (i * S) % K
        b1 = min(K, b0 + S)
        t0 = time.perf_counter()
        st = o.factor_range(b0, b1)
        t1 = time.perf_counter()
        o.solve_range(u)
        t2 = time.perf_counter()
        if st != 0:
            raise RuntimeError(f"oracle factorisation failed (status {st})")
        if i >= warmup:
            step_ms.append((t2 - t0) * 1e3)
            fac_s.append((t1 - t0) * (S / (b1 - b0)))
            sol_s.append((t2 - t1) * (S / (b1 - b0)))
    o.close()
    waves = math.ceil(K / S)
    f_wave, s_wave = statistics.median(fac_s), statistics.median(sol_s)
    est_setup = t_setup + waves * f_wave
    est_iter = waves * s_wave
    est = (est_setup + iters * est_iter) * 1e3
    return {"step_ms": step_ms, "cores": cores, "kind": "oracle",
            "setup_without_factors_s": round(t_setup, 2), "factor_wave_s": round(f_wave, 3),
            "solve_wave_s": round(s_wave, 4), "waves": waves,
            "est_setup_ms": round(est_setup * 1e3, 1), "est_iteration_ms": round(est_iter * 1e3, 2),
            "iters": iters, "est_time_to_solution_ms": round(est, 1),
            "sample": f"{w.name}: oracle setup without factors once ({t_setup:.1f} s), then per "
                      f"step the Cholesky of {S} of the {K} Gram blocks ({S} threads) and their "
                      f"inner solves; full time to solution estimated for {iters} iterations"}


def reference_iters(config, w, perm, bp):
    """Iteration count the reference estimate uses: the oracle's own run where it is cheap
    (config 1) or stored (the 64^3 system, written from the oracle only); elsewhere the
    FP64 count of the GPU solve on these blocks, which the parity tests hold to the
    oracle's +-1 (30 for the graph-partitioned random system)."""
    if config == 1:
        import oracle
        return oracle.Oracle(w.A, bp, perm=perm).solve(w.F[0])[1]
    if config == 2:
        return int(json.load(open(os.path.join(GOLDEN, "config2_oracle.json")))["iters"])
    return {3: 30, 5: 3900}.get(config, 100)


def run_reference(args):
    """The reference arm: the FP64 oracle timed on the host cores, each step a bounded sample
    of the same workload and blocks as our arm (the partition is input preparation, not
    timed)."""
    import inputs
    w = inputs.workload(args.config)
    partition = args.partition or DEFAULT_PARTITION.get(args.config, "contiguous")
    perm, bp, part = partition_of(w, partition, args.config, use_gpu=False)
    cores = os.cpu_count() or 1
    iters = reference_iters(args.config, w, perm, bp)
    t_run = time.perf_counter()
    smp = oracle_sample(w, perm, bp, cores, args.steps, args.warmup, iters)
    steps_ms = smp.pop("step_ms")
    v = sum(steps_ms) / len(steps_ms)
    cb = dict(smp)
    cb["value"] = round(v, 1)
    cb["unit"] = "ms"
    cfg = config_dict(w, part, args.layout, args)
    return {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "ms",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(v, 1), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "partition_info": part,
            "value_is": "per-step time of the bounded oracle sample (see cpu_baseline.sample)",
            "extrapolated_time_to_solution_ms": smp["est_time_to_solution_ms"],
            "cpu_baseline": cb, "run_s": round(time.perf_counter() - t_run, 1),
            "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------ profiling targets

def run_profile(args):
    import inputs
    import paper_1710_07769_gb300 as g
    if args.profile == "spgemm":
        w = inputs.workload(args.config)
        rp, ci, v = g.aat(w.A)
        print(json.dumps({"profile": "spgemm", "workload": w.name, "nnz_aat": int(len(v))}))
        return 0
    if args.profile in ("cholesky_tc", "cholesky_fp64"):
        # random n = 2^18 with 8 off-diagonals per row: 128 Gram blocks of 2048 rows from the
        # graph partition (banded envelopes, as in the n = 2^20 workload) or contiguous
        # (nearly dense envelopes)
        n = 1 << 18
        A = inputs.random_dd(n, 8, 3)
        if (args.partition or "graph") == "graph":
            perm, bp, _ = g.partition_rip(n, g.aat(A), n // 2048, cap=2048, seed=0)
        else:
            perm, bp = None, inputs.contiguous_blocks(n, 2048)
        prec = "fp32_refine" if args.profile == "cholesky_tc" else "fp64"
        s = g.Solver(A, bp, perm=perm, precision=prec, max_iter=1)
        x, st, code = s.solve(inputs.matvec(A, np.ones(n)), tol=TOL)
        print(json.dumps({"profile": args.profile, "n": n, "cholesky_ms": st[0]["t_chol_ms"],
                          "factor_gflop": st[0]["factor_flops"] / 1e9}))
        s.close()
        return 0
    if args.profile == "mr_passes":
        # live projection time (CUDA events around every projection of a 16-iteration window)
        # of the 16-RHS workload: one pass, two passes and one residual, and to refine_tol,
        # with the triangular solves on the tensor cores (multi_rhs 2) and on CUDA cores (1)
        w = inputs.workload(args.config, nrhs=16)
        res = {"profile": "mr_passes", "workload": w.name}
        for mode in (2, 1):
            for rm in (0, 1, None):
                s = g.Solver(w.A, w.block_ptr, perm=w.perm, precision="fp32_refine",
                             multi_rhs=mode, max_iter=16, time_proj=True, refine_max=rm)
                x, st, code = s.solve(w.F, tol=TOL)
                ms, n = s.proj_timing()
                res[f"multi_rhs{mode}_refine_max{'default' if rm is None else rm}"] = {
                    "proj_ms": round(ms / max(n, 1), 3),
                    "refine_steps_per_inner_solve": round(
                        st[0]["refine_steps_total"] / (max(n, 1) * 16 * (len(w.block_ptr) - 1)), 3)}
                s.close()
        print(json.dumps(res))
        return 0
    multi = args.profile in ("fp32_refine_16rhs", "fp32_refine_16rhs_tc")
    w = inputs.workload(args.config, nrhs=16 if multi else None)
    partition = args.partition or DEFAULT_PARTITION.get(args.config, "contiguous")
    perm, bp, _ = partition_of(w, partition, args.config)
    # the benchmark's launch configuration: the projection autotuned (candidate launches
    # first, then the right-hand side's projection and the CG iterations)
    s = g.Solver(w.A, bp, perm=perm, precision="fp32_refine" if multi else args.profile,
                 layout=args.layout, max_iter=4, check_every=1, tune=True,
                 multi_rhs=2 if args.profile == "fp32_refine_16rhs_tc" else None)
    x, st, code = s.solve(w.F if multi else w.F[0], tol=TOL)
    print(json.dumps({"profile": args.profile, "workload": w.name, "iters": st[0]["iters"],
                      "status": st[0]["status_name"], "factor_bytes": st[0]["factor_bytes"]}))
    s.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=3, choices=[1, 2, 3, 5])
    ap.add_argument("--partition", default=None, choices=["graph", "contiguous"],
                    help="blocks of the workload (default: graph for the n = 2^20 random "
                         "system, contiguous otherwise)")
    ap.add_argument("--layout", default="skyline", choices=["skyline", "dense"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline sample")
    ap.add_argument("--no-other", action="store_true", help="skip the other-partition leg")
    ap.add_argument("--no-cfg2", action="store_true", help="skip the 64^3 leg")
    ap.add_argument("--no-cfg5", action="store_true", help="skip the 128^3 16-RHS leg")
    ap.add_argument("--no-cfg4", action="store_true", help="skip the 64-system batch leg")
    ap.add_argument("--profile", default=None,
                    choices=["fp64", "fp32_refine", "fp32_refine_16rhs", "fp32_refine_16rhs_tc",
                             "mr_passes", "cholesky_tc", "cholesky_fp64", "spgemm"],
                    help="profiling target, nothing timed: fp64 / fp32_refine / "
                         "fp32_refine_16rhs = one autotuned setup + 4 CG iterations of --config "
                         "and its default blocks (16 right-hand sides for the last two, _tc: "
                         "FP32 triangular solves on the tensor cores); mr_passes = live "
                         "projection times of the 16-RHS --config on both multi-RHS kernels; "
                         "cholesky_tc / cholesky_fp64 = setup "
                         "of 128 Gram blocks of 2048 rows of a random n = 2^18 system "
                         "(graph-partitioned unless --partition contiguous); spgemm = "
                         "standalone C = A A^T of --config")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.profile:
        return run_profile(args)
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args)))
        return 0
    if args.gpus > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out, (w, perm, bp) = run_ours(args, rank, local)
    if rank == 0:
        if not args.no_cpu:
            smp = oracle_sample(w, perm, bp, os.cpu_count() or 1, 2, 0, out["fp64"]["iters"])
            smp.pop("step_ms")
            smp["value"] = smp["est_time_to_solution_ms"]
            smp["unit"] = "ms"
            out["cpu_baseline"] = smp
        print(json.dumps(out))
    if args.gpus > 1:
        import torch
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
