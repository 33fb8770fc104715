"""Benchmark: time to a 1e-10 relative residual of the CG-accelerated block Cimmino
solve (setup + solve) and HBM GB/s per CG iteration, FP64 vs FP32+refinement, on
one GB300.

Workload (default): 3D convection-diffusion 64^3 (n = 262,144), 7-point upwind
stencil, b = (30, 20, 10), K = 128 contiguous blocks of 2048 rows, f = A x_true,
x_true ~ U[-1, 1] (seed 2).  A step = one full pass of the hot path: row scaling +
permutation, A^T, C = A A^T, Gram blocks, batched Cholesky, then Algorithm 2 to
||f - A x|| <= 1e-10 ||f||, with A and f already resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own copy of the workload (replicas
only: the solve does not shard); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-10 rel. residual & HBM GB/s per CG iter; FP32+refine vs FP64 on GB300"
TOL = 1e-10
FP64_PEAK_TFLOPS = 1.25  # GB300 FP64 (recipe table); the FMA probe measured 1.196
# DRAM bytes per k_proj launch from one ncu capture of the current kernel (ncu
# --set full, 64^3 workload, CG iteration 1)
PROJ_TRAFFIC = {"fp64": 659753728, "fp32": 726496512}


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
    """nvidia-smi sampling (SM clock, throttle reasons) during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None
        self.path = os.path.join(tempfile.gettempdir(), f"cimmino_clocks_{os.getpid()}_{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
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
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


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


def algorithmic_bytes(n, nnz, factor_bytes, w_factor, refine_mean, nnz_bd):
    """Minimum bytes one CG iteration must move (1 right-hand side).

    projection: one solve pass streams pass_bytes = 2 x factor_bytes (N tiles and
      inv(L_II) for the forward solve, their transposed copies for the backward
      solve), times (1 + refinement steps); each refinement step also reads the
      exact Gram block (12 B per entry); u read, y written.
    u = A p with the residual of x: CSR (12 B/entry + 8 B/row), p and x gathered,
      f_s and d read, u written.
    psi = A^T y with p^T psi: transpose (12 B/entry + 8 B/column), y gathered,
      p read, psi written.
    x, r update (4 read, 2 written) and p update (2 read, 1 written).
    """
    proj = (1 + refine_mean) * 2 * factor_bytes + refine_mean * 12 * nnz_bd + 16 * n
    spmv = 12 * nnz + 8 * n + 16 * n + 16 * n + 8 * n
    spmv_t = 12 * nnz + 8 * n + 8 * n + 8 * n + 8 * n
    upd = 6 * 8 * n + 3 * 8 * n
    return {"proj": proj, "iteration": proj + spmv + spmv_t + upd}


def run_ours(args, rank, local):
    import torch

    import inputs
    import paper_1710_07769_gb300 as g

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = inputs.workload(args.config)
    A = w.A
    n = A.n
    stream = torch.cuda.Stream(device=dev)

    class DevCSR:
        pass

    dA = DevCSR()
    dA.n = n
    dA.row_ptr = torch.from_numpy(A.row_ptr).to(dev)
    dA.col_idx = torch.from_numpy(A.col_idx).to(dev)
    dA.val = torch.from_numpy(A.val).to(dev)
    dF = torch.from_numpy(w.F[0]).to(dev)
    dX = torch.empty_like(dF)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    torch.cuda.synchronize()

    def step(precision, relax=False, time_proj=False):
        with torch.cuda.stream(stream):
            s = g.Solver(dA, w.block_ptr, perm=w.perm, precision=precision, layout=args.layout,
                         refine_relax=relax, time_proj=time_proj)
            x, st, code = s.solve(dF, tol=TOL, X=dX)
        return s, st[0], code

    def timed(precision, k, w_, relax=False):
        for _ in range(w_):
            s, st, code = step(precision, relax)
            s.close()
        times, last = [], None
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            s, st, code = step(precision, relax)
            with torch.cuda.stream(stream):
                e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            if last is not None:
                last[0].close()
            last = (s, st, code)
        return times, last

    if args.gpus > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    t_wall0 = time.time()
    with clocks:
        t64, (s64, st64, code64) = timed("fp64", args.steps, args.warmup)
    torch.cuda.synchronize()
    wall = time.time() - t_wall0
    ms_step = sum(t64) / len(t64)
    if args.gpus > 1:
        ms_step = max_over_ranks(ms_step, dev)
        torch.distributed.barrier()
    def proj_live(precision):
        """Average device time of the projection launches inside the CG loop of one more
        solve of the same workload (CUDA events on the library's stream around every
        projection launch, iterations launched eagerly), and the isolated back-to-back
        figure beside it."""
        s, st, code = step(precision, time_proj=True)
        ms, nl = s.proj_timing()
        kt = s.time_kernels(reps=10)
        s.close()
        kt["proj_ms_isolated"] = kt["proj_ms"]
        kt["proj_ms"] = ms / max(1, nl)
        kt["proj_launches_timed"] = nl
        return kt

    kt64 = proj_live("fp64")
    # FP32 + refinement on the same workload (fewer steps, same rules)
    t32, (s32, st32, code32) = timed("fp32_refine", max(1, min(args.steps, 2)), 1)
    kt32 = proj_live("fp32_refine")
    # FP32 with the relaxed inner tolerance refine_tol / relres_t (an inexact-Krylov variant:
    # same stopping test, a few more iterations, fewer second factor passes)
    tr, (sr, str_, coder) = timed("fp32_refine", max(1, min(args.steps, 2)), 1, relax=True)

    if rank != 0:
        s64.close()
        s32.close()
        sr.close()
        return None

    # e2e: host CSR and host f / x through the C ABI, copies inside the timed region
    e2e_t = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        se = g.Solver(A, w.block_ptr, perm=w.perm, precision="fp64", layout=args.layout)
        xe, ste, ce = se.solve(w.F[0], tol=TOL)
        e2e_t.append((time.perf_counter() - t0) * 1e3)
        se.close()
    h2d = A.row_ptr.nbytes + A.col_idx.nbytes + A.val.nbytes + w.F[0].nbytes
    d2h = xe.nbytes

    pk = peaks()
    nnz_bd_est = None
    def per_iter(st, kt, t_steps):
        nblk = len(w.block_ptr) - 1
        launches = st["iters"] + 1
        refine_mean = st["refine_steps_total"] / max(1, nblk * (launches + 1))
        wf = 8 if st is st64 else 4
        # the exact Gram blocks have ~25 entries per row for the 7-point stencil
        b = algorithmic_bytes(n, A.nnz, st["pass_bytes"] / 2, wf, refine_mean, 25 * n)
        it_ms = st["t_solve_ms"] / max(1, st["iters"] + 1)
        return {"time_to_solution_ms": sum(t_steps) / len(t_steps), "iters": st["iters"],
                "rel_res": st["rel_res"], "backward_err": st["backward_err"],
                "setup_ms": st["t_setup_ms"], "factor_ms": st["t_factor_ms"],
                "solve_ms": st["t_solve_ms"], "per_iter_ms": it_ms,
                "hbm_gbps_per_iter": b["iteration"] / (it_ms * 1e-3) / 1e9,
                "proj_ms": kt["proj_ms"], "proj_ms_isolated": kt["proj_ms_isolated"],
                "proj_launches_timed": kt["proj_launches_timed"], "proj_bytes": b["proj"],
                "proj_gbps": b["proj"] / (kt["proj_ms"] * 1e-3) / 1e9,
                "refine_steps_mean": refine_mean, "fallbacks": st["fallbacks"],
                "factor_bytes": st["factor_bytes"], "pass_bytes": st["pass_bytes"],
                "kernel_launches": st["kernel_launches"]}

    r64 = per_iter(st64, kt64, t64)
    r32 = per_iter(st32, kt32, t32)
    rrx = {"time_to_solution_ms": round(sum(tr) / len(tr), 3), "iters": str_["iters"],
           "rel_res": str_["rel_res"], "status": coder, "solve_ms": round(str_["t_solve_ms"], 3),
           "refine_steps_total": str_["refine_steps_total"],
           "inner_solves": (len(w.block_ptr) - 1) * (str_["iters"] + 1)}
    s64.close()
    s32.close()
    sr.close()
    gp = None if args.no_gp else gp_leg(w, dA, dF, dX, stream, args.layout)
    hbm = float(pk.get("hbm_gbs", 6800.0))
    # FP64 projection: every streamed FP64 factor element feeds one FMA, so it is bound by
    # GB300's FP64 pipe (ncu: FP64 pipe 73% / DRAM 35% busy); FP32 projection: HBM-bound.
    flops64 = st64["pass_bytes"] / 4.0           # 2 flops per 8-byte element, one pass
    tf64 = flops64 / (kt64["proj_ms"] * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": round(tf64, 4), "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": round(tf64 / FP64_PEAK_TFLOPS, 4),
            "traffic": PROJ_TRAFFIC.get("fp64"), "kernel": "k_proj (FP64 tile solves)",
            "peak_source": "nominal FP64 1.25 TFLOP/s (probe measured 1.196)",
            "hbm_view": {"achieved_gbs": round(r64["proj_gbps"], 1), "frac": round(r64["proj_gbps"] / hbm, 4)}}
    roof32 = {"bound": "hbm", "achieved": round(r32["proj_gbps"], 1), "peak": hbm, "unit": "GB/s",
              "frac": round(r32["proj_gbps"] / hbm, 4), "traffic": PROJ_TRAFFIC.get("fp32"),
              "kernel": "k_proj (FP32 tile solves + FP64 refinement)",
              "peak_source": "measured" if "fallback" not in pk else "fallback"}
    out = {
        "metric": METRIC, "value": round(ms_step, 3), "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "n": n, "nnz": int(A.nnz), "K": len(w.block_ptr) - 1,
                   "partition": "contiguous", "layout": args.layout, "tol": TOL,
                   "precision": "fp64", "l2": "flushed (512 MB write) before every timed step",
                   "parallelism": "replicas" if args.gpus > 1 else "single"},
        "fp64": r64, "fp32_refine": r32, "fp32_refine_relaxed": rrx,
        "fp32_vs_fp64_time_ratio": round(r32["time_to_solution_ms"] / r64["time_to_solution_ms"], 4),
        "graph_partition": gp,
        "roofline": roof,
        "roofline_fp32": roof32,
        "e2e": {"value": round(min(e2e_t), 3), "unit": "ms", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(st64["kernel_launches"]) * args.steps,
        "clocks": clocks.summary(),
        "wall_s": round(wall, 3),
    }
    return out


def contiguous_cut(C, block_ptr):
    """Cutsize (Eq. 2.6, cosine weights of the row-scaled A) of the partition into
    consecutive row ranges, from C = A A^T of the unscaled A."""
    rp, ci, v = C
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    d = np.zeros(n)
    dg = rows == ci
    d[rows[dg]] = np.sqrt(v[dg])
    blk = np.searchsorted(block_ptr, np.arange(n), side="right") - 1
    m = (ci > rows) & (blk[rows] != blk[ci])
    return float(np.sum(np.abs(v[m]) / (d[rows[m]] * d[ci[m]])))


def gp_leg(w, dA, dF, dX, stream, layout, eps=0.05):
    """The graph-partitioned variant of the workload (Section 2): C = A A^T on the GPU, the
    host multilevel partitioner on G_RIP with blocks of at most (1 + eps) n / K rows, then
    both precisions solved with those blocks (one warm-up and one timed solve each)."""
    import torch

    import paper_1710_07769_gb300 as g
    n = w.A.n
    K = len(w.block_ptr) - 1
    t0 = time.perf_counter()
    C = g.aat(w.A)
    t_aat = time.perf_counter() - t0
    cap = int(np.floor((1.0 + eps) * n / K))
    t0 = time.perf_counter()
    perm, bp, cut = g.partition_rip(n, C, K, cap=cap, seed=0)
    t_part = time.perf_counter() - t0
    out = {"eps": eps, "cap": cap, "aat_s": round(t_aat, 3), "partition_s": round(t_part, 2),
           "cutsize": round(cut, 2), "cutsize_contiguous": round(contiguous_cut(C, w.block_ptr), 2),
           "block_rows_min": int(np.diff(bp).min()), "block_rows_max": int(np.diff(bp).max())}
    for precision in ("fp64", "fp32_refine"):
        times = []
        for _ in range(2):
            with torch.cuda.stream(stream):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s = g.Solver(dA, bp, perm=perm, precision=precision, layout=layout)
                x, st, code = s.solve(dF, tol=TOL, X=dX)
                e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            s.close()
        out[precision] = {"time_to_solution_ms": round(times[-1], 3), "iters": st[0]["iters"],
                          "rel_res": st[0]["rel_res"], "status": code,
                          "factor_ms": round(st[0]["t_factor_ms"], 3),
                          "solve_ms": round(st[0]["t_solve_ms"], 3),
                          "factor_bytes": st[0]["factor_bytes"]}
    return out


def cpu_sample(config, nthreads=None, iters_sample=10, full_iters=None):
    """Oracle on the host cores: full setup (scaling, A A^T, all Cholesky factors) plus a
    bounded number of CG iterations, extrapolated to the full iteration count."""
    import inputs
    import oracle
    nthreads = nthreads or os.cpu_count()
    w = inputs.workload(config)
    t0 = time.perf_counter()
    o = oracle.Oracle(w.A, w.block_ptr, perm=w.perm, nthreads=nthreads)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    x, it, rr, gm, st = o.solve(w.F[0], maxit=iters_sample)
    t_it = (time.perf_counter() - t0) / max(it, 1)
    full = full_iters if full_iters is not None else it
    est_ms = (t_setup + full * t_it) * 1e3
    return {"value": round(est_ms, 1), "unit": "ms", "cores": nthreads, "kind": "oracle",
            "workload": w.name,
            "sample": f"{w.name}: full oracle setup ({t_setup:.1f} s) + {it} CG iterations "
                      f"({t_it * 1e3:.1f} ms each) extrapolated to {full} iterations"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--layout", default="skyline", choices=["skyline", "dense"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline sample")
    ap.add_argument("--no-gp", action="store_true", help="skip the graph-partitioned leg")
    ap.add_argument("--profile", default=None,
                    choices=["fp64", "fp32_refine", "fp32_refine_16rhs", "cholesky_tc", "spgemm"],
                    help="profiling target, nothing timed: fp64 / fp32_refine / "
                         "fp32_refine_16rhs = one setup + 4 CG iterations of the workload "
                         "(16 right-hand sides sharing the factors for the last); cholesky_tc = "
                         "setup of 128 dense 2048-row Gram blocks (random n = 2^18, 8 entries "
                         "per row); spgemm = standalone C = A A^T of the workload")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.profile:
        import numpy as np

        import inputs
        import paper_1710_07769_gb300 as g
        if args.profile == "spgemm":
            w = inputs.workload(args.config)
            rp, ci, v = g.aat(w.A)
            print(json.dumps({"profile": "spgemm", "workload": w.name, "nnz_aat": int(len(v))}))
            return 0
        if args.profile == "cholesky_tc":
            n = 1 << 18
            A = inputs.random_dd(n, 8, 3)
            s = g.Solver(A, inputs.contiguous_blocks(n, 2048), precision="fp32_refine", max_iter=1)
            x, st, code = s.solve(inputs.matvec(A, np.ones(n)), tol=TOL)
            print(json.dumps({"profile": "cholesky_tc", "n": n, "factor_ms": st[0]["t_factor_ms"]}))
            s.close()
            return 0
        multi = args.profile == "fp32_refine_16rhs"
        w = inputs.workload(args.config, nrhs=16 if multi else None)
        s = g.Solver(w.A, w.block_ptr, perm=w.perm,
                     precision="fp32_refine" if multi else args.profile, layout=args.layout,
                     max_iter=4, check_every=1)
        x, st, code = s.solve(w.F if multi else w.F[0], tol=TOL)
        print(json.dumps({"profile": args.profile, "workload": w.name, "iters": st[0]["iters"],
                          "status": st[0]["status_name"], "factor_bytes": st[0]["factor_bytes"]}))
        s.close()
        return 0
    if args.impl == "reference":
        if rank != 0:
            return 0
        # the oracle as it stands, on the host cores; each step a bounded sample (full setup
        # plus 5 CG iterations), extrapolated to the oracle's own iteration count to 1e-10,
        # which tests/golden/config2_oracle.json records for the default workload (written
        # from oracle/ only); other workloads report the sample itself
        full = None
        gold = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                            "config2_oracle.json")
        if args.config == 2 and os.path.exists(gold):
            full = int(json.load(open(gold))["iters"])
        samples = []
        for i in range(args.warmup + args.steps):
            r = cpu_sample(args.config, iters_sample=5, full_iters=full)
            if i >= args.warmup:
                samples.append(r)
        v = sum(s["value"] for s in samples) / len(samples)
        cb = dict(samples[-1])
        cb["value"] = round(v, 1)
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "ms",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": round(v, 1), "higher_is_better": False, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": cb.pop("workload"), "partition": "contiguous",
                                     "tol": TOL, "precision": "fp64"},
                          "cpu_baseline": cb,
                          "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return 0
    if args.gpus > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, local)
    if rank == 0:
        if not args.no_cpu:
            cb = cpu_sample(args.config, full_iters=out["fp64"]["iters"])
            cb.pop("workload")
            out["cpu_baseline"] = cb
        print(json.dumps(out))
    if args.gpus > 1:
        import torch
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
