"""Writes the stored expected values of the full-size parity tests by running ONLY the
FP64 oracle (oracle/) on the seeded synthetic inputs (inputs/).

  python tests/golden/make_golden.py [nthreads]

config2_oracle.json: Algorithm 2 on the 3D convection-diffusion 64^3 system
(b = (30, 20, 10), K = 128 contiguous blocks of 2048 rows, f = A x_true, seed 2)
from x = 0 to ||f - A x||_2 <= 1e-10 ||f||_2: iteration count, final relative
residual, a checksum of x and x itself at 512 seeded sample rows (the first and the
last row included), for an element-wise comparison.  About 4 minutes on 8 cores.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import inputs  # noqa: E402
import oracle  # noqa: E402


def main():
    nthreads = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    w = inputs.workload(2)
    t0 = time.time()
    o = oracle.Oracle(w.A, w.block_ptr, perm=w.perm, nthreads=nthreads)
    x, it, rr, gm, st = o.solve(w.F[0], tol=1e-10)
    n = w.A.n
    idx = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(2).choice(n, 510, replace=False)]))
    out = {"workload": w.name, "tol": 1e-10, "status": st, "iters": it, "rel_res": rr,
           "backward_err": gm, "x_sum": float(np.sum(x)), "x_norm2": float(np.linalg.norm(x)),
           "x_err_vs_true_max": float(np.abs(x - w.x_true[0]).max()),
           "x_max_abs": float(np.abs(x).max()),
           "x_sample_idx": idx.tolist(), "x_sample": [float(v) for v in x[idx]],
           "oracle_seconds": round(time.time() - t0, 1), "nthreads": nthreads,
           "source": "written by tests/golden/make_golden.py from oracle/ only"}
    with open(os.path.join(HERE, "config2_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
