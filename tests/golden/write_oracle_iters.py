"""Writes tests/golden/oracle_fgmres_iters.json: for each named workload, the FP64 oracle's
FGMRES iteration count to rtol 1e-8 and a digest of its solution (the 2-norm and the
values at `SAMPLES` evenly spaced indices, see `sample_index`). Calls only oracle/ and
the seeded generators. The full-size GPU tests compare against these records.

    python tests/golden/write_oracle_iters.py aniso2d_1024_p64 [poisson2d_64_p4 ...]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2303_08881_gb300 import problems as P  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_fgmres_iters.json")
SAMPLES = 1024


def sample_index(n: int) -> np.ndarray:
    """The indices of the solution digest: SAMPLES points evenly spaced over 0..n-1."""
    return np.unique(np.linspace(0, n - 1, min(SAMPLES, n)).round().astype(np.int64))


def main(keys):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for k in keys:
        sol = dict(P.WORKLOAD_SOLVER[k])
        restart = sol.pop("restart")
        sol.pop("prec")
        pr = P.make_workload(k)
        t0 = time.perf_counter()
        o = O.Oracle.from_problem(pr, **sol)
        t1 = time.perf_counter()
        out = o.fgmres(pr.b, rtol=1e-8, restart=restart, maxit=20000)
        t2 = time.perf_counter()
        x = out["x"]
        data[k] = dict(workload=pr.name, n=int(pr.n), iters=out["iters"], relres=out["relres"], restart=restart,
                       setup_s=round(t1 - t0, 3), solve_s=round(t2 - t1, 3), status=out["status"],
                       x_norm2=float(np.linalg.norm(x)), x_absmax=float(np.abs(x).max()),
                       x_sample=[float(v) for v in x[sample_index(pr.n)]])
        print(k, {kk: vv for kk, vv in data[k].items() if kk != "x_sample"}, flush=True)
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["aniso2d_1024_p64"])
