"""Benchmark: FGMRES(50) time-to-rtol 1e-8 with the two-level ILU preconditioner on one
GB300 (or N replicas), plus the preconditioner-apply bandwidth, mixed vs FP64, the
roofline of the dominant kernel, an end-to-end number through the C ABI with host
buffers, and the FP64 CPU oracle as the baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload aniso2d_1024_p64] [--impl ilu2l|reference]

A step is one complete solve: FGMRES from x0 = 0 to ||b - Ax|| <= 1e-8 ||b|| on the
workload's synthetic right-hand side with the factors resident (the setup is timed
separately and inside the end-to-end number). value = solves per second over all
ranks (each rank solves its own replica; no data-path collective exists).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2303_08881_gb300 import problems as P  # noqa: E402

METRIC = "GMRES time-to-rtol 1e-8, PC-apply HBM GB/s, mixed vs FP64, p50/p99 latency"
UNIT = "solves/s"
# the workload a default run times: the 2D rotated anisotropic 9-point problem on a 1024^2
# grid in 8 x 8 subdomains, two-level ILU(0)/MILU(0), FP32 preconditioner, FGMRES(50)
DEFAULT_WORKLOAD = "aniso2d_1024_p64"
RTOL = 1e-8


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------------------
# algorithmic bytes (each array read or written once per pass; gathers counted once)


def prog_bytes(prog, sv, svv=None):
    """sv: bytes of a vector element and pivot inverse; svv: of a stored value (default sv)"""
    svv = sv if svv is None else svv
    return prog["entries"] * (4 + svv) + prog["rows"] * (8 + sv) + prog["levels"] * 4


# DRAM bytes per launch of a kernel (dram__bytes_read.sum + dram__bytes_write.sum averaged
# over every launch of one timed solve, from an ncu capture) on one workload. Each record
# names the SHA-256 prefix of the kernel's source file at capture time: when the file has
# changed since, the record no longer describes the kernel and the line reports no traffic.
MEASURED_TRAFFIC = {
    ("aniso2d_boxes_side1024_boxes8_schur_ilu0+milu0_fp32pc_fgmres50_rtol1e-8", "fg_cgs"):
        dict(bytes=221.3e6, source="kernels_krylov.cu", sha256="724c2ae38ffb830b"),
}


def source_sha(name):
    import hashlib
    path = os.path.join(ROOT, "paper_2303_08881_gb300", "csrc", name)
    try:
        return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]
    except OSError:
        return None


def measured_traffic(workload, kernel):
    rec = MEASURED_TRAFFIC.get((workload, kernel))
    if rec is None:
        return None, "no ncu capture of this kernel on this workload"
    if source_sha(rec["source"]) != rec["sha256"]:
        return None, f"{rec['source']} changed since the ncu capture"
    return rec["bytes"], "ncu capture of this source (sha256 prefix " + rec["sha256"] + ")"


def class_bytes(sz, prec, iters, m, k, gs="mixed3"):
    """Algorithmic bytes summed over the working launches of every kernel class of one
    solve with `iters` Arnoldi steps in cycles of m, inner GMRES of k steps; gs = the
    Gram-Schmidt arithmetic (ilu_opts.gs_precision: the first pass's dots and, with
    mixed2 and mixed3, the second pass's update read the FP32 copy of the basis; mixed3
    reads the basis for the first update and the second pass's dots as two FP32 parts)."""
    n, nnz, n1, n2, ncoff = sz["n"], sz["nnz"], sz["n1"], sz["n2"], sz["nnz_coff"]
    sv = 8 if prec == "fp64" else 4
    svv = 2 if prec == "bf16" else sv  # stored factor values
    full, rem = divmod(iters, m)
    steps = [m] * full + ([rem] if rem else [])
    js = [j for s in steps for j in range(s)]
    cycles = len(steps)
    b = {}
    spmv = 12 * nnz + 4 * (n + 1)
    mixed = gs in ("mixed1", "mixed2", "mixed3")
    v1 = 4 if mixed else 8                          # bytes per basis element read by the first pass's dots
    v2 = 4 if gs in ("mixed2", "mixed3") else 8     # ... by the second pass's update
    w32 = 8 * n if mixed else 0                     # the FP32 copy of w written and read
    vlo = 4 * n if gs == "mixed3" else 0            # the low FP32 part of each new basis vector
    b["fg_spmv_dot"] = sum(spmv + 16 * n + w32 + v1 * (j + 1) * n for j in js)
    if gs == "mixed3":
        # k_fg_cgs_df: both FP32 parts of the basis, w read and written, w1 split written; it
        # ends the step, k_fg_norm exits at once, and k_fg_next forms w2 from the FP32 copy
        # (w1's two parts read; V, V32 and Vlo written)
        b["fg_cgs"] = sum(8 * (j + 1) * n + 24 * n for j in js)
        b["fg_norm"] = 0
        b["fg_next"] = sum(4 * (j + 1) * n + 24 * n for j in js if j + 1 < m)
    else:
        # the first update and the second pass's dots from the FP64 basis
        b["fg_cgs"] = sum(8 * (j + 1) * n + 16 * n for j in js)
        b["fg_norm"] = sum(v2 * (j + 1) * n + 16 * n for j in js)
        b["fg_next"] = sum((16 + (4 if w32 else 0)) * n + vlo for j in js if j + 1 < m)
    b["fg_update"] = sum(8 * s * n + 16 * n for s in steps)
    b["fg_resid"] = (cycles + 1) * (spmv + 24 * n)
    b["fg_scale0"] = (cycles + 1) * 16 * n
    if sz["prog_bj"]["rows"]:
        b["apply_bj"] = iters * (prog_bytes(sz["prog_bj"], sv, svv) + 20 * n)
    else:
        fwd = prog_bytes(sz["prog_fwd"], sv, svv) + prog_bytes(sz["prog_s"], sv, svv) + 12 * n + sv * n
        inner = 0
        for j in range(k):
            inner += (ncoff * (4 + sv) + 4 * (n2 + 1) + prog_bytes(sz["prog_s"], sv, svv)
                      + 3 * sv * n2 + (j + 1) * sv * n2)                      # part A
            inner += 2 * ((j + 1) * sv * n2 + 2 * sv * n2)                     # parts B, C
        bwd = prog_bytes(sz["prog_bwd"], sv, svv) + sv * n1 + k * sv * n2 + 12 * n
        b["apply_fwd"] = iters * fwd
        b["apply_inner"] = iters * inner
        b["apply_bwd"] = iters * bwd
        b["_apply_one"] = fwd + inner + bwd
    return b


# FP64 arithmetic of the outer FGMRES kernels (flops = 2 per multiply-add). The FP64 peak
# they are compared with is measured on the run's GPU (ilu_measure_fp64_peak); the nominal
# figure, 2 fused multiply-adds per SM per clock (152 SMs x 2 x 2 flops x 2.07 GHz), is
# only the fallback when the probe fails.
FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def class_flops64(sz, iters, m, gs="mixed3"):
    """FP64 flops per class (the FP32 arithmetic of the mixed Gram-Schmidt forms is not
    counted: it does not load the FP64 pipe)."""
    n, nnz = sz["n"], sz["nnz"]
    full, rem = divmod(iters, m)
    steps = [m] * full + ([rem] if rem else [])
    js = [j for s in steps for j in range(s)]
    cycles = len(steps)
    f = {}
    mixed = gs in ("mixed1", "mixed2", "mixed3")
    f["fg_spmv_dot"] = sum(2 * nnz + (0 if mixed else 2 * (j + 1) * n) for j in js)
    # mixed3: the update and the dots in double-float (FP32) arithmetic, one FP64 subtraction per
    # row; the second update and the normalisation in k_fg_next, one FP64 addition per row
    f["fg_cgs"] = sum((n if gs == "mixed3" else 4 * (j + 1) * n) for j in js)
    if gs == "mixed3":
        f["fg_norm"] = 0
    else:
        f["fg_norm"] = sum((3 * n if gs == "mixed2" else 2 * (j + 1) * n + 2 * n) for j in js)
    f["fg_next"] = sum(n for j in js if j + 1 < m)
    f["fg_update"] = sum(2 * s * n for s in steps)
    f["fg_resid"] = (cycles + 1) * (2 * nnz + 3 * n)
    f["fg_scale0"] = (cycles + 1) * n
    return f


# ---------------------------------------------------------------------------------------
# clocks


class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = f"/tmp/ilu2l_clocks_{os.getpid()}.csv"

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "power_w_max": max(r["power"] for r in rows), "samples": len(rows), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------


def solver_opts(cfg, prec):
    sol = dict(P.WORKLOAD_SOLVER[cfg])
    restart = sol.pop("restart")
    sol.pop("prec")
    sol["pc_precision"] = prec
    return sol, restart


def host_info():
    """The host's CPU count and model, recorded beside every oracle time."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def oracle_core():
    """The CPU the oracle is pinned to: the last one this process may run on."""
    return max(os.sched_getaffinity(0))


def oracle_leg(cfg, cycles_warmup=0):
    """Runs in a child process pinned to one CPU: oracle setup, then one complete FP64
    FGMRES solve from x0 = 0 to rtol 1e-8 (factors resident). Prints one JSON line."""
    import oracle as O
    core = oracle_core()
    os.sched_setaffinity(0, {core})
    sol, restart = solver_opts(cfg, "fp64")
    sol.pop("pc_precision")
    pr = P.make_workload(cfg)
    t0 = time.perf_counter()
    o = O.Oracle.from_problem(pr, **sol)
    t1 = time.perf_counter()
    for _ in range(cycles_warmup):
        o.fgmres(pr.b, rtol=RTOL, restart=restart, maxit=restart)
    t2 = time.perf_counter()
    out = o.fgmres(pr.b, rtol=RTOL, restart=restart, maxit=20000)
    t3 = time.perf_counter()
    print(json.dumps({"setup_s": t1 - t0, "solve_s": t3 - t2, "iters": out["iters"], "relres": out["relres"],
                      "status": out["status"], "core": core, "name": pr.name}))


def cpu_baseline(cfg):
    """The FP64 oracle as it stands, on one pinned host CPU: setup, then one complete
    FGMRES solve to rtol 1e-8 (no extrapolation)."""
    import oracle
    oracle.build()
    p = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-leg", cfg],
                       capture_output=True, text=True, timeout=3600)
    if p.returncode != 0:
        raise RuntimeError("oracle leg failed: " + p.stderr[-2000:])
    r = json.loads(p.stdout.strip().splitlines()[-1])
    hi = host_info()
    return dict(value=1.0 / r["solve_s"], unit=UNIT, cores=1, kind="oracle",
                sample=(f"one complete FP64 oracle FGMRES solve of {r['name']} to rtol 1e-8 "
                        f"({r['iters']} Arnoldi steps, {r['solve_s']:.1f} s; factors resident, setup "
                        f"{r['setup_s']:.2f} s timed apart), pinned to CPU {r['core']} with sched_setaffinity"),
                time_to_rtol_s=r["solve_s"], setup_s=r["setup_s"], iters=r["iters"], rel_res=r["relres"],
                pinned_cpu=r["core"], **hi)


def max_over_ranks(v, world, device):
    """The largest of every rank's v (collective over the default process group)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(t_ms_local, steps, world, device):
    """N independent replicas, each timing `steps` solves: whole-job solves per second = the
    solves of all ranks over the slowest rank's time. Returns (value, slowest ms)."""
    t_ms = max_over_ranks(t_ms_local, world, device)
    return world * steps / (t_ms / 1000.0), t_ms


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, pinned to one host CPU. Every step
    is one complete FGMRES solve to rtol 1e-8 with the oracle's factors resident (as the
    GPU arm's steps are); a warm-up step runs one FGMRES cycle."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    core = oracle_core()
    os.sched_setaffinity(0, {core})
    cfg = args.workload
    sol, restart = solver_opts(cfg, "fp64")
    sol.pop("pc_precision")
    pr = P.make_workload(cfg)
    t0 = time.perf_counter()
    o = oracle.Oracle.from_problem(pr, **sol)
    setup_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        o.fgmres(pr.b, rtol=RTOL, restart=restart, maxit=restart)
    times, iters = [], None
    t0 = time.perf_counter()
    for _ in range(args.steps):
        t1 = time.perf_counter()
        out = o.fgmres(pr.b, rtol=RTOL, restart=restart, maxit=20000)
        times.append(time.perf_counter() - t1)
        iters = out["iters"]
    wall = time.perf_counter() - t0
    v = args.steps / sum(times)
    hi = host_info()
    cb = dict(value=v, unit=UNIT, cores=1, kind="oracle",
              sample=(f"{args.steps} complete FP64 oracle FGMRES solves of {pr.name} to rtol 1e-8 "
                      f"({iters} Arnoldi steps each; factors resident, setup {setup_s:.2f} s before the clock), "
                      f"pinned to CPU {core} with sched_setaffinity"),
              time_to_rtol_s=sum(times) / len(times), setup_s=setup_s, iters=iters, pinned_cpu=core, **hi)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(cfg, sol_for_config(cfg, args), pr, args.gpus),
            "impl": "reference", "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall, "rel_res": out["relres"]}
    print(json.dumps(line))


def sol_for_config(cfg, args):
    """The GPU arm's solver options (what its `config` describes)."""
    sol, restart = solver_opts(cfg, args.prec or P.WORKLOAD_SOLVER[cfg]["prec"])
    if args.variant:
        sol["variant"] = args.variant
        if args.variant == "rap":
            sol.update(factor_B="ilu0", factor_S="milu0")
    sol["restart"] = restart
    return sol


def bench_config(cfg, sol, pr, world):
    return {"workload": workload_name(cfg), "variant": sol["variant"],
            "factors": f"{sol['factor_B']}+{sol['factor_S']}", "n": pr.n, "nnz": pr.nnz, "p": pr.p,
            "restart": sol["restart"], "rtol": RTOL, "pc_precision": sol["pc_precision"],
            "parallelism": f"replicas{world}",
            "l2": "working set larger than L2 (FGMRES basis alone 0.8 GB)"}


def workload_name(cfg):
    pr_spec = dict(P.WORKLOADS[cfg])
    sol = P.WORKLOAD_SOLVER[cfg]
    fn = pr_spec.pop("fn")
    shape = "_".join(f"{k}{v}" for k, v in pr_spec.items())
    return (f"{fn}_{shape}_{sol['variant']}_{sol['factor_B']}+{sol['factor_S']}_"
            f"{sol['prec']}pc_fgmres{sol['restart']}_rtol1e-8")


def apply_only(args, ilu, h, pr, dev, stream, setup_s, prec, restart, sol):
    """Setup, W warm-up applies, K timed applies (CUDA events); one JSON line."""
    import torch
    r = torch.randn(pr.n, dtype=torch.float64, device=dev)
    z = torch.empty_like(r)
    for _ in range(args.warmup):
        ilu.ilu_apply(h, r, z)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()
    e0.record(stream)
    for _ in range(args.steps):
        ilu.ilu_apply(h, r, z)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    sz = h.sizes()
    by = class_bytes(sz, prec, 1, restart, sol.get("inner_iters", 3))
    byte = by.get("_apply_one") or by.get("apply_bj")
    hbm, kind = _peaks()
    st = h.stats()
    print(json.dumps({"mode": "apply", "workload": workload_name(args.workload), "pc_precision": prec,
                      "apply_ms": ms, "bytes": byte, "gbs": byte / ms / 1e6, "frac": byte / ms / 1e6 / hbm,
                      "setup_s": setup_s, "stream_path": st["stream_path"], "device_error": st["device_error"],
                      "levels": {k: sz[f"prog_{k}"]["levels"] for k in ("bj", "fwd", "s", "bwd")}}))
    h.close()


def latency_floor(ilu, h, stream, k_inner):
    """The least time the apply's dependent steps can take on this GPU, in SM cycles: every
    group barrier of the longest subdomain program of each streamed kernel (forward, k
    inner steps of the local Schur program, backward; or block Jacobi) costs at least one
    dependent level, whose latency for that consumer-group size is measured here
    (ilu_measure_level_latency)."""
    if not h.stats()["stream_path"]:
        return None
    parts = [("bj", 1)] if h.stream_stats("bj")["threads"] else [("fwd", 1), ("s", k_inner), ("bwd", 1)]
    cyc_of, out, total = {}, {}, 0.0
    for prog, mult in parts:
        st = h.stream_stats(prog)
        nt = st["threads"]
        if nt not in cyc_of:
            cyc_of[nt] = ilu.measure_level_latency(nt, stream.cuda_stream)
        c = mult * st["max_barriers"] * cyc_of[nt]
        out[prog] = {"barriers": st["max_barriers"], "times": mult, "threads": nt, "cycles_per_level": cyc_of[nt]}
        total += c
    return {"cycles": total, "programs": out}


def serve_leg(n_requests, workers):
    """The serving workload: Poisson arrivals at 200/s of 2D 9-point / 3D 7-point
    anisotropic problems (30 % repeat an earlier matrix with a new right-hand side) through
    the serving runtime (worker streams, factor cache, 120 GB admission cap). Each
    request's matrix and right-hand side are built before the clock starts (the client's
    input, in host memory at arrival); latency = arrival to solution back on the host."""
    from paper_2303_08881_gb300 import serve as S
    specs = P.serving_trace(n_requests, seed=0)
    built = {}
    reqs = []
    t0 = time.perf_counter()
    for sp in specs:
        pr = P.problem_of_request(sp) if sp.key not in built else None
        if pr is None:  # a repeat: same matrix, new right-hand side
            base = built[sp.key]
            rng = np.random.default_rng(sp.rhs_seed)
            xt = rng.uniform(-1.0, 1.0, base.n)
            pr = P.Problem(name=base.name, n=base.n, rowptr=base.rowptr, colind=base.colind, val=base.val,
                           part=base.part, p=base.p, x_true=xt, b=base.scipy() @ xt, meta=base.meta)
        else:
            built[sp.key] = pr
        reqs.append(S.Request(sp.rid, sp.arrival, sp.key, pr))
    t_build = time.perf_counter() - t0
    rep = S.serve(reqs, workers=workers, cap_bytes=120 << 30, restart=50, rtol=RTOL,
                  opts=dict(variant="schur", factor_B="ilu0", factor_S="milu0", pc_precision="fp32"))
    st = dict(rep.stats)
    st.update(workers=workers, cap_gb=120, cache_hits=rep.cache_hits, evictions=rep.evictions,
              peak_device_gb=rep.peak_bytes / 2**30, wall_s=rep.wall, arrivals_s=specs[-1].arrival,
              unique_matrices=len(built), input_build_s=t_build,
              rows_mean=float(np.mean([r.problem.n for r in reqs])))
    return st


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=list(P.WORKLOADS))
    ap.add_argument("--impl", default="ilu2l", choices=["ilu2l", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving trace in the default run (0 = skip)")
    ap.add_argument("--serve-workers", type=int, default=16)
    ap.add_argument("--variant", default=None, choices=[None, "bj", "schur", "rap"],
                    help="preconditioner variant override (rap: ILU(0) smoother, MILU(0) transfer)")
    ap.add_argument("--mode", default="solve", choices=["solve", "apply", "serve"],
                    help="apply: only time the preconditioner apply (used for kernel profiling)")
    ap.add_argument("--prec", default=None, choices=[None, "fp32", "fp64", "bf16"],
                    help="preconditioner precision (bf16: bfloat16 factor values, FP32 arithmetic)")
    ap.add_argument("--threads", type=int, default=0, help="consumer-group threads override (0 = auto)")
    ap.add_argument("--kernel-path", default="stream", choices=["stream", "generic"])
    ap.add_argument("--order", default="natural", choices=["natural", "rcm", "color"],
                    help="local order inside each group of a subdomain")
    ap.add_argument("--gs", default=None, choices=[None, "fp64", "mixed1", "mixed2", "mixed3"],
                    help="arithmetic of the outer Gram-Schmidt passes (ilu_opts.gs_precision)")
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="measure the consumer-group size of each streamed program at setup (1) or use the rule (0)")
    ap.add_argument("--side", type=int, default=0, help="grid side override (smaller cases for profiling)")
    ap.add_argument("--boxes", type=int, default=0, help="subdomain boxes per side override")
    ap.add_argument("--oracle-leg", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_leg:
        return oracle_leg(args.oracle_leg)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_2303_08881_gb300 as ilu
    from paper_2303_08881_gb300 import _build
    _build.build()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()


    if args.mode == "serve":
        if rank == 0:
            st = serve_leg(args.serve_requests or 2000, args.serve_workers)
            print(json.dumps({"metric": "p50/p99 latency of the serving trace", "value": st["p99_ms"],
                              "unit": "ms (p99)", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
                              "latency": st}))
        return

    cfg = args.workload
    sol, restart = solver_opts(cfg, args.prec or P.WORKLOAD_SOLVER[cfg]["prec"])
    if args.variant:
        sol["variant"] = args.variant
        if args.variant == "rap":
            sol.update(factor_B="ilu0", factor_S="milu0")
    prec = sol["pc_precision"]
    override = {k: v for k, v in (("side", args.side), ("boxes", args.boxes)) if v}
    pr = P.make_workload(cfg, seed=0, **override)
    stream = torch.cuda.current_stream()

    sol["block_threads"] = args.threads
    sol["kernel_path"] = args.kernel_path
    sol["autotune"] = bool(args.autotune) and not args.threads
    if args.order != "natural":
        sol["local_order"] = args.order
    if args.gs:
        sol["gs_precision"] = args.gs
    t0 = time.perf_counter()
    h = ilu.ilu_setup_problem(pr, ilu.Opts(**sol))
    setup_s = time.perf_counter() - t0
    tuning = h.tuning()
    b = torch.from_numpy(pr.b).to(dev)
    x = torch.zeros_like(b)
    if args.mode == "apply":
        return apply_only(args, ilu, h, pr, dev, stream, setup_s, prec, restart, sol)

    def solve(hh):
        x.zero_()
        return ilu.gmres_solve(hh, b, x, rtol=RTOL, restart=restart, maxit=20000)

    for _ in range(args.warmup):
        info = solve(h)
    torch.cuda.synchronize()
    launches0 = h.stats()["kernel_launches"]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()   # an external profiler started with capture off sees only this region
        ev0.record(stream)
        infos = [solve(h) for _ in range(args.steps)]
        ev1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        barrier()
    value, t_ms = replica_value(ev0.elapsed_time(ev1), args.steps, world, dev)
    launches = h.stats()["kernel_launches"] - launches0
    info = infos[-1]
    xs = x.cpu().numpy()
    relres = float(np.linalg.norm(pr.b - pr.scipy() @ xs) / np.linalg.norm(pr.b))
    err_true = float(np.linalg.norm(xs - pr.x_true) / np.linalg.norm(pr.x_true))
    time_to_rtol = t_ms / 1000.0 / args.steps

    # ---- preconditioner apply bandwidth (standalone applies, events on the same stream)
    sz = h.sizes()
    k_inner = sol.get("inner_iters", 3)
    r = torch.randn(pr.n, dtype=torch.float64, device=dev)
    z = torch.empty_like(r)
    for _ in range(3):
        ilu.ilu_apply(h, r, z)
    reps = 20
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ea.record(stream)
    for _ in range(reps):
        ilu.ilu_apply(h, r, z)
    eb.record(stream)
    torch.cuda.synchronize()
    apply_ms = ea.elapsed_time(eb) / reps
    cb_model = class_bytes(sz, prec, 1, restart, k_inner)
    apply_bytes = cb_model.get("_apply_one") or cb_model.get("apply_bj")
    hbm, peak_kind = _peaks()
    pc_apply = {"ms": apply_ms, "bytes": apply_bytes, "gbs": apply_bytes / apply_ms / 1e6,
                "frac": apply_bytes / apply_ms / 1e6 / hbm, "peak_gbs": hbm, "peak_kind": peak_kind,
                "levels": {k: sz[f"prog_{k}"]["levels"] for k in ("bj", "fwd", "s", "bwd")}}

    # ---- measured denominators: FP64 FMA rate and the latency of one dependent level
    try:
        fp64_peak, fp64_kind = ilu.measure_fp64_peak(stream.cuda_stream), "measured: ilu_measure_fp64_peak on this GPU"
    except Exception:
        fp64_peak, fp64_kind = FP64_NOMINAL_TFLOPS, "nominal: 2 FP64 FMA/SM/clock x 152 SMs x 2.07 GHz"
    floor = latency_floor(ilu, h, stream, k_inner)

    # ---- profiled solve: per kernel class device time (events on the launching stream)
    h.profile(True)
    pinfo = solve(h)
    prof = h.profile_read()
    h.profile(False)
    gs = sol.get("gs_precision", "mixed3")
    cbytes = class_bytes(sz, prec, pinfo["iters"], restart, k_inner, gs)
    cflops = class_flops64(sz, pinfo["iters"], restart, gs)
    classes = {}
    for name, (ms, nl) in prof.items():
        if nl == 0:
            continue
        by, fl = cbytes.get(name), cflops.get(name)
        c = {"ms": ms, "launches": nl, "avg_us": 1000.0 * ms / nl, "gbs": (by / ms / 1e6) if by else None}
        # the binding roofline: the larger of bytes / HBM peak and FP64 flops / FP64 peak
        t_hbm = by / (hbm * 1e9) if by else 0.0
        t_alu = fl / (fp64_peak * 1e12) if fl else 0.0
        if t_alu > t_hbm:
            c.update(bound="alu", achieved=fl / ms / 1e9, peak=fp64_peak, unit="TFLOP/s", arith="f64")
        else:
            c.update(bound="hbm", achieved=c["gbs"], peak=hbm, unit="GB/s")
        c["frac"] = (c["achieved"] / c["peak"]) if c["achieved"] else None
        classes[name] = c
    dom = max(classes, key=lambda k: classes[k]["ms"])
    total_prof = sum(c["ms"] for c in classes.values())
    d = classes[dom]
    traffic, traffic_src = measured_traffic(workload_name(cfg), dom)
    alg_bytes = cbytes.get(dom) / d["launches"] if cbytes.get(dom) else None
    roofline = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"],
                "unit": d["unit"], "frac": d["frac"], "traffic": traffic,
                "traffic_unit": "DRAM bytes per launch", "traffic_source": traffic_src,
                "algorithmic_bytes_per_launch": alg_bytes,
                "traffic_per_algorithmic": (traffic / alg_bytes) if (traffic and alg_bytes) else None,
                "arith": d.get("arith"),
                "share": d["ms"] / total_prof,
                "peak_kind": fp64_kind if d["bound"] == "alu" else peak_kind,
                "avg_launch_us": d["avg_us"], "launches": d["launches"]}
    # the preconditioner apply (the method's hot path) against HBM and against the floor its
    # dependent levels set
    clk_mhz = 2070.0
    roofline_pc = {"kernel": "pc_apply (forward + inner + backward)", "bound": "hbm", "achieved": pc_apply["gbs"],
                   "peak": hbm, "unit": "GB/s", "frac": pc_apply["frac"], "peak_kind": peak_kind,
                   "algorithmic_bytes": apply_bytes, "apply_us": 1000.0 * apply_ms,
                   "latency_floor_us": floor["cycles"] / clk_mhz if floor else None,
                   "frac_of_latency_floor": (floor["cycles"] / clk_mhz) / (1000.0 * apply_ms) if floor else None,
                   "latency_floor": floor}

    # ---- mixed vs FP64 (same workload, FP64 preconditioner)
    mixed = None
    if not args.no_fp64 and prec == "fp32":
        sol64 = dict(sol)
        sol64["pc_precision"] = "fp64"
        h64 = ilu.ilu_setup_problem(pr, ilu.Opts(**sol64))
        for _ in range(max(1, args.warmup - 1)):
            i64 = solve(h64)
        torch.cuda.synchronize()
        ev0.record(stream)
        n64 = max(1, min(args.steps, 3))
        for _ in range(n64):
            i64 = solve(h64)
        ev1.record(stream)
        torch.cuda.synchronize()
        t64 = ev0.elapsed_time(ev1) / 1000.0 / n64
        mixed = {"fp64_time_to_rtol_s": t64, "fp64_iters": i64["iters"], "fp32_time_to_rtol_s": time_to_rtol,
                 "fp32_iters": info["iters"], "speedup": t64 / time_to_rtol,
                 "fp64_rel_res_true": i64["rel_res_true"]}
        h64.close()

    # ---- end to end through the C ABI with host buffers (setup included)
    e2e = None
    if not args.no_e2e:
        b_host = torch.from_numpy(pr.b).pin_memory()
        x_host = torch.empty(pr.n, dtype=torch.float64).pin_memory()
        ne2e = max(1, min(args.steps, 3))
        o = ilu.Opts(**sol)
        he = ilu.ilu_setup_problem(pr, o)   # warm (first-touch allocations, module load)
        he.close()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(ne2e):
            he = ilu.ilu_setup_problem(pr, o)
            bd = b_host.to(dev, non_blocking=True)
            xd = torch.zeros_like(bd)
            ilu.gmres_solve(he, bd, xd, rtol=RTOL, restart=restart, maxit=20000)
            x_host.copy_(xd, non_blocking=True)
            torch.cuda.synchronize()
            he.close()
        te = max_over_ranks((time.perf_counter() - t0) / ne2e, world, dev)
        h2d = pr.rowptr.nbytes + pr.colind.nbytes + pr.val.nbytes + pr.part.nbytes + pr.b.nbytes
        e2e = {"value": world / te, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(8 * pr.n),
               "time_s": te, "includes": "ilu_setup from host CSR + H2D b + gmres_solve + D2H x + ilu_free"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cpu = cpu_baseline(cfg)

    h.close()
    latency = None
    if rank == 0 and world == 1 and args.serve_requests > 0 and cfg == DEFAULT_WORKLOAD:
        latency = serve_leg(args.serve_requests, args.serve_workers)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
            "config": dict(bench_config(cfg, dict(sol, restart=restart), pr, world),
                           **({"grid_override": override} if override else {})),
            "roofline": roofline, "roofline_pc_apply": roofline_pc,
            "time_to_rtol_s": time_to_rtol, "iters": info["iters"], "rel_res_true": relres,
            "err_vs_x_true": err_true, "setup_s": setup_s, "tuning": tuning, "fp64_peak_tflops": fp64_peak,
            "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": int(launches),
            "clocks": clk.summary(), "mixed_vs_fp64": mixed, "pc_apply": pc_apply, "latency": latency,
            "kernels": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in c.items()}
                        for k, c in classes.items()},
        }
        if line["clocks"] and line["clocks"].get("sm_mhz"):
            clk_mhz = line["clocks"]["sm_mhz"]
            if floor:
                roofline_pc["latency_floor_us"] = floor["cycles"] / clk_mhz
                roofline_pc["frac_of_latency_floor"] = roofline_pc["latency_floor_us"] / (1000.0 * apply_ms)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
