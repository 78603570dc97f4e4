"""Python binding of ilu2l, the GB300-native two-level ILU domain-decomposition
preconditioner and flexible GMRES solver (C ABI in ``include/ilu2l.h``).

Argument marshalling only: every step of the setup's numeric phase, the apply and the
solver runs in the CUDA kernels of ``libilu2l.so``. Device vectors are torch CUDA
float64 tensors (PyTorch provides device memory and streams); matrices and partitions
are host numpy arrays. There is no CPU fallback: without the built library every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libilu2l.so")

ILU_OK, ILU_ERR_ARG, ILU_ERR_CSR, ILU_ERR_OOM, ILU_ERR_ZERO_PIVOT = 0, 1, 2, 3, 4
ILU_ERR_NOT_CONVERGED, ILU_ERR_BREAKDOWN, ILU_ERR_TIMEOUT, ILU_ERR_CUDA = 5, 6, 7, 8
ILU_ERR_TOO_LARGE, ILU_ERR_UNSUPPORTED = 9, 10
VARIANTS = {"bj": 0, "schur": 1, "rap": 2}
FACTORS = {"ilu0": 0, "milu0": 1, "ilut": 2, "pmilu0": 3}  # pmilu0: factor_S of SCHUR only
FORMS = {"auto": 0, "wz": 1, "ef": 2}
PRECS = {"fp64": 0, "fp32": 1, "bf16": 2}  # bf16: FP32 arithmetic, bfloat16 factor values
LEVELS = {"LA": 0, "UA": 1, "LB": 2, "UB": 3, "LS": 4, "US": 5}


class IluError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_str(status)} (status {status})")
        self.status = status


class ilu_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("rowptr", C.c_void_p),
                ("colind", C.c_void_p), ("val", C.c_void_p)]


class ilu_opts(C.Structure):
    _fields_ = [("variant", C.c_int32), ("factor_B", C.c_int32), ("factor_S", C.c_int32),
                ("form", C.c_int32), ("ilut_tau", C.c_double), ("ilut_p", C.c_int32),
                ("inner_iters", C.c_int32), ("pc_precision", C.c_int32), ("ordering", C.c_int32),
                ("pivot_eps", C.c_double), ("stream", C.c_void_p), ("spin_limit", C.c_uint64),
                ("use_graphs", C.c_int32), ("block_threads", C.c_int32),
                ("analysis_only", C.c_int32), ("kernel_path", C.c_int32), ("inner_launch", C.c_int32),
                ("fill_level", C.c_int32), ("l1_block", C.c_int32), ("chain_sched", C.c_int32),
                ("gs_precision", C.c_int32), ("autotune", C.c_int32), ("ilut_setup", C.c_int32)]


class ilu_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("rel_res_true", C.c_double),
                ("rel_res_est", C.c_double), ("setup_ms", C.c_double), ("solve_ms", C.c_double),
                ("status", C.c_int32), ("npert", C.c_int32)]


_lib = None


def lib():
    """Load libilu2l.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        P, I, D, I64 = C.c_void_p, C.c_int32, C.c_double, C.c_int64
        sig = {
            "ilu_opts_default": (None, [P]),
            "ilu_setup": (I, [P, P, I, P, P]),
            "ilu_apply": (I, [P, P, P]),
            "gmres_solve": (I, [P, P, P, D, I, I, P]),
            "ilu_free": (I, [P]),
            "ilu_status_str": (C.c_char_p, [I]),
            "ilu_get_sizes": (I, [P, P]),
            "ilu_get_perm": (I, [P, P, P, P, P, P]),
            "ilu_get_levels": (I, [P, I, P, P]),
            "ilu_get_local_factor": (I, [P, I, I, P]),
            "ilu_get_local_pattern": (I, [P, I, P, P, P]),
            "ilu_spmv": (I, [P, P, P]),
            "ilu_inner_solve": (I, [P, P, P]),
            "ilu_profile": (I, [P, I]),
            "ilu_profile_read": (I, [P, P, P, P, P]),
            "ilu_get_stats": (I, [P, P]),
            "ilu_get_stream_stats": (I, [P, I, P]),
            "ilu_get_times": (I, [P, P]),
            "ilu_get_stream": (I, [P, I, P, P, P]),
            "ilu_inner_solve_noalloc": (I, [P, P, P]),
            "ilu_measure_fp64_peak": (I, [P, P]),
            "ilu_get_krylov": (I, [P, I, I, P]),
            "ilu_get_tuning": (I, [P, P, P, P]),
            "ilu_measure_level_latency": (I, [P, I, P]),
            "ilu_get_ilut_factor": (I, [P, I, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_str(s: int) -> str:
    try:
        return lib().ilu_status_str(int(s)).decode()
    except RuntimeError:
        return "unknown"


def _ptr(t, n=None, device=None):
    """device pointer of a contiguous torch CUDA float64 tensor; with n, its length must be
    n, and with device (a CUDA ordinal), it must live on that device (the kernels read and
    write exactly n elements on the handle's device)"""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    if device is not None and t.device.index != device:
        raise ValueError(f"tensor on cuda:{t.device.index}, the handle on cuda:{device}")
    return C.c_void_p(t.data_ptr())


def _np(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


@dataclass
class Opts:
    """Mirror of ilu_opts with readable enums."""
    variant: str = "schur"
    factor_B: str = "ilu0"
    factor_S: str = "milu0"
    form: str = "auto"
    ilut_tau: float = 1e-3
    ilut_p: int = 10
    inner_iters: int = 3
    pc_precision: str = "fp32"
    pivot_eps: float = 1e-8
    use_graphs: bool = True
    block_threads: int = 0
    stream: int | None = None
    spin_limit: int = 0
    analysis_only: bool = False
    kernel_path: str = "stream"     # "stream" (TMA-streamed level programs) or "generic"
    inner_launch: str = "single"    # inner Schur GMRES: "single" cooperative launch or "per_step"
    local_order: str = "natural"    # order inside each group of a subdomain: "natural", "rcm" or "color"
    fill_level: int = 0             # k > 0: ILU(k) / MILU(k) in the level-k fill pattern
    l1_block: bool = False          # block Jacobi: l1-BJ diagonal augmentation
    chain_sched: str = "auto"       # interface rows: "auto" (cheaper of levels / chains), "levels", "chains"
    gs_precision: str = "mixed3"    # FGMRES Gram-Schmidt: "fp64", "mixed1" (FP32 first-pass dots), "mixed2" (+ FP32 second update),
    #                                 "mixed3" (+ the first update and second-pass dots in double-float from a split basis)
    autotune: bool = False          # measure the consumer-group size of each streamed program at setup
    ilut_setup: str = "device"      # factor_B = "ilut": numeric factorisation on the "device" or the "host"

    def to_c(self) -> ilu_opts:
        o = ilu_opts()
        lib().ilu_opts_default(C.byref(o))
        o.variant = VARIANTS[self.variant]
        o.factor_B = FACTORS[self.factor_B]
        o.factor_S = FACTORS[self.factor_S]
        o.form = FORMS[self.form]
        o.ilut_tau = float(self.ilut_tau)
        o.ilut_p = int(self.ilut_p)
        o.inner_iters = int(self.inner_iters)
        o.pc_precision = PRECS[self.pc_precision]
        o.pivot_eps = float(self.pivot_eps)
        o.use_graphs = int(bool(self.use_graphs))
        o.block_threads = int(self.block_threads)
        o.spin_limit = int(self.spin_limit)
        o.analysis_only = int(bool(self.analysis_only))
        o.kernel_path = {"stream": 0, "generic": 1}[self.kernel_path]
        o.inner_launch = {"single": 0, "per_step": 1}[self.inner_launch]
        o.ordering = {"natural": 0, "rcm": 1, "color": 2}[self.local_order]
        o.fill_level = int(self.fill_level)
        o.l1_block = int(bool(self.l1_block))
        o.chain_sched = {"auto": 0, "levels": 1, "chains": 2}[self.chain_sched]
        o.gs_precision = {"fp64": 0, "mixed1": 1, "mixed2": 2, "mixed3": 3}[self.gs_precision]
        o.autotune = int(bool(self.autotune))
        o.ilut_setup = {"device": 0, "host": 1}[self.ilut_setup]
        if self.analysis_only:
            o.stream = None
        elif self.stream is None:
            import torch
            o.stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        else:
            o.stream = C.c_void_p(int(self.stream))
        return o


class Handle:
    """Owns one ilu2l handle (ilu_free on close / garbage collection)."""

    def __init__(self, ptr: C.c_void_p, n: int, p: int, opts: Opts):
        self._h = ptr
        self.n = n
        self.p = p
        self.opts = opts
        self.device = None  # the CUDA ordinal current at setup (None: analysis only / no GPU)
        if not opts.analysis_only:
            import torch
            if torch.cuda.is_available():
                self.device = torch.cuda.current_device()

    @property
    def ptr(self):
        if not self._h:
            raise RuntimeError("handle already freed")
        return self._h

    def close(self):
        if self._h:
            lib().ilu_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- introspection ----
    def sizes(self) -> dict:
        out = np.zeros(24, np.int64)
        _check(lib().ilu_get_sizes(self.ptr, out.ctypes.data_as(C.c_void_p)), "ilu_get_sizes")
        keys = ["n", "p", "n1", "n2", "nnz", "nnz_coff", "npert", "nlev_LB", "nlev_UB",
                "nlev_LS", "nlev_US", "max_ns"]
        d = dict(zip(keys, [int(v) for v in out[:12]]))
        for i, name in enumerate(["bj", "fwd", "s", "bwd"]):
            d[f"prog_{name}"] = dict(rows=int(out[12 + 3 * i]), entries=int(out[13 + 3 * i]),
                                     levels=int(out[14 + 3 * i]))
        return d

    def perm(self) -> dict:
        n, p = self.n, self.p
        perm = np.empty(n, np.int32)
        iperm = np.empty(n, np.int32)
        int_ptr = np.empty(p + 1, np.int32)
        if_ptr = np.empty(p + 1, np.int32)
        iface = np.empty(n, np.int32)
        _check(lib().ilu_get_perm(self.ptr, *[a.ctypes.data_as(C.c_void_p) for a in
                                              (perm, iperm, int_ptr, if_ptr, iface)]), "ilu_get_perm")
        return dict(perm=perm, iperm=iperm, int_ptr=int_ptr, if_ptr=if_ptr, iface=iface)

    def levels(self, which) -> tuple[np.ndarray, int]:
        w = LEVELS[which] if isinstance(which, str) else int(which)
        lev = np.empty(self.n, np.int32)
        nl = C.c_int32(0)
        _check(lib().ilu_get_levels(self.ptr, w, lev.ctypes.data_as(C.c_void_p), C.byref(nl)),
               "ilu_get_levels")
        return lev, nl.value

    def local_pattern(self, s: int):
        """(rowptr, colind) of local block s as stored for the factorisation."""
        pm = self.perm()
        rows = int(pm["int_ptr"][s + 1] - pm["int_ptr"][s] + pm["if_ptr"][s + 1] - pm["if_ptr"][s])
        nnz = C.c_int32(0)
        _check(lib().ilu_get_local_pattern(self.ptr, int(s), None, None, C.byref(nnz)), "ilu_get_local_pattern")
        rp = np.empty(rows + 1, np.int32)
        ci = np.empty(nnz.value, np.int32)
        _check(lib().ilu_get_local_pattern(self.ptr, int(s), rp.ctypes.data_as(C.c_void_p),
                                           ci.ctypes.data_as(C.c_void_p), C.byref(nnz)), "ilu_get_local_pattern")
        return rp, ci

    def local_factor(self, s: int, fact: int, nnz: int) -> np.ndarray:
        v = np.empty(nnz)
        _check(lib().ilu_get_local_factor(self.ptr, int(s), int(fact), v.ctypes.data_as(C.c_void_p)),
               "ilu_get_local_factor")
        return v

    def ilut_factor(self, s: int):
        """ILUT factor of local block s (B_s, or A_s for block Jacobi): combined L\\U CSR rows
        (rowptr, colind, FP64 values) in the local order."""
        nnz = C.c_int32(0)
        _check(lib().ilu_get_ilut_factor(self.ptr, int(s), None, None, None, C.byref(nnz)), "ilu_get_ilut_factor")
        pm = self.perm()
        rows = int(pm["int_ptr"][s + 1] - pm["int_ptr"][s])
        if self.opts.variant == "bj":
            rows += int(pm["if_ptr"][s + 1] - pm["if_ptr"][s])
        rp = np.empty(rows + 1, np.int32)
        ci = np.empty(nnz.value, np.int32)
        v = np.empty(nnz.value)
        _check(lib().ilu_get_ilut_factor(self.ptr, int(s), rp.ctypes.data_as(C.c_void_p),
                                         ci.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p),
                                         C.byref(nnz)), "ilu_get_ilut_factor")
        return rp, ci, v

    def spmv(self, x, y):
        _check(lib().ilu_spmv(self.ptr, _ptr(x, self.n, self.device), _ptr(y, self.n, self.device)), "ilu_spmv")

    def inner_solve(self, gp, y):
        n2 = self.sizes()["n2"]
        _check(lib().ilu_inner_solve(self.ptr, _ptr(gp, n2, self.device), _ptr(y, n2, self.device)),
               "ilu_inner_solve")

    def stats(self) -> dict:
        out = np.zeros(16, np.int64)
        _check(lib().ilu_get_stats(self.ptr, out.ctypes.data_as(C.c_void_p)), "ilu_get_stats")
        progs = {name: dict(record_entries=int(out[6 + 2 * i]), threads=int(out[7 + 2 * i]))
                 for i, name in enumerate(["bj", "fwd", "s", "bwd"])}
        return dict(kernel_launches=int(out[0]), graph_launches=int(out[1]),
                    kernels_per_cycle=int(out[2]), row_ctas=int(out[3]), device_error=int(out[4]),
                    stream_path=bool(out[5]), programs=progs, inner_single_launch=bool(out[14]),
                    device_bytes=int(out[15]))

    def times(self) -> dict:
        """Wall-clock ms: host analysis and device part of the setup, the last solve and
        its graph build, the ILUT factorisation (inside the host analysis) and where it ran."""
        out = np.zeros(7)
        _check(lib().ilu_get_times(self.ptr, out.ctypes.data_as(C.c_void_p)), "ilu_get_times")
        return dict(host_ms=float(out[0]), device_ms=float(out[1]), solve_ms=float(out[2]), graph_ms=float(out[3]),
                    ilut_ms=float(out[4]), ilut_on_device=bool(out[5]), ilut_kernel_ms=float(out[6]))

    def stream_stats(self, program: str) -> dict:
        """Shape of a streamed level program ("bj", "fwd", "s", "bwd"): record width,
        consumer threads, chunks, waves, records, skip records, group barriers of the
        longest subdomain program, levels of the deepest one, ring bytes, whether the
        working vectors stay in shared memory, scan waves, dependent steps (barriers + scan
        waves) and the subdomains whose interface rows run as chains."""
        out = np.zeros(13, np.int64)
        idx = ["bj", "fwd", "s", "bwd"].index(program)
        _check(lib().ilu_get_stream_stats(self.ptr, idx, out.ctypes.data_as(C.c_void_p)), "ilu_get_stream_stats")
        keys = ["record_entries", "threads", "chunks", "waves", "records", "skips", "max_barriers", "max_levels",
                "ring_bytes", "vector_in_shared", "max_scan_waves", "max_steps", "chain_sections"]
        return {k: int(v) for k, v in zip(keys, out)}

    def stream(self, program: str) -> dict:
        """The streamed program ("bj", "fwd", "s", "bwd") as built on the host: raw chunk
        bytes, per-subdomain chunk offsets and the record geometry."""
        idx = ["bj", "fwd", "s", "bwd"].index(program)
        meta = np.zeros(6, np.int64)
        _check(lib().ilu_get_stream(self.ptr, idx, None, None, meta.ctypes.data_as(C.c_void_p)), "ilu_get_stream")
        blob = np.zeros(int(meta[0]), np.uint8)
        ch0 = np.zeros(self.sizes()["p"] + 1, np.int32)
        _check(lib().ilu_get_stream(self.ptr, idx, blob.ctypes.data_as(C.c_void_p), ch0.ctypes.data_as(C.c_void_p),
                                    meta.ctypes.data_as(C.c_void_p)), "ilu_get_stream")
        return dict(blob=blob, ch0=ch0, chunk=int(meta[1]), rw=int(meta[2]), val_bytes=int(meta[3]),
                    threads=int(meta[4]), x_bytes=int(meta[5]))

    def tuning(self) -> dict:
        """Consumer threads chosen per streamed program, the measured apply times of the
        candidates (32, 64, 96, 128 threads; 0 = not measured) and how they were chosen."""
        nt = np.zeros(4, np.int32)
        ms = np.zeros(16)
        st = C.c_int32(0)
        _check(lib().ilu_get_tuning(self.ptr, nt.ctypes.data_as(C.c_void_p), ms.ctypes.data_as(C.c_void_p),
                                    C.byref(st)), "ilu_get_tuning")
        names = ["bj", "fwd", "s", "bwd"]
        return {"state": ["rule", "measured", "remembered"][st.value],
                "threads": {names[i]: int(nt[i]) for i in range(4) if nt[i]},
                "apply_ms": {names[i]: {c: float(ms[4 * i + k]) for k, c in enumerate((32, 64, 96, 128))
                                        if ms[4 * i + k] > 0} for i in range(4) if nt[i]}}

    def krylov(self, which: str, k: int) -> np.ndarray:
        """The last solve's basis vectors v_0..v_{k-1} ("V") or z_0..z_{k-1} ("Z"), k x n."""
        out = np.empty((k, self.n))
        _check(lib().ilu_get_krylov(self.ptr, {"V": 0, "Z": 1}[which], int(k), out.ctypes.data_as(C.c_void_p)),
               "ilu_get_krylov")
        return out

    def inner_solve_noalloc(self, gp, y):
        """ilu_inner_solve with the library's fixed workspace instead of the handle's
        (allocates nothing; see include/ilu2l.h)."""
        n2 = self.sizes()["n2"]
        _check(lib().ilu_inner_solve_noalloc(self.ptr, _ptr(gp, n2, self.device), _ptr(y, n2, self.device)),
               "ilu_inner_solve_noalloc")

    def profile(self, enable: bool):
        _check(lib().ilu_profile(self.ptr, int(enable)), "ilu_profile")

    def profile_read(self) -> dict:
        cap = 32
        names = (C.c_char_p * cap)()
        ms = np.zeros(cap)
        nl = np.zeros(cap, np.int64)
        cnt = C.c_int32(cap)
        _check(lib().ilu_profile_read(self.ptr, C.cast(names, C.c_void_p), ms.ctypes.data_as(C.c_void_p),
                                      nl.ctypes.data_as(C.c_void_p), C.byref(cnt)), "ilu_profile_read")
        return {names[i].decode(): (float(ms[i]), int(nl[i])) for i in range(min(cnt.value, cap))}


def _check(st, what):
    if st != ILU_OK:
        raise IluError(st, what)


# ---- the C-ABI calls, same names ----------------------------------------------------


def ilu_setup(n, rowptr, colind, val, part, p, opts: Opts | None = None) -> Handle:
    """Setup of the preconditioner for the host CSR matrix (rowptr, colind, val) and the
    partition part[n] into p subdomains. Raises IluError on a non-OK status."""
    opts = opts or Opts()
    rowptr = _np(rowptr, np.int32)
    colind = _np(colind, np.int32)
    val = _np(val, np.float64)
    part = _np(part, np.int32)
    A = ilu_csr(int(n), int(rowptr[-1]) if rowptr.size else 0, rowptr.ctypes.data,
                colind.ctypes.data, val.ctypes.data)
    o = opts.to_c()
    h = C.c_void_p()
    _check(lib().ilu_setup(C.byref(A), part.ctypes.data_as(C.c_void_p), int(p), C.byref(o), C.byref(h)),
           "ilu_setup")
    return Handle(h, int(n), int(p), opts)


def ilu_setup_problem(prob, opts: Opts | None = None) -> Handle:
    return ilu_setup(prob.n, prob.rowptr, prob.colind, prob.val, prob.part, prob.p, opts)


def ilu_apply(h: Handle, r, z) -> None:
    """z = M^{-1} r for torch CUDA float64 vectors in the original ordering."""
    _check(lib().ilu_apply(h.ptr, _ptr(r, h.n, h.device), _ptr(z, h.n, h.device)), "ilu_apply")


def gmres_solve(h: Handle, b, x, rtol: float = 1e-8, restart: int = 50, maxit: int = 10000,
                raise_on_fail: bool = False) -> dict:
    """FGMRES(restart) for A x = b; x (torch CUDA float64) holds x0 on entry."""
    info = ilu_solve_info()
    st = lib().gmres_solve(h.ptr, _ptr(b, h.n, h.device), _ptr(x, h.n, h.device), float(rtol), int(restart), int(maxit), C.byref(info))
    if st not in (ILU_OK, ILU_ERR_NOT_CONVERGED) or (raise_on_fail and st != ILU_OK):
        raise IluError(st, "gmres_solve")
    return dict(status=int(st), iters=info.iters, restarts=info.restarts,
                rel_res_true=info.rel_res_true, rel_res_est=info.rel_res_est,
                setup_ms=info.setup_ms, solve_ms=info.solve_ms, npert=info.npert)


def ilu_free(h: Handle) -> None:
    h.close()


def measure_fp64_peak(stream=None) -> float:
    """FP64 FMA throughput of the current device in TFLOP/s (ilu_measure_fp64_peak)."""
    v = C.c_double(0.0)
    _check(lib().ilu_measure_fp64_peak(C.c_void_p(int(stream) if stream else 0), C.byref(v)),
           "ilu_measure_fp64_peak")
    return v.value


def measure_level_latency(threads: int, stream=None) -> float:
    """SM clock cycles of one dependent level of `threads` threads (ilu_measure_level_latency)."""
    v = C.c_double(0.0)
    _check(lib().ilu_measure_level_latency(C.c_void_p(int(stream) if stream else 0), int(threads), C.byref(v)),
           "ilu_measure_level_latency")
    return v.value


__all__ = ["Opts", "Handle", "IluError", "ilu_setup", "ilu_setup_problem", "ilu_apply",
           "gmres_solve", "ilu_free", "status_str", "lib", "LIB_PATH"]
