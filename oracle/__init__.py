"""FP64 CPU oracle (plain C, ``oracle.c``) and its ctypes binding.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg may import this package. It shares no code with the CUDA path; it is
compiled from ``oracle.c`` by :func:`build` with plain ``gcc -O2 -ffp-contract=off``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")

ILU0, MILU0, ILUT, EXACT, PMILU0 = 0, 1, 2, 3, 4
BJ, SCHUR, RAP = 0, 1, 2
FORM_AUTO, FORM_WZ, FORM_EF = 0, 1, 2
ORDER_NATURAL, ORDER_RCM, ORDER_COLOR = 0, 1, 2
OK, ERR_ARG, ERR_CSR, ERR_OOM, ERR_ZERO_PIVOT, ERR_NOT_CONVERGED = 0, 1, 2, 3, 4, 5

_FACT = {"ilu0": ILU0, "milu0": MILU0, "ilut": ILUT, "exact": EXACT, "pmilu0": PMILU0}
_VAR = {"bj": BJ, "schur": SCHUR, "rap": RAP}


def build(force: bool = False) -> str:
    """Compile liborc.so (plain C, no floating-point contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Opts(C.Structure):
    _fields_ = [("variant", C.c_int), ("factor_B", C.c_int), ("factor_S", C.c_int),
                ("form", C.c_int), ("ilut_tau", C.c_double), ("ilut_p", C.c_int),
                ("inner_iters", C.c_int), ("pivot_eps", C.c_double), ("local_order", C.c_int),
                ("fill_level", C.c_int), ("l1_block", C.c_int), ("store_bf16", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        I = C.c_int
        D = C.c_double
        sig = {
            "orc_csr_check": (I, [I, P, P]),
            "orc_spmv": (None, [I, P, P, P, P, P]),
            "orc_ilu0_csr": (I, [I, P, P, P, I, D, P, P]),
            "orc_ilut_csr": (P, [I, P, P, P, D, I, D, P]),
            "orc_factor_nnz": (I, [P]),
            "orc_factor_get": (None, [P, P, P, P]),
            "orc_factor_free": (None, [P]),
            "orc_trsv_lower_unit": (None, [I, P, P, P, P, P]),
            "orc_trsv_upper": (None, [I, P, P, P, P, P]),
            "orc_levels_csr": (I, [I, P, P, I, P]),
            "orc_classify": (I, [I, P, P, P, I, P]),
            "orc_permutation": (I, [I, P, I, P, P, P, P, P]),
            "orc_rcm": (I, [I, P, P, P]),
            "orc_color": (I, [I, P, P, P, P]),
            "orc_round_bf16": (D, [D]),
            "orc_iluk_pattern": (P, [I, P, P, P, I, P]),
            "orc_opts_default": (None, [P]),
            "orc_setup": (P, [I, P, P, P, P, I, P, P]),
            "orc_free": (None, [P]),
            "orc_sizes": (None, [P, P]),
            "orc_get_perm": (None, [P, P, P, P, P, P]),
            "orc_get_levels": (I, [P, I, P]),
            "orc_local_nnz": (I, [P, I]),
            "orc_local_rows": (I, [P, I]),
            "orc_local_csr": (None, [P, I, P, P, P]),
            "orc_local_factor": (I, [P, I, I, P]),
            "orc_coff_nnz": (I, [P]),
            "orc_coff_csr": (None, [P, P, P, P]),
            "orc_schur_dense": (I, [P, P]),
            "orc_sapprox_dense": (I, [P, P]),
            "orc_apply": (I, [P, P, P]),
            "orc_inner_gmres": (I, [P, P, P]),
            "orc_fgmres": (I, [P, P, P, D, I, I, P, P, P, I, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- primitives ----------------------------------------------------------------------


def csr_check(n, rowptr, colind) -> int:
    rowptr, colind = _i32(rowptr), _i32(colind)
    return lib().orc_csr_check(n, _p(rowptr), _p(colind))


def spmv(n, rowptr, colind, val, x):
    rowptr, colind, val, x = _i32(rowptr), _i32(colind), _f64(val), _f64(x)
    y = np.empty(n)
    lib().orc_spmv(n, _p(rowptr), _p(colind), _p(val), _p(x), _p(y))
    return y


def ilu0(n, rowptr, colind, val, milu=False, pivot_eps=1e-8):
    """Combined L\\U values in the pattern of A; returns (values, status, npert)."""
    rowptr, colind, val = _i32(rowptr), _i32(colind), _f64(val)
    out = np.empty_like(val)
    npert = C.c_int(0)
    st = lib().orc_ilu0_csr(n, _p(rowptr), _p(colind), _p(val), int(milu), pivot_eps, _p(out),
                            C.byref(npert))
    return out, st, npert.value


def ilut(n, rowptr, colind, val, tau, p, pivot_eps=1e-8):
    """Returns (rowptr, colind, val) of the combined factor."""
    rowptr, colind, val = _i32(rowptr), _i32(colind), _f64(val)
    st = C.c_int(0)
    f = lib().orc_ilut_csr(n, _p(rowptr), _p(colind), _p(val), tau, int(p), pivot_eps,
                           C.byref(st))
    if st.value != OK:
        raise RuntimeError(f"ilut status {st.value}")
    nnz = lib().orc_factor_nnz(f)
    rp = np.empty(n + 1, np.int32)
    ci = np.empty(nnz, np.int32)
    v = np.empty(nnz)
    lib().orc_factor_get(f, _p(rp), _p(ci), _p(v))
    lib().orc_factor_free(f)
    return rp, ci, v


def trsv_lower_unit(n, rowptr, colind, val, b):
    rowptr, colind, val, b = _i32(rowptr), _i32(colind), _f64(val), _f64(b)
    x = np.empty(n)
    lib().orc_trsv_lower_unit(n, _p(rowptr), _p(colind), _p(val), _p(b), _p(x))
    return x


def trsv_upper(n, rowptr, colind, val, b):
    rowptr, colind, val, b = _i32(rowptr), _i32(colind), _f64(val), _f64(b)
    x = np.empty(n)
    lib().orc_trsv_upper(n, _p(rowptr), _p(colind), _p(val), _p(b), _p(x))
    return x


def levels(n, rowptr, colind, upper=False):
    rowptr, colind = _i32(rowptr), _i32(colind)
    lev = np.empty(n, np.int32)
    nl = lib().orc_levels_csr(n, _p(rowptr), _p(colind), int(upper), _p(lev))
    return lev, nl


def classify(n, rowptr, colind, part, p):
    rowptr, colind, part = _i32(rowptr), _i32(colind), _i32(part)
    iface = np.empty(n, np.int32)
    st = lib().orc_classify(n, _p(rowptr), _p(colind), _p(part), p, _p(iface))
    if st != OK:
        raise ValueError(f"classify status {st}")
    return iface


def iluk_pattern(n, rowptr, colind, val, k):
    """Level-k fill pattern of ILU(k): (rowptr, colind, val) with A's values and zeros at
    the fill positions."""
    rowptr, colind, val = _i32(rowptr), _i32(colind), _f64(val)
    st = C.c_int(0)
    f = lib().orc_iluk_pattern(int(n), _p(rowptr), _p(colind), _p(val), int(k), C.byref(st))
    if not f:
        raise ValueError(f"iluk_pattern status {st.value}")
    nnz = lib().orc_factor_nnz(f)
    rp = np.empty(n + 1, np.int32)
    ci = np.empty(nnz, np.int32)
    v = np.empty(nnz)
    lib().orc_factor_get(f, _p(rp), _p(ci), _p(v))
    lib().orc_factor_free(f)
    return rp, ci, v


def round_bf16(x: float) -> float:
    """x rounded to the nearest bfloat16 value, ties to even."""
    return lib().orc_round_bf16(float(x))


def color(n, rowptr, colind):
    """Greedy multicolouring of the symmetrised graph of a square pattern (ascending index,
    smallest colour free among the earlier neighbours): (colour of each node, the nodes
    listed by (colour, index), number of colours)."""
    rowptr, colind = _i32(rowptr), _i32(colind)
    col = np.empty(max(n, 1), np.int32)
    order = np.empty(max(n, 1), np.int32)
    nc = lib().orc_color(int(n), _p(rowptr), _p(colind), _p(col), _p(order))
    if nc < 0:
        raise RuntimeError(f"color status {nc}")
    return col[:n], order[:n], nc


def rcm(n, rowptr, colind):
    """Reverse Cuthill-McKee order of the symmetrised graph of a square pattern:
    order[k] = the node placed k-th."""
    rowptr, colind = _i32(rowptr), _i32(colind)
    order = np.empty(n, np.int32)
    st = lib().orc_rcm(int(n), _p(rowptr), _p(colind), _p(order))
    if st != OK:
        raise RuntimeError(f"rcm status {st}")
    return order


def permutation(n, part, p, iface):
    part, iface = _i32(part), _i32(iface)
    perm = np.empty(n, np.int32)
    iperm = np.empty(n, np.int32)
    int_ptr = np.empty(p + 1, np.int32)
    if_ptr = np.empty(p + 1, np.int32)
    n1 = lib().orc_permutation(n, _p(part), p, _p(iface), _p(perm), _p(iperm), _p(int_ptr),
                               _p(if_ptr))
    return perm, iperm, int_ptr, if_ptr, n1


# ---- the preconditioner ------------------------------------------------------------


@dataclass
class Sizes:
    n: int
    p: int
    n1: int
    n2: int
    nnz_coff: int
    npert: int
    nnz: int
    nlev_max: int


class Oracle:
    """Setup of the two-level preconditioner on (A, part); apply / inner GMRES / FGMRES."""

    def __init__(self, n, rowptr, colind, val, part, p, variant="schur", factor_B="ilu0",
                 factor_S="milu0", form="auto", ilut_tau=1e-3, ilut_p=10, inner_iters=3,
                 pivot_eps=1e-8, local_order="natural", fill_level=0, l1_block=False,
                 store_bf16=False):
        self._keep = [_i32(rowptr), _i32(colind), _f64(val), _i32(part)]
        o = _Opts()
        lib().orc_opts_default(C.byref(o))
        o.variant = _VAR[variant] if isinstance(variant, str) else int(variant)
        o.factor_B = _FACT[factor_B] if isinstance(factor_B, str) else int(factor_B)
        o.factor_S = _FACT[factor_S] if isinstance(factor_S, str) else int(factor_S)
        o.form = {"auto": FORM_AUTO, "wz": FORM_WZ, "ef": FORM_EF}[form]
        o.ilut_tau = ilut_tau
        o.ilut_p = int(ilut_p)
        o.inner_iters = int(inner_iters)
        o.pivot_eps = pivot_eps
        o.local_order = {"natural": ORDER_NATURAL, "rcm": ORDER_RCM, "color": ORDER_COLOR}[local_order]
        o.fill_level = int(fill_level)
        o.l1_block = int(bool(l1_block))
        o.store_bf16 = int(bool(store_bf16))
        self.opts = o
        st = C.c_int(0)
        rp, ci, v, pt = self._keep
        self.h = lib().orc_setup(int(n), _p(rp), _p(ci), _p(v), _p(pt), int(p), C.byref(o),
                                 C.byref(st))
        self.status = st.value
        if not self.h:
            raise RuntimeError(f"oracle setup failed with status {st.value}")
        self.n = int(n)
        self.p = int(p)

    @classmethod
    def from_problem(cls, prob, **kw):
        return cls(prob.n, prob.rowptr, prob.colind, prob.val, prob.part, prob.p, **kw)

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.orc_free(h)
            self.h = None

    def sizes(self) -> Sizes:
        out = np.empty(8, np.int32)
        lib().orc_sizes(self.h, _p(out))
        return Sizes(*[int(x) for x in out])

    def perm(self):
        s = self.sizes()
        perm = np.empty(s.n, np.int32)
        iperm = np.empty(s.n, np.int32)
        int_ptr = np.empty(s.p + 1, np.int32)
        if_ptr = np.empty(s.p + 1, np.int32)
        iface = np.empty(s.n, np.int32)
        lib().orc_get_perm(self.h, _p(perm), _p(iperm), _p(int_ptr), _p(if_ptr), _p(iface))
        return dict(perm=perm, iperm=iperm, int_ptr=int_ptr, if_ptr=if_ptr, iface=iface,
                    n1=s.n1, n2=s.n2)

    def levels(self, which: int):
        lev = np.empty(self.n, np.int32)
        nl = lib().orc_get_levels(self.h, int(which), _p(lev))
        return lev, nl

    def local_csr(self, s):
        nr = lib().orc_local_rows(self.h, s)
        nnz = lib().orc_local_nnz(self.h, s)
        rp = np.empty(nr + 1, np.int32)
        ci = np.empty(nnz, np.int32)
        v = np.empty(nnz)
        lib().orc_local_csr(self.h, s, _p(rp), _p(ci), _p(v))
        return rp, ci, v

    def local_factor(self, s, fact):
        nnz = lib().orc_local_nnz(self.h, s)
        v = np.empty(nnz)
        st = lib().orc_local_factor(self.h, s, int(fact), _p(v))
        if st != OK:
            raise ValueError("factor pattern differs from the local block")
        return v

    def coff(self):
        s = self.sizes()
        nnz = lib().orc_coff_nnz(self.h)
        rp = np.empty(s.n2 + 1, np.int32)
        ci = np.empty(nnz, np.int32)
        v = np.empty(nnz)
        lib().orc_coff_csr(self.h, _p(rp), _p(ci), _p(v))
        return rp, ci, v

    def schur_dense(self):
        n2 = self.sizes().n2
        S = np.empty((n2, n2))
        st = lib().orc_schur_dense(self.h, _p(S))
        if st != OK:
            raise RuntimeError(f"schur_dense status {st}")
        return S

    def sapprox_dense(self):
        n2 = self.sizes().n2
        S = np.empty((n2, n2))
        st = lib().orc_sapprox_dense(self.h, _p(S))
        if st != OK:
            raise RuntimeError(f"sapprox_dense status {st}")
        return S

    def apply(self, r):
        r = _f64(r)
        z = np.empty(self.n)
        st = lib().orc_apply(self.h, _p(r), _p(z))
        if st != OK:
            raise RuntimeError(f"apply status {st}")
        return z

    def inner_gmres(self, gp):
        gp = _f64(gp)
        y = np.empty(gp.size)
        lib().orc_inner_gmres(self.h, _p(gp), _p(y))
        return y

    def fgmres(self, b, x0=None, rtol=1e-8, restart=50, maxit=10000, hist_len=0):
        b = _f64(b)
        x = np.zeros(self.n) if x0 is None else _f64(x0).copy()
        iters = C.c_int(0)
        relres = C.c_double(0.0)
        hist = np.empty(max(hist_len, 1))
        used = C.c_int(0)
        st = lib().orc_fgmres(self.h, _p(b), _p(x), float(rtol), int(restart), int(maxit),
                              C.byref(iters), C.byref(relres), _p(hist), int(hist_len),
                              C.byref(used))
        return dict(x=x, status=st, iters=iters.value, relres=relres.value,
                    hist=hist[:used.value].copy())
