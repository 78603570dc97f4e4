"""The library's host-side setup (analysis-only handles, no GPU): interior/interface
classification, interior-first permutation, level sets of every factor pattern (ILUT's
included) match the oracle bit for bit."""
import numpy as np
import scipy.sparse as sp
import pytest

import oracle as O
from paper_2303_08881_gb300 import problems as P

CASES = {
    "poisson64": lambda: P.make_workload("poisson2d_64_p4"),
    "aniso2d_ragged": lambda: P.aniso2d_boxes(70, 3, seed=1),
    "conv3d": lambda: P.convdiff3d_boxes(14, 2, seed=2),
    "cuts3d": lambda: P.aniso3d_cuts(20, ncuts=(2, 2, 1), seed=3),
    "rand": lambda: P.randsparse(3000, 8, mean_k=4.0, seed=4),
    "p1": lambda: P.aniso2d_boxes(30, 1, seed=5),
    "dense_rows": lambda: P.randsparse(1500, 2, mean_k=24.0, seed=6),
}
CFGS = [
    dict(variant="bj", factor_B="ilu0", factor_S="ilu0"),
    dict(variant="schur", factor_B="ilu0", factor_S="milu0"),
    dict(variant="schur", factor_B="ilut", factor_S="milu0", ilut_tau=1e-3, ilut_p=10),
    dict(variant="schur", factor_B="ilut", factor_S="milu0", ilut_tau=1e-2, ilut_p=3),
    dict(variant="bj", factor_B="ilut", factor_S="ilu0", ilut_tau=1e-3, ilut_p=5),
    dict(variant="rap", factor_B="ilu0", factor_S="milu0"),
    dict(variant="bj", factor_B="ilu0", factor_S="ilu0", local_order="rcm"),
    dict(variant="schur", factor_B="ilu0", factor_S="milu0", local_order="rcm"),
    dict(variant="schur", factor_B="ilut", factor_S="milu0", ilut_tau=1e-3, ilut_p=10, local_order="rcm"),
    dict(variant="rap", factor_B="ilu0", factor_S="milu0", local_order="rcm"),
    dict(variant="bj", factor_B="ilu0", factor_S="ilu0", fill_level=1),
    dict(variant="schur", factor_B="ilu0", factor_S="milu0", fill_level=2),
    dict(variant="rap", factor_B="ilu0", factor_S="milu0", fill_level=1, local_order="rcm"),
    dict(variant="bj", factor_B="ilu0", factor_S="ilu0", l1_block=True, local_order="rcm"),
    dict(variant="bj", factor_B="ilu0", factor_S="ilu0", local_order="color"),
    dict(variant="schur", factor_B="ilu0", factor_S="milu0", local_order="color"),
    dict(variant="schur", factor_B="ilut", factor_S="milu0", ilut_tau=1e-3, ilut_p=10, local_order="color"),
    dict(variant="schur", factor_B="ilu0", factor_S="pmilu0"),
]


@pytest.fixture(scope="module")
def ilu():
    import __graft_entry__ as g
    g.build()
    import paper_2303_08881_gb300 as m
    return m


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("cfg", CFGS, ids=lambda c: "-".join(map(str, c.values())))
def test_host_analysis_matches_oracle(ilu, name, cfg):
    pr = CASES[name]()
    h = ilu.ilu_setup_problem(pr, ilu.Opts(analysis_only=True, **cfg))
    orc = O.Oracle.from_problem(pr, **cfg)
    pm, hp = orc.perm(), h.perm()
    for k in ("perm", "iperm", "int_ptr", "if_ptr", "iface"):
        assert np.array_equal(hp[k], pm[k]), k
    s, so = h.sizes(), orc.sizes()
    assert (s["n1"], s["n2"], s["nnz_coff"], s["nnz"]) == (so.n1, so.n2, so.nnz_coff, so.nnz)
    # an analysis-only handle counts the perturbed pivots of the host ILUT only; the oracle
    # counts those of every factorisation (with the colour order MILU(0) of A_i has many)
    if cfg.get("local_order") == "color":
        assert s["npert"] <= so.npert
    else:
        assert s["npert"] == (so.npert if cfg["factor_B"] == "ilut" else 0)
    for w in range(6):
        lg, nlg = h.levels(w)
        lo, nlo = orc.levels(w)
        assert np.array_equal(lg, lo) and nlg == nlo, f"levels {w}"
    for sd in range(pr.p):  # the stored local blocks (the level-k fill pattern if any)
        rp, ci = h.local_pattern(sd)
        orp, oci, _ = orc.local_csr(sd)
        assert np.array_equal(rp, orp) and np.array_equal(ci, oci), f"pattern of block {sd}"
    h.close()


def test_fill_level_option_is_validated(ilu):
    pr = CASES["poisson64"]()
    with pytest.raises(ilu.IluError):
        ilu.ilu_setup_problem(pr, ilu.Opts(analysis_only=True, factor_B="ilut", fill_level=1))
    with pytest.raises(ilu.IluError):
        ilu.ilu_setup_problem(pr, ilu.Opts(analysis_only=True, fill_level=-1))
    with pytest.raises(ilu.IluError):
        ilu.ilu_setup_problem(pr, ilu.Opts(analysis_only=True, variant="schur", l1_block=True))


def test_full_size_2d_workload_structure(ilu):
    """1024^2 9-point anisotropic problem on 8x8 boxes: the counts of the interior /
    interface split and the level depth of L_B (natural order: level x + 2y; the corner
    boxes have a 127 x 127 interior, so 126 + 2*126 + 1 levels)."""
    pr = P.make_workload("aniso2d_1024_p64")
    h = ilu.ilu_setup_problem(pr, ilu.Opts(analysis_only=True))
    s = h.sizes()
    assert (s["n"], s["nnz"], s["n1"], s["n2"], s["nnz_coff"]) == (
        1048576, 9424900, 1020100, 28476, 85764)
    assert s["nlev_LB"] == 3 * 126 + 1
    h.close()


def test_analysis_handle_refuses_device_calls(ilu):
    pr = P.make_workload("poisson2d_64_p4")
    h = ilu.ilu_setup_problem(pr, ilu.Opts(analysis_only=True))
    import ctypes as C
    assert ilu.lib().ilu_apply(h.ptr, C.c_void_p(16), C.c_void_p(32)) == ilu.ILU_ERR_ARG
    h.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("cfg", CFGS[:3], ids=lambda c: "-".join(map(str, c.values())))
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_streamed_programs_are_built(ilu, name, cfg, prec):
    """every test workload keeps the TMA-streamed level programs (no silent fallback)"""
    pr = CASES[name]()
    h = ilu.ilu_setup_problem(pr, ilu.Opts(analysis_only=True, pc_precision=prec, **cfg))
    assert h.stats()["stream_path"]
    h.close()


def _analysis_digest(h):
    import hashlib
    m = hashlib.sha256()
    for k, v in sorted(h.perm().items()):
        m.update(np.ascontiguousarray(v).tobytes())
    for prog in ("bj", "fwd", "s", "bwd"):
        try:
            st = h.stream(prog)
        except Exception:
            continue
        m.update(st["blob"].tobytes())
        m.update(st["ch0"].tobytes())
    for sd in range(h.sizes()["p"]):
        rp, ci = h.local_pattern(sd)
        m.update(rp.tobytes())
        m.update(ci.tobytes())
    return m.hexdigest()


@pytest.mark.parametrize("cfg", [dict(variant="schur"), dict(variant="rap", local_order="rcm", fill_level=1)],
                         ids=["schur", "rap-rcm-iluk"])
def test_concurrent_setups_build_the_same_analysis(ilu, cfg):
    """The host analysis runs its per-subdomain phases on worker threads and divides the
    threads among setups running at the same time; the result must not depend on the split:
    four concurrent setups give byte-identical orders, patterns and streams to a lone one."""
    import threading
    pr = CASES["aniso2d_ragged"]()
    h = ilu.ilu_setup_problem(pr, ilu.Opts(analysis_only=True, **cfg))
    ref = _analysis_digest(h)
    h.close()
    got, errs = [], []

    def one():
        try:
            hh = ilu.ilu_setup_problem(pr, ilu.Opts(analysis_only=True, **cfg))
            got.append(_analysis_digest(hh))
            hh.close()
        except Exception as e:  # reported below
            errs.append(repr(e))

    ts = [threading.Thread(target=one) for _ in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(120)
    assert not errs and got == [ref] * 4


@pytest.mark.parametrize("opts,ok", [
    (dict(variant="bj", factor_S="pmilu0"), False),            # PMILU0 is an S factor of SCHUR
    (dict(variant="rap", factor_S="pmilu0"), False),
    (dict(variant="schur", factor_B="pmilu0"), False),
    (dict(variant="schur", factor_S="ilut"), False),           # ILUT only for the B factor
    (dict(variant="rap", factor_B="ilut"), False),
    (dict(variant="schur", l1_block=True), False),             # l1 augmentation: block Jacobi only
    (dict(variant="schur", factor_B="ilut", fill_level=1), False),
    (dict(variant="schur", factor_S="pmilu0", fill_level=1), True),
    (dict(variant="schur", factor_S="pmilu0", local_order="rcm"), True),
    (dict(variant="bj", l1_block=True, fill_level=2, local_order="rcm"), True),
    (dict(variant="rap", fill_level=1, pc_precision="bf16"), True),
    (dict(variant="schur", factor_B="ilut", pc_precision="bf16"), False),
    (dict(variant="schur", form="ef", pc_precision="bf16"), False),
    (dict(variant="schur", kernel_path="generic", pc_precision="bf16"), False),
    (dict(variant="rap", kernel_path="generic"), False),
], ids=lambda v: str(v) if isinstance(v, bool) else "-".join(f"{k}={x}" for k, x in v.items()))
def test_option_combinations(ilu, opts, ok):
    pr = CASES["aniso2d_ragged"]()
    if ok:
        h = ilu.ilu_setup_problem(pr, ilu.Opts(analysis_only=True, **opts))
        assert h.sizes()["n"] == pr.n
        h.close()
    else:
        with pytest.raises(ilu.IluError):
            ilu.ilu_setup_problem(pr, ilu.Opts(analysis_only=True, **opts))


def _corrupt(kind, r, n, rp, ci, part, p):
    rp, ci, part = rp.copy(), ci.copy(), part.copy()
    b, e = int(rp[r]), int(rp[r + 1])
    if kind == "unsorted":
        ci[b], ci[b + 1] = ci[b + 1], ci[b]
    elif kind == "duplicate":
        ci[b + 1] = ci[b]
    elif kind == "out_of_range":
        ci[e - 1] = n
    elif kind == "negative":
        ci[b] = -1
    elif kind == "no_diagonal":
        d = b + int(np.nonzero(ci[b:e] == r)[0][0])
        ci = np.delete(ci, d)
        rp[r + 1:] -= 1
    elif kind == "part":
        part[r] = p
    elif kind == "row_and_part":
        ci[b], ci[b + 1] = ci[b + 1], ci[b]
        part[(r + n // 3) % n] = -1
    return rp, ci, part


@pytest.mark.parametrize("where", ["first", "middle", "last"])
@pytest.mark.parametrize("kind,status", [("unsorted", "ILU_ERR_CSR"), ("duplicate", "ILU_ERR_CSR"),
                                         ("out_of_range", "ILU_ERR_CSR"), ("negative", "ILU_ERR_CSR"),
                                         ("no_diagonal", "ILU_ERR_CSR"), ("part", "ILU_ERR_ARG"),
                                         ("row_and_part", "ILU_ERR_CSR")])
def test_input_checks_find_every_bad_row(ilu, kind, status, where):
    """The input checks run on host threads over row ranges: a bad row or partition entry
    anywhere gives the same status a sequential scan would (a bad row wins over a bad
    partition entry)."""
    pr = P.poisson2d_boxes(40, 2)
    n = pr.n
    r = {"first": 0, "middle": n // 2, "last": n - 1}[where]
    rp, ci, part = _corrupt(kind, r, n, pr.rowptr, pr.colind, pr.part, pr.p)
    val = np.ones(ci.size)
    with pytest.raises(ilu.IluError) as ei:
        ilu.ilu_setup(n, rp, ci, val, part, pr.p, ilu.Opts(analysis_only=True))
    assert ei.value.status == getattr(ilu, status)


@pytest.mark.parametrize("name", ["aniso2d_ragged", "cuts3d", "dense_rows"])
@pytest.mark.parametrize("cfg", [dict(variant="schur", factor_S="milu0", ilut_tau=1e-3, ilut_p=10),
                                 dict(variant="bj", factor_S="ilu0", ilut_tau=0.0, ilut_p=32),
                                 dict(variant="schur", factor_S="milu0", ilut_tau=1e-3, ilut_p=0)],
                         ids=lambda c: "-".join(map(str, c.values())))
def test_host_ilut_factor_matches_oracle(ilu, name, cfg):
    """The host ILUT of each B_s (A_s for block Jacobi), read through ilu_get_ilut_factor,
    equals the oracle's ILUT of the same block bit for bit; analysis-only handles factorise
    on the host."""
    pr = CASES[name]()
    h = ilu.ilu_setup_problem(pr, ilu.Opts(analysis_only=True, factor_B="ilut", **cfg))
    t = h.times()
    assert not t["ilut_on_device"] and t["ilut_ms"] > 0.0
    orc = O.Oracle.from_problem(pr, factor_B="ilut", **cfg)
    pm = orc.perm()
    for s in range(pr.p):
        rp, ci, v = orc.local_csr(s)
        nr = len(rp) - 1
        m = nr if cfg["variant"] == "bj" else int(pm["int_ptr"][s + 1] - pm["int_ptr"][s])
        B = sp.csr_matrix((v, ci, rp), shape=(nr, nr))[:m, :m]
        B.sort_indices()
        ref = O.ilut(m, B.indptr, B.indices, B.data, tau=cfg["ilut_tau"], p=cfg["ilut_p"])
        for a, b in zip(h.ilut_factor(s), ref):
            assert np.array_equal(a, b), f"block {s}"
    h.close()


def test_ilut_factor_needs_ilut(ilu):
    pr = CASES["p1"]()
    h = ilu.ilu_setup_problem(pr, ilu.Opts(analysis_only=True))
    with pytest.raises(ilu.IluError) as ei:
        h.ilut_factor(0)
    assert ei.value.status == ilu.ILU_ERR_ARG
    assert h.times()["ilut_ms"] == 0.0
    h.close()
