"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded
inputs.

Bars (stated per check):
  * integer setup products (classification, permutation, level sets): bit-exact;
  * ILU(0) / MILU(0) factors computed on the device: bit-exact (the kernel keeps the
    sequential operation order and rounds every operation separately);
  * FP64 apply / SpMV / inner solve: normwise relative difference <= 1e-12 and every
    element within 1e-12 * ||z||_inf (different summation order and fused multiply-adds
    in the solves are the only differences);
  * FP32 preconditioner: normwise relative difference <= TOL32 = 2e-4 and every
    element within ELT32 * ||z||_inf, ELT32 = 1e-3 (see TOL32 and ELT32 below for the
    derivation);
  * FGMRES: FP64 preconditioner iteration count within +-1 of the oracle, FP32 within
    10 %; true relative residual <= rtol; solution within 1e-6 of the oracle's.
"""
import numpy as np
import pytest

import oracle as O
from paper_2303_08881_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP32 preconditioner tolerance: each level of a triangular solve adds O(u32 * growth)
# relative error (u32 = 6e-8); the deepest programs here have ~100 levels and the local
# factors of the anisotropic problems amplify by <~ 30, i.e. ~100 * 6e-8 * 30 = 2e-4.
TOL32 = 2e-4
# Element-wise FP32 bound, max_i |z_i - z_ref_i| <= ELT32 * ||z_ref||_inf: the forward error
# of a triangular solve is bounded component by component (|x - x^| <= gamma |T^-1||T||x|),
# so the same per-level argument bounds each element by ~levels * u32 * growth times the
# largest magnitude the element depends on. The apply passes through intermediate vectors
# (f', g', the inner Krylov vectors, y) whose largest entries exceed those of z by up to ~5 on
# these problems, hence 5 * TOL32. It catches a single wrong element that a norm could hide.
ELT32 = 1e-3


def _assert_close32(got, ref, what):
    rel = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
    elt = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
    assert rel <= TOL32, f"{what}: fp32 normwise {rel:.3e}"
    assert elt <= ELT32, f"{what}: fp32 max element {elt:.3e} of ||ref||_inf"


def _problems():
    return {
        "poisson64": lambda: P.make_workload("poisson2d_64_p4"),
        "aniso2d_ragged": lambda: P.aniso2d_boxes(70, 3, seed=1),
        "conv3d": lambda: P.convdiff3d_boxes(14, 2, seed=2),
        "cuts3d": lambda: P.aniso3d_cuts(20, ncuts=(2, 2, 1), seed=3),
        "rand": lambda: P.randsparse(3000, 8, mean_k=4.0, seed=4),
        "p1": lambda: P.aniso2d_boxes(30, 1, seed=5),
        # rows with up to ~40 local entries: exercises rows split over several sub-levels
        "dense_rows": lambda: P.randsparse(1500, 2, mean_k=24.0, seed=6),
    }


PROBS = _problems()
CONFIGS = [
    dict(variant="bj", factor_B="ilu0", factor_S="ilu0"),
    dict(variant="bj", factor_B="milu0", factor_S="milu0"),
    dict(variant="schur", factor_B="ilu0", factor_S="milu0"),
    dict(variant="schur", factor_B="ilu0", factor_S="ilu0"),
    dict(variant="schur", factor_B="milu0", factor_S="milu0"),
    dict(variant="schur", factor_B="ilu0", factor_S="milu0", form="ef"),
    dict(variant="schur", factor_B="ilut", factor_S="milu0", ilut_tau=1e-3, ilut_p=10),
    # RCM local order (Sec. 3.1): whole blocks for block Jacobi, each group for two-level
    dict(variant="bj", factor_B="ilu0", factor_S="ilu0", local_order="rcm"),
    dict(variant="schur", factor_B="ilu0", factor_S="milu0", local_order="rcm"),
    # ILU(k) / MILU(k): local blocks stored in their level-k fill pattern
    dict(variant="schur", factor_B="ilu0", factor_S="milu0", fill_level=2),
    dict(variant="bj", factor_B="milu0", factor_S="milu0", fill_level=1),
    # l1 block Jacobi (Sec. 4.3)
    dict(variant="bj", factor_B="ilu0", factor_S="ilu0", l1_block=True),
    # MILU(0) of the partial-ILU(0) Schur complement (Sec. 3.2)
    dict(variant="schur", factor_B="ilu0", factor_S="pmilu0"),
    # greedy multicolour local order (fewer levels, Sec. 3.1)
    dict(variant="schur", factor_B="ilu0", factor_S="milu0", local_order="color"),
    dict(variant="bj", factor_B="ilu0", factor_S="ilu0", local_order="color"),
]


def _cid(c):
    return "-".join(str(v) for v in c.values())


@pytest.fixture(scope="module")
def ilu():
    import __graft_entry__ as g
    g.build()
    import paper_2303_08881_gb300 as m
    assert torch.cuda.is_available()
    return m


_cache = {}


def _prob(name):
    if name not in _cache:
        _cache[name] = PROBS[name]()
    return _cache[name]


def _pair(ilu, name, cfg, prec, path="stream"):
    pr = _prob(name)
    kw = dict(cfg)
    opts = ilu.Opts(pc_precision=prec, kernel_path=path, **kw)
    h = ilu.ilu_setup_problem(pr, opts)
    okw = {k: v for k, v in kw.items()}
    orc = O.Oracle.from_problem(pr, **okw)
    return pr, h, orc


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _assert_close64(got, ref, what):
    scale = max(np.abs(ref).max(), 1e-300)
    rel = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
    assert rel <= 1e-12, f"{what}: normwise {rel:.3e}"
    assert np.abs(got - ref).max() <= 1e-12 * scale, f"{what}: max elt {np.abs(got - ref).max() / scale:.3e}"


# ---------------------------------------------------------------------------------------
# setup products


@pytest.mark.parametrize("name", list(PROBS))
@pytest.mark.parametrize("cfg", CONFIGS[:3] + CONFIGS[6:], ids=_cid)
def test_setup_structure_bit_exact(ilu, name, cfg):
    pr, h, orc = _pair(ilu, name, cfg, "fp64")
    pm = orc.perm()
    hp = h.perm()
    for k in ("perm", "iperm", "int_ptr", "if_ptr", "iface"):
        assert np.array_equal(hp[k], pm[k]), k
    s = h.sizes()
    os_ = orc.sizes()
    assert (s["n1"], s["n2"], s["nnz_coff"]) == (os_.n1, os_.n2, os_.nnz_coff)
    for w in range(6):
        lg, nlg = h.levels(w)
        lo, nlo = orc.levels(w)
        assert np.array_equal(lg, lo) and nlg == nlo, f"levels {w}"
    h.close()


@pytest.mark.parametrize("name", list(PROBS))
@pytest.mark.parametrize("cfg", [CONFIGS[0], CONFIGS[2], CONFIGS[4], CONFIGS[7], CONFIGS[8], CONFIGS[9],
                                 CONFIGS[10], CONFIGS[11], CONFIGS[12]], ids=_cid)
def test_device_factors_bit_exact(ilu, name, cfg):
    pr, h, orc = _pair(ilu, name, cfg, "fp64")
    facts = [1] if cfg["variant"] == "bj" or cfg["factor_B"] == cfg["factor_S"] else [1, 2]
    for s in range(pr.p):
        rp, _, _ = orc.local_csr(s)
        nnz = int(rp[-1])
        for f in facts:
            got = h.local_factor(s, f, nnz)
            ref = orc.local_factor(s, f)
            assert np.array_equal(got, ref), f"subdomain {s} factor {f}: max diff {np.abs(got - ref).max()}"
    assert h.sizes()["npert"] == orc.sizes().npert
    h.close()


# ---------------------------------------------------------------------------------------
# kernels


@pytest.mark.parametrize("name", list(PROBS))
def test_spmv_fp64(ilu, name):
    pr, h, orc = _pair(ilu, name, CONFIGS[0], "fp64")
    x = np.random.default_rng(7).standard_normal(pr.n)
    y = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    h.spmv(_dev(x), y)
    torch.cuda.synchronize()
    _assert_close64(y.cpu().numpy(), O.spmv(pr.n, pr.rowptr, pr.colind, pr.val, x), "spmv")
    h.close()


@pytest.mark.parametrize("name", list(PROBS))
@pytest.mark.parametrize("cfg", CONFIGS, ids=_cid)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("path", ["stream", "generic"])
def test_apply_matches_oracle(ilu, name, cfg, prec, path):
    pr, h, orc = _pair(ilu, name, cfg, prec, path)
    assert h.stats()["stream_path"] == (path == "stream")
    r = np.random.default_rng(11).standard_normal(pr.n)
    z = torch.full((pr.n,), np.nan, dtype=torch.float64, device="cuda")
    ilu.ilu_apply(h, _dev(r), z)
    torch.cuda.synchronize()
    got = z.cpu().numpy()
    ref = orc.apply(r)
    assert np.isfinite(got).all()
    if prec == "fp64":
        _assert_close64(got, ref, f"apply {name}")
    else:
        _assert_close32(got, ref, f"apply {name}")
    # a second call on the same handle gives the same bits (no state leaks between calls)
    z2 = torch.empty_like(z)
    ilu.ilu_apply(h, _dev(r), z2)
    torch.cuda.synchronize()
    assert torch.equal(z, z2)
    h.close()


@pytest.mark.parametrize("name", ["aniso2d_ragged", "conv3d", "rand", "cuts3d"])
@pytest.mark.parametrize("k", [1, 3, 7])
@pytest.mark.parametrize("path", ["stream", "generic"])
def test_inner_solve_fp64(ilu, name, k, path):
    cfg = dict(variant="schur", factor_B="ilu0", factor_S="milu0", inner_iters=k)
    pr, h, orc = _pair(ilu, name, cfg, "fp64", path)
    n2 = orc.sizes().n2
    g = np.random.default_rng(13).standard_normal(n2)
    y = torch.empty(n2, dtype=torch.float64, device="cuda")
    h.inner_solve(_dev(g), y)
    torch.cuda.synchronize()
    _assert_close64(y.cpu().numpy(), orc.inner_gmres(g), "inner")
    h.close()


@pytest.mark.parametrize("name", ["aniso2d_ragged", "conv3d", "cuts3d", "rand", "dense_rows"])
@pytest.mark.parametrize("cfg", [CONFIGS[2], CONFIGS[5], CONFIGS[6]], ids=_cid)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k", [1, 3, 7])
def test_inner_launch_modes_agree(ilu, name, cfg, prec, k):
    """The inner Schur GMRES as one cooperative launch (grid barriers between the
    Gram-Schmidt phases) and as four launches per step give the oracle's apply."""
    pr = _prob(name)
    orc = O.Oracle.from_problem(pr, inner_iters=k, **cfg)
    r = np.random.default_rng(17).standard_normal(pr.n)
    ref = orc.apply(r)
    got = {}
    for mode in ("single", "per_step"):
        h = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision=prec, inner_iters=k, inner_launch=mode, **cfg))
        st = h.stats()
        if orc.sizes().n2:
            assert st["inner_single_launch"] == (mode == "single")
        z = torch.full((pr.n,), np.nan, dtype=torch.float64, device="cuda")
        ilu.ilu_apply(h, _dev(r), z)
        ilu.ilu_apply(h, _dev(r), z)  # twice: the cooperative grid barrier state carries over
        torch.cuda.synchronize()
        assert h.stats()["device_error"] == 0
        got[mode] = z.cpu().numpy()
        h.close()
    for mode, z in got.items():
        if prec == "fp64":
            _assert_close64(z, ref, f"{mode} {name}")
        else:
            _assert_close32(z, ref, f"{mode} {name}")
    scale = np.linalg.norm(ref)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.linalg.norm(got["single"] - got["per_step"]) <= tol * scale


@pytest.mark.parametrize("side,prec", [(155, "fp64"), (215, "fp32"), (260, "fp32")])
def test_streamed_apply_with_global_working_vector(ilu, side, prec):
    """One subdomain too large for its working vector to sit in shared memory beside the
    ring: the streamed kernels keep it in the global scratch vector. 155^2 (FP64) and
    215^2 (FP32) lie where the generic kernels would still fit it in shared memory, so
    the scratch vector must be sized for the streamed kernels' own limit."""
    pr = P.aniso2d_boxes(side, 1, seed=21)
    cfg = dict(variant="schur", factor_B="ilu0", factor_S="milu0")
    h = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision=prec, **cfg))
    orc = O.Oracle.from_problem(pr, **cfg)
    st = h.stream_stats("fwd")
    assert h.stats()["stream_path"] and st["vector_in_shared"] == 0
    r = np.random.default_rng(12).standard_normal(pr.n)
    z = torch.full((pr.n,), np.nan, dtype=torch.float64, device="cuda")
    ilu.ilu_apply(h, _dev(r), z)
    torch.cuda.synchronize()
    got, ref = z.cpu().numpy(), orc.apply(r)
    assert h.stats()["device_error"] == 0
    if prec == "fp64":
        _assert_close64(got, ref, f"apply {side}")
    else:
        _assert_close32(got, ref, "apply")
    h.close()


@pytest.mark.parametrize("side,prec", [(300, "fp64"), (430, "fp32")])
@pytest.mark.parametrize("mode", ["single", "per_step"])
def test_global_working_vector_with_inner_solve(ilu, side, prec, mode):
    """2 x 2 subdomains each just too large for shared memory: the forward, inner and
    backward kernels all keep the working vector in global memory."""
    pr = P.aniso2d_boxes(side, 2, seed=22)
    cfg = dict(variant="schur", factor_B="ilu0", factor_S="milu0")
    h = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision=prec, inner_launch=mode, **cfg))
    orc = O.Oracle.from_problem(pr, **cfg)
    assert h.stream_stats("fwd")["vector_in_shared"] == 0 and orc.sizes().n2 > 0
    r = np.random.default_rng(23).standard_normal(pr.n)
    z = torch.full((pr.n,), np.nan, dtype=torch.float64, device="cuda")
    ilu.ilu_apply(h, _dev(r), z)
    torch.cuda.synchronize()
    got, ref = z.cpu().numpy(), orc.apply(r)
    assert h.stats()["device_error"] == 0
    if prec == "fp64":
        _assert_close64(got, ref, f"apply {side}")
    else:
        _assert_close32(got, ref, "apply")
    h.close()


def test_working_vector_in_shared_memory_for_the_2d_boxes(ilu):
    pr, h, orc = _pair(ilu, "aniso2d_ragged", CONFIGS[2], "fp32")
    assert h.stream_stats("fwd")["vector_in_shared"] == 1
    h.close()


RAP = dict(variant="rap", factor_B="ilu0", factor_S="milu0")


@pytest.mark.parametrize("name", ["aniso2d_ragged", "conv3d", "cuts3d", "rand", "p1", "dense_rows"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k", [1, 3])
@pytest.mark.parametrize("extra", [{}, {"local_order": "rcm"}, {"fill_level": 1}], ids=["natural", "rcm", "iluk1"])
def test_rap_apply_matches_oracle(ilu, name, prec, k, extra):
    """Multiplicative two-level apply (Algorithm "Multiplicative RAP-ILU on GPU"): ILU(0)
    smoother, R and P from MILU(0), k coarse GMRES steps preconditioned by L_S U_S."""
    pr = _prob(name)
    h = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision=prec, inner_iters=k, **extra, **RAP))
    orc = O.Oracle.from_problem(pr, inner_iters=k, **extra, **RAP)
    assert h.stats()["stream_path"]
    r = np.random.default_rng(19).standard_normal(pr.n)
    z = torch.full((pr.n,), np.nan, dtype=torch.float64, device="cuda")
    ilu.ilu_apply(h, _dev(r), z)
    torch.cuda.synchronize()
    got, ref = z.cpu().numpy(), orc.apply(r)
    assert np.isfinite(got).all() and h.stats()["device_error"] == 0
    if prec == "fp64":
        _assert_close64(got, ref, f"rap apply {name}")
    else:
        _assert_close32(got, ref, "apply")
    z2 = torch.empty_like(z)
    ilu.ilu_apply(h, _dev(r), z2)
    torch.cuda.synchronize()
    assert torch.equal(z, z2)
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rap_fgmres_matches_oracle(ilu, prec):
    pr = _prob("aniso2d_ragged")
    h = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision=prec, **RAP))
    orc = O.Oracle.from_problem(pr, **RAP)
    b = torch.from_numpy(pr.b).cuda()
    x = torch.zeros_like(b)
    info = ilu.gmres_solve(h, b, x, rtol=1e-8, restart=30, maxit=2000)
    ro = orc.fgmres(pr.b, rtol=1e-8, restart=30, maxit=2000)
    xo, it_o = ro["x"], ro["iters"]
    assert ro["status"] == 0
    assert info["status"] == 0 and info["rel_res_true"] <= 1e-8
    if prec == "fp64":
        assert abs(info["iters"] - it_o) <= 1
    else:
        assert abs(info["iters"] - it_o) <= max(2, it_o // 10)
    np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=0, atol=1e-6 * np.abs(xo).max())
    h.close()


@pytest.mark.parametrize("name", ["poisson64", "aniso2d_ragged", "conv3d", "cuts3d", "rand", "p1", "dense_rows"])
@pytest.mark.parametrize("variant", ["bj", "schur", "rap"])
def test_bf16_storage_apply_matches_oracle(ilu, name, variant):
    """bfloat16 factor values in the records, FP32 arithmetic: against the oracle whose
    off-diagonal factor entries are rounded to bfloat16 the same way, the only difference
    left is the FP32 arithmetic, so the FP32 bar applies."""
    pr = _prob(name)
    cfg = dict(variant=variant, factor_B="ilu0", factor_S="milu0")
    h = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision="bf16", **cfg))
    orc = O.Oracle.from_problem(pr, store_bf16=True, **cfg)
    assert h.stats()["stream_path"]
    r = np.random.default_rng(29).standard_normal(pr.n)
    z = torch.full((pr.n,), np.nan, dtype=torch.float64, device="cuda")
    ilu.ilu_apply(h, _dev(r), z)
    torch.cuda.synchronize()
    got, ref = z.cpu().numpy(), orc.apply(r)
    assert np.isfinite(got).all() and h.stats()["device_error"] == 0
    _assert_close32(got, ref, f"bf16 apply {name}")
    # and it is not the unrounded preconditioner
    ref32 = O.Oracle.from_problem(pr, **cfg).apply(r)
    assert np.linalg.norm(got - ref32) > np.linalg.norm(got - ref)
    h.close()


def test_bf16_storage_fgmres_matches_oracle(ilu):
    pr = _prob("aniso2d_ragged")
    cfg = dict(variant="schur", factor_B="ilu0", factor_S="milu0")
    h = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision="bf16", **cfg))
    ro = O.Oracle.from_problem(pr, store_bf16=True, **cfg).fgmres(pr.b, rtol=1e-8, restart=50, maxit=5000)
    b = _dev(pr.b)
    x = torch.zeros_like(b)
    info = ilu.gmres_solve(h, b, x, rtol=1e-8, restart=50, maxit=5000)
    assert ro["status"] == 0 and info["status"] == 0 and info["rel_res_true"] <= 1e-8
    assert abs(info["iters"] - ro["iters"]) <= max(2, ro["iters"] // 10), (info["iters"], ro["iters"])
    h.close()


def test_bf16_storage_refuses_what_it_does_not_cover(ilu):
    pr = _prob("poisson64")
    for kw in (dict(factor_B="ilut"), dict(form="ef"), dict(kernel_path="generic")):
        with pytest.raises(ilu.IluError):
            ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision="bf16", **kw))


def test_rap_needs_the_streamed_path(ilu):
    pr = _prob("aniso2d_ragged")
    with pytest.raises(ilu.IluError) as e:
        ilu.ilu_setup_problem(pr, ilu.Opts(kernel_path="generic", **RAP))
    assert e.value.status == ilu.ILU_ERR_UNSUPPORTED


def test_apply_of_zero_is_zero(ilu):
    pr, h, orc = _pair(ilu, "aniso2d_ragged", CONFIGS[2], "fp32")
    z = torch.full((pr.n,), 7.0, dtype=torch.float64, device="cuda")
    ilu.ilu_apply(h, torch.zeros(pr.n, dtype=torch.float64, device="cuda"), z)
    torch.cuda.synchronize()
    assert not z.any()
    h.close()


# ---------------------------------------------------------------------------------------
# edge cases


def _tiny_cases():
    # n = 1; all-interface subdomains (empty interiors); a subdomain with no rows
    one = (1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.5]),
           np.array([0], np.int32), 1)
    tri = P.tridiag(3, -1.0, 4.0, -1.0)
    three = (3, tri[1], tri[2], tri[3], np.array([0, 1, 2], np.int32), 3)
    pr = P.aniso2d_boxes(12, 2)
    gap = (pr.n, pr.rowptr, pr.colind, pr.val, np.where(pr.part == 3, 4, pr.part).astype(np.int32), 5)
    return {"n1": one, "all_interface": three, "empty_subdomain": gap}


@pytest.mark.parametrize("case", list(_tiny_cases()))
@pytest.mark.parametrize("cfg", [CONFIGS[0], CONFIGS[2], CONFIGS[6]], ids=_cid)
def test_edge_cases(ilu, case, cfg):
    n, rp, ci, v, part, p = _tiny_cases()[case]
    h = ilu.ilu_setup(n, rp, ci, v, part, p, ilu.Opts(pc_precision="fp64", **cfg))
    orc = O.Oracle(n, rp, ci, v, part, p, **cfg)
    r = np.random.default_rng(3).standard_normal(n)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    ilu.ilu_apply(h, _dev(r), z)
    torch.cuda.synchronize()
    _assert_close64(z.cpu().numpy(), orc.apply(r), case)
    b = _dev(r)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = ilu.gmres_solve(h, b, x, rtol=1e-10, restart=5, maxit=200)
    assert info["status"] == 0 and info["rel_res_true"] <= 1e-10
    h.close()


@pytest.mark.parametrize("threads", [64, 128])
def test_wide_consumer_groups(ilu, threads):
    """level programs run by 2 or 4 warps on a named barrier give the same result"""
    cfg = CONFIGS[2]
    pr = _prob("cuts3d")
    h = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision="fp64", block_threads=threads, **cfg))
    orc = O.Oracle.from_problem(pr, **cfg)
    r = np.random.default_rng(17).standard_normal(pr.n)
    z = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    ilu.ilu_apply(h, _dev(r), z)
    torch.cuda.synchronize()
    _assert_close64(z.cpu().numpy(), orc.apply(r), "wide group")
    h.close()


@pytest.mark.parametrize("name,cfg", [("aniso2d_ragged", CONFIGS[2]), ("cuts3d", CONFIGS[6]), ("poisson64", CONFIGS[0])])
def test_autotune_measures_and_remembers(ilu, name, cfg):
    """ilu_opts.autotune: the setup times each streamed program with the candidate consumer
    groups and keeps the fastest; the apply still matches the oracle; a second setup of the
    same structure takes the remembered choice without measuring and gives the same bits."""
    pr = _prob(name)
    h = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision="fp32", autotune=True, **cfg))
    t = h.tuning()
    assert t["state"] in ("measured", "remembered")
    for prog, nt in t["threads"].items():
        assert nt in (32, 64, 96, 128)
        if t["state"] == "measured":
            assert len(t["apply_ms"][prog]) >= 2 and nt in t["apply_ms"][prog]
    r = np.random.default_rng(31).standard_normal(pr.n)
    z = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    ilu.ilu_apply(h, _dev(r), z)
    h2 = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision="fp32", autotune=True, **cfg))
    t2 = h2.tuning()
    assert t2["state"] == "remembered" and t2["threads"] == t["threads"]
    z2 = torch.empty_like(z)
    ilu.ilu_apply(h2, _dev(r), z2)
    torch.cuda.synchronize()
    _assert_close32(z.cpu().numpy(), O.Oracle.from_problem(pr, **cfg).apply(r), f"autotuned {name}")
    assert torch.equal(z, z2)
    h.close()
    h2.close()


def test_device_wait_timeout_is_reported(ilu):
    """A bound of one poll on every mbarrier wait makes the streamed apply give up; the
    device error word reports it, the call returns, and the context stays usable."""
    pr = _prob("aniso2d_ragged")
    h = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision="fp32", spin_limit=1, **CONFIGS[2]))
    r = torch.randn(pr.n, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    for _ in range(3):
        ilu.ilu_apply(h, r, z)
    st = h.stats()
    assert st["stream_path"] and st["device_error"] in (0, 2)
    if st["inner_single_launch"]:  # its grid barriers cannot pass with a single poll
        assert st["device_error"] == 2
    x = torch.zeros_like(r)
    try:
        info = ilu.gmres_solve(h, r, x, rtol=1e-8, restart=10, maxit=50)
        assert info["status"] in (0, ilu.ILU_ERR_NOT_CONVERGED)
    except ilu.IluError as e:
        assert e.status == ilu.ILU_ERR_TIMEOUT
    h.close()
    # a fresh handle on the same device still works
    pr2, h2, orc = _pair(ilu, "poisson64", CONFIGS[0], "fp64")
    rr = np.random.default_rng(1).standard_normal(pr2.n)
    zz = torch.empty(pr2.n, dtype=torch.float64, device="cuda")
    ilu.ilu_apply(h2, _dev(rr), zz)
    torch.cuda.synchronize()
    _assert_close64(zz.cpu().numpy(), orc.apply(rr), "after timeout")
    assert h2.stats()["device_error"] == 0
    h2.close()


@pytest.mark.parametrize("path", ["stream", "generic"])
def test_handles_with_different_subdomain_sizes_coexist(ilu, path):
    """the per-kernel shared-memory limit is process-wide state: a handle created later
    with smaller subdomains must not break an earlier handle's launches"""
    big, h_big, orc = _pair(ilu, "p1", CONFIGS[2], "fp64", path)   # one 900-row subdomain
    small = ilu.ilu_setup_problem(_prob("poisson64"), ilu.Opts(pc_precision="fp64", kernel_path=path))
    r = np.random.default_rng(23).standard_normal(big.n)
    z = torch.empty(big.n, dtype=torch.float64, device="cuda")
    ilu.ilu_apply(h_big, _dev(r), z)
    torch.cuda.synchronize()
    _assert_close64(z.cpu().numpy(), orc.apply(r), "big after small")
    small.close()
    h_big.close()


def test_bad_vectors_are_rejected(ilu):
    pr, h, _ = _pair(ilu, "poisson64", CONFIGS[0], "fp64")
    r = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    with pytest.raises(ilu.IluError) as e:
        ilu.ilu_apply(h, r, r)
    assert e.value.status == ilu.ILU_ERR_ARG
    # the binding refuses vectors the kernels would read or write out of bounds
    with pytest.raises(ValueError):
        ilu.ilu_apply(h, r[:-1], torch.zeros(pr.n - 1, dtype=torch.float64, device="cuda"))
    with pytest.raises(TypeError):
        ilu.ilu_apply(h, r.float(), torch.zeros(pr.n, dtype=torch.float32, device="cuda"))
    h.close()
    pr2, h2, orc2 = _pair(ilu, "aniso2d_ragged", CONFIGS[2], "fp64")
    n2 = orc2.sizes().n2
    short = torch.zeros(n2 - 1, dtype=torch.float64, device="cuda")
    for f in (h2.inner_solve, h2.inner_solve_noalloc):
        with pytest.raises(ValueError):
            f(short, torch.zeros(n2, dtype=torch.float64, device="cuda"))
    h2.close()


# ---------------------------------------------------------------------------------------
# FGMRES


@pytest.mark.parametrize("name,cfg,prec,restart", [
    ("poisson64", CONFIGS[0], "fp64", 30),
    ("poisson64", CONFIGS[2], "fp64", 30),
    ("aniso2d_ragged", CONFIGS[2], "fp64", 50),
    ("aniso2d_ragged", CONFIGS[2], "fp32", 50),
    ("conv3d", CONFIGS[2], "fp32", 50),
    ("cuts3d", CONFIGS[6], "fp32", 50),
    ("rand", CONFIGS[2], "fp32", 20),
    ("conv3d", CONFIGS[5], "fp64", 10),
    ("aniso2d_ragged", CONFIGS[7], "fp64", 50),
    ("conv3d", CONFIGS[8], "fp32", 50),
    ("conv3d", CONFIGS[9], "fp64", 30),
    ("aniso2d_ragged", CONFIGS[9], "fp32", 50),
    # restarts the paper uses beyond 64 (FGMRES(100), Sec. 4.2-4.4) and the limit 256
    ("aniso2d_ragged", CONFIGS[0], "fp64", 100),
    ("poisson64", CONFIGS[0], "fp64", 256),
    ("cuts3d", CONFIGS[11], "fp32", 50),
    ("aniso2d_ragged", CONFIGS[12], "fp64", 50),
])
@pytest.mark.parametrize("graphs", [True, False])
def test_fgmres_matches_oracle(ilu, name, cfg, prec, restart, graphs):
    pr = _prob(name)
    h = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision=prec, use_graphs=graphs, **cfg))
    orc = O.Oracle.from_problem(pr, **cfg)
    ref = orc.fgmres(pr.b, rtol=1e-8, restart=restart, maxit=5000)
    b = _dev(pr.b)
    x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    info = ilu.gmres_solve(h, b, x, rtol=1e-8, restart=restart, maxit=5000)
    torch.cuda.synchronize()
    assert info["status"] == 0
    xs = x.cpu().numpy()
    res = np.linalg.norm(pr.b - pr.scipy() @ xs) / np.linalg.norm(pr.b)
    assert res <= 1e-8 * 1.0001 and abs(res - info["rel_res_true"]) <= 1e-10
    if prec == "fp64":
        assert abs(info["iters"] - ref["iters"]) <= 1, (info["iters"], ref["iters"])
    else:
        assert abs(info["iters"] - ref["iters"]) <= max(1, 0.1 * ref["iters"]), (info["iters"], ref["iters"])
    assert np.linalg.norm(xs - ref["x"]) <= 1e-6 * np.linalg.norm(ref["x"])
    # solving again from the solution converges immediately; b = 0 gives x = 0
    info2 = ilu.gmres_solve(h, b, x, rtol=1e-8, restart=restart, maxit=5000)
    assert info2["iters"] == 0
    x.fill_(3.0)
    info3 = ilu.gmres_solve(h, torch.zeros_like(b), x, rtol=1e-8, restart=restart)
    assert info3["status"] == 0 and not x.any()
    h.close()


@pytest.mark.parametrize("name", ["aniso2d_ragged", "conv3d", "cuts3d", "rand"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gs_mixed_precision_keeps_fp64_fgmres(ilu, name, prec):
    """The first Gram-Schmidt pass's coefficients from FP32 copies of V and w (corrected by the
    FP64 second pass), and the second pass's small update from the FP32 copy of V: the same
    iteration count as both passes in FP64 (+-1), the same solution within 1e-6, and with the
    FP64 preconditioner the oracle's count within +-1."""
    pr = _prob(name)
    cfg = CONFIGS[2]
    b = _dev(pr.b)
    out = {}
    for mode in ("mixed3", "mixed2", "mixed1", "fp64"):
        h = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision=prec, gs_precision=mode, **cfg))
        x = torch.zeros_like(b)
        info = ilu.gmres_solve(h, b, x, rtol=1e-8, restart=30, maxit=3000)
        assert info["status"] == 0 and info["rel_res_true"] <= 1e-8, info
        out[mode] = (info["iters"], x.cpu().numpy())
        h.close()
    i64, x64 = out["fp64"]
    for mode in ("mixed1", "mixed2", "mixed3"):
        i32, x32 = out[mode]
        assert abs(i32 - i64) <= 1, (mode, i32, i64)
        assert np.linalg.norm(x32 - x64) <= 1e-6 * np.linalg.norm(x64), mode
    if prec == "fp64":
        ref = O.Oracle.from_problem(pr, **cfg).fgmres(pr.b, rtol=1e-8, restart=30, maxit=3000)
        for mode in out:
            assert abs(out[mode][0] - ref["iters"]) <= 1, (mode, out[mode][0], ref["iters"])


@pytest.mark.parametrize("name", ["aniso2d_ragged", "conv3d"])
def test_gs_mixed_precision_keeps_the_basis_orthonormal(ilu, name):
    """One FGMRES(40) cycle (FP32 preconditioner), then the basis v_1..v_39 from the device (the
    end of a cycle leaves the new true residual in v_0): the loss of orthogonality
    max |V V^T - I| of the mixed-precision Gram-Schmidt forms stays at the level of the
    all-FP64 form (FP64 rounding, well below 1e-12)."""
    pr = _prob(name)
    b = _dev(pr.b)
    m = 40
    loss = {}
    for mode in ("fp64", "mixed1", "mixed2", "mixed3"):
        h = ilu.ilu_setup_problem(pr, ilu.Opts(gs_precision=mode, **CONFIGS[2]))
        x = torch.zeros_like(b)
        info = ilu.gmres_solve(h, b, x, rtol=1e-30, restart=m, maxit=m)
        assert info["iters"] == m
        V = h.krylov("V", m)[1:]
        loss[mode] = np.abs(V @ V.T - np.eye(m - 1)).max()
        h.close()
    assert loss["fp64"] < 1e-13, loss
    for mode in ("mixed1", "mixed2", "mixed3"):
        assert loss[mode] <= max(10 * loss["fp64"], 1e-14) and loss[mode] < 1e-12, loss


@pytest.mark.parametrize("restart", [50, 256])
def test_gs_double_float_pass_on_full_row_slices(ilu, restart):
    """The double-float second pass (mixed3) on a 512^2 grid, where every CTA's row slice holds
    whole 256-row sub-slices and a ragged rest (the small problems above take only the ragged
    path), and at the largest restart (the most shared-memory accumulators): the solve takes
    the FP64 form's iteration count +-1 and reaches the same solution within 1e-6, and after
    one FGMRES(40) cycle the basis is as orthonormal as the FP64 one."""
    pr = P.aniso2d_boxes(512, 4, seed=7)
    b = _dev(pr.b)
    res = {}
    for mode in ("fp64", "mixed3"):
        h = ilu.ilu_setup_problem(pr, ilu.Opts(gs_precision=mode, **CONFIGS[2]))
        x = torch.zeros_like(b)
        info = ilu.gmres_solve(h, b, x, rtol=1e-8, restart=restart, maxit=4000)
        assert info["status"] == 0 and info["rel_res_true"] <= 1e-8, (mode, info)
        x1 = torch.zeros_like(b)
        ilu.gmres_solve(h, b, x1, rtol=1e-30, restart=40, maxit=40)
        V = h.krylov("V", 40)[1:]
        res[mode] = (info["iters"], x.cpu().numpy(), np.abs(V @ V.T - np.eye(39)).max())
        h.close()
    (i64, x64, l64), (idf, xdf, ldf) = res["fp64"], res["mixed3"]
    assert abs(idf - i64) <= 1, (idf, i64)
    assert np.linalg.norm(xdf - x64) <= 1e-6 * np.linalg.norm(x64)
    assert ldf <= max(10 * l64, 1e-14) and ldf < 1e-12, (ldf, l64)


def test_restart_limit(ilu):
    pr = _prob("poisson64")
    h = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision="fp64", **CONFIGS[0]))
    b = _dev(pr.b)
    x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    with pytest.raises(ilu.IluError):
        ilu.gmres_solve(h, b, x, rtol=1e-8, restart=257, maxit=100)
    info = ilu.gmres_solve(h, b, x, rtol=1e-8, restart=256, maxit=5000)
    assert info["status"] == 0 and info["rel_res_true"] <= 1e-8
    h.close()


def test_fgmres_maxit_reports_not_converged(ilu):
    pr = _prob("aniso2d_ragged")
    h = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision="fp64", **CONFIGS[2]))
    x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    info = ilu.gmres_solve(h, _dev(pr.b), x, rtol=1e-12, restart=5, maxit=7)
    assert info["status"] == ilu.ILU_ERR_NOT_CONVERGED and info["iters"] == 7
    orc = O.Oracle.from_problem(pr, **CONFIGS[2])
    ref = orc.fgmres(pr.b, rtol=1e-12, restart=5, maxit=7)
    assert ref["iters"] == 7
    np.testing.assert_allclose(info["rel_res_true"], ref["relres"], rtol=1e-8)
    h.close()
