"""The ILUT(tau, p) numeric factorisation on the device (kernels_ilut.cu) against the oracle's
ILUT of the same local blocks (Sec. 4.2 runs ILUT for B; the dual-threshold rule as the oracle
states it), bit for bit: row pointers, columns and FP64 values.

Bit-exactness is the bar because nothing but a mistake can make the two differ: the kernel
eliminates the pivots of a row in ascending order, rounds each product and difference
separately, sums the row norm in CSR order and breaks ties of the p-largest selection by the
smaller column, as the sequential definition does.

Also: the device result equals the host factorisation's (ilut_setup="host"); a row wider than
the kernel's 512-slot table takes the large-table retry; p > 32 takes the host factorisation;
an exactly zero pivot with the perturbation off is reported as it is by the host; a bounded
wait that gives up returns ILU_ERR_TIMEOUT with the context still usable.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_2303_08881_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ilu():
    import __graft_entry__ as g
    g.build()
    import paper_2303_08881_gb300 as m
    assert torch.cuda.is_available()
    return m


PROBS = {
    "aniso2d_ragged": lambda: P.aniso2d_boxes(70, 3, seed=1),
    "conv3d": lambda: P.convdiff3d_boxes(14, 2, seed=2),
    "cuts3d": lambda: P.aniso3d_cuts(20, ncuts=(2, 2, 1), seed=3),
    "rand": lambda: P.randsparse(3000, 8, mean_k=4.0, seed=4),
    "dense_rows": lambda: P.randsparse(1500, 2, mean_k=24.0, seed=6),
    "p1": lambda: P.aniso2d_boxes(30, 1, seed=5),
}
_cache = {}


def _prob(name):
    if name not in _cache:
        _cache[name] = PROBS[name]()
    return _cache[name]


CFGS = [
    dict(variant="schur", ilut_tau=1e-3, ilut_p=10),
    dict(variant="schur", ilut_tau=1e-2, ilut_p=3),
    dict(variant="bj", ilut_tau=1e-3, ilut_p=5),
    dict(variant="schur", ilut_tau=0.0, ilut_p=32),      # every entry a candidate, 32 picks a part
    dict(variant="schur", ilut_tau=1e-3, ilut_p=0),      # the pivots only
    dict(variant="schur", ilut_tau=1e-4, ilut_p=20, local_order="rcm"),
    dict(variant="schur", ilut_tau=1e-3, ilut_p=10, local_order="color"),
    dict(variant="bj", ilut_tau=1e-1, ilut_p=1, local_order="rcm"),
]


def _cid(c):
    return "-".join(f"{k}={v}" for k, v in c.items())


def _opts(ilu, cfg, **kw):
    fs = "ilu0" if cfg["variant"] == "bj" else "milu0"
    return ilu.Opts(factor_B="ilut", factor_S=fs, pc_precision="fp64", **cfg, **kw)


def _oracle_blocks(pr, cfg, pivot_eps=1e-8):
    """The oracle's ILUT of each B_s (SCHUR: interior rows and columns of A_s in the local
    order) or A_s (block Jacobi)."""
    fs = "ilu0" if cfg["variant"] == "bj" else "milu0"
    orc = O.Oracle.from_problem(pr, factor_B="ilut", factor_S=fs, pivot_eps=pivot_eps, **cfg)
    pm = orc.perm()
    out = []
    for s in range(pr.p):
        rp, ci, v = orc.local_csr(s)
        m = len(rp) - 1 if cfg["variant"] == "bj" else int(pm["int_ptr"][s + 1] - pm["int_ptr"][s])
        nr = len(rp) - 1
        B = sp.csr_matrix((v, ci, rp), shape=(nr, nr))[:m, :m]
        B.sort_indices()
        out.append(O.ilut(m, B.indptr, B.indices, B.data, tau=cfg["ilut_tau"], p=cfg["ilut_p"],
                          pivot_eps=pivot_eps))
    return out


def _assert_blocks_equal(h, ref, what):
    for s, (rp_o, ci_o, v_o) in enumerate(ref):
        rp, ci, v = h.ilut_factor(s)
        assert np.array_equal(rp, rp_o), f"{what}: block {s} row pointers"
        assert np.array_equal(ci, ci_o), f"{what}: block {s} columns"
        assert np.array_equal(v, v_o), f"{what}: block {s} values, max diff {np.abs(v - v_o).max():.3e}"


@pytest.mark.parametrize("name", list(PROBS))
@pytest.mark.parametrize("cfg", CFGS, ids=_cid)
def test_device_ilut_matches_oracle(ilu, name, cfg):
    pr = _prob(name)
    h = ilu.ilu_setup_problem(pr, _opts(ilu, cfg))
    assert h.times()["ilut_on_device"]
    _assert_blocks_equal(h, _oracle_blocks(pr, cfg), f"{name} device")
    h.close()


@pytest.mark.parametrize("name", ["aniso2d_ragged", "cuts3d", "dense_rows"])
@pytest.mark.parametrize("cfg", [CFGS[0], CFGS[2], CFGS[3]], ids=_cid)
def test_device_ilut_matches_host_factorisation(ilu, name, cfg):
    """Device and host factorisations give the same factor, hence the same apply."""
    pr = _prob(name)
    hd = ilu.ilu_setup_problem(pr, _opts(ilu, cfg))
    hh = ilu.ilu_setup_problem(pr, _opts(ilu, cfg, ilut_setup="host"))
    assert hd.times()["ilut_on_device"] and not hh.times()["ilut_on_device"]
    assert hd.sizes()["npert"] == hh.sizes()["npert"]
    for s in range(pr.p):
        for a, b in zip(hd.ilut_factor(s), hh.ilut_factor(s)):
            assert np.array_equal(a, b), f"block {s}"
    r = torch.from_numpy(np.random.default_rng(7).standard_normal(pr.n)).cuda()
    zd, zh = torch.empty_like(r), torch.empty_like(r)
    ilu.ilu_apply(hd, r, zd)
    ilu.ilu_apply(hh, r, zh)
    torch.cuda.synchronize()
    assert torch.equal(zd, zh)
    hd.close()
    hh.close()


def _arrow_problem(width=700):
    """2D Poisson on 48 x 48, two boxes; one interior node of box 0 coupled (-1e-3, both ways)
    to `width` other interior nodes of box 0, their diagonals raised to keep dominance: the
    arrow row's working row holds more columns than the 512-slot table."""
    nx = 48
    n, rp, ci, v = P.poisson2d_5pt(nx, nx)
    part, p = P.box_partition((nx, nx), (2, 1))
    A = sp.csr_matrix((v, ci, rp), shape=(n, n))
    coo = A.tocoo()
    cross = part[coo.row] != part[coo.col]
    iface = np.zeros(n, bool)
    iface[coo.row[cross]] = True
    interior0 = np.flatnonzero((part == 0) & ~iface)
    a = int(interior0[3])
    others = interior0[interior0 != a][:width]
    assert len(others) == width
    E = sp.coo_matrix((np.full(width, -1e-3), (np.full(width, a), others)), shape=(n, n))
    D = sp.diags(np.where(np.isin(np.arange(n), others), 1e-3, 0.0)) + sp.diags(
        np.where(np.arange(n) == a, 1e-3 * width, 0.0))
    M = (A + E + E.T + D).tocsr()
    M.sort_indices()
    mat = (n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))
    return P._problem("arrow2d_48", mat, (part, p), seed=9)


@pytest.mark.parametrize("cfg", [dict(variant="schur", ilut_tau=1e-6, ilut_p=10),
                                 dict(variant="bj", ilut_tau=0.0, ilut_p=32)], ids=_cid)
def test_wide_row_takes_the_large_table(ilu, cfg):
    pr = _arrow_problem()
    h = ilu.ilu_setup_problem(pr, _opts(ilu, cfg))
    assert h.times()["ilut_on_device"]
    _assert_blocks_equal(h, _oracle_blocks(pr, cfg), "arrow")
    h.close()


def test_p_above_32_uses_the_host_factorisation(ilu):
    cfg = dict(variant="schur", ilut_tau=1e-4, ilut_p=40)
    pr = _prob("conv3d")
    h = ilu.ilu_setup_problem(pr, _opts(ilu, cfg))
    assert not h.times()["ilut_on_device"]
    _assert_blocks_equal(h, _oracle_blocks(pr, cfg), "host ilut")
    h.close()


def _zero_pivot_problem():
    """Tridiagonal 64 x 64 (2 on the diagonal, -0.5 off it) with rows 10 and 11 replaced by
    the block [[1, 1], [1, 1]] and no other coupling: ILUT's pivot of row 11 is 1 - 1 * 1 = 0
    exactly."""
    n = 64
    A = sp.diags([np.full(n - 1, -0.5), np.full(n, 2.0), np.full(n - 1, -0.5)], [-1, 0, 1]).tolil()
    for r in (10, 11):
        A[r, :] = 0.0
        A[:, r] = 0.0
    A[10, 10] = A[10, 11] = A[11, 10] = A[11, 11] = 1.0
    M = A.tocsr()
    M.eliminate_zeros()
    M.sort_indices()
    mat = (n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))
    return P._problem("zero_pivot_64", mat, P.contiguous_partition(n, 1), seed=3)


@pytest.mark.parametrize("where", ["device", "host"])
def test_zero_pivot_reported(ilu, where):
    pr = _zero_pivot_problem()
    cfg = dict(variant="bj", ilut_tau=1e-6, ilut_p=5)
    with pytest.raises(ilu.IluError) as ei:
        ilu.ilu_setup_problem(pr, _opts(ilu, cfg, pivot_eps=0.0, ilut_setup=where))
    assert ei.value.status == ilu.ILU_ERR_ZERO_PIVOT
    with pytest.raises(RuntimeError):
        _oracle_blocks(pr, cfg, pivot_eps=0.0)
    # with the perturbation on, the device factor is the oracle's, the pivot perturbed
    h = ilu.ilu_setup_problem(pr, _opts(ilu, cfg, ilut_setup=where))
    assert h.sizes()["npert"] >= 1
    _assert_blocks_equal(h, _oracle_blocks(pr, cfg), "perturbed")
    h.close()


def test_wait_that_gives_up_returns_timeout(ilu):
    """spin_limit = 1: a row whose pivot row is not finished at its first look gives up; the
    setup then fails with ILU_ERR_TIMEOUT (or, if every pivot row happened to be finished in
    time, succeeds with the oracle's factor), and the context stays usable."""
    pr = _prob("aniso2d_ragged")
    cfg = CFGS[0]
    try:
        h = ilu.ilu_setup_problem(pr, _opts(ilu, cfg, spin_limit=1))
    except ilu.IluError as e:
        assert e.status == ilu.ILU_ERR_TIMEOUT, e
    else:
        _assert_blocks_equal(h, _oracle_blocks(pr, cfg), "spin 1")
        h.close()
    h = ilu.ilu_setup_problem(pr, _opts(ilu, cfg))
    _assert_blocks_equal(h, _oracle_blocks(pr, cfg), "after timeout")
    h.close()
