"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: values printed in the
paper (tests/golden), textbook identities (exact LU, Schur complement = inverse of the
(2,2) block of A^{-1}), library routines (scipy LU / triangular solves / dense solves),
structural properties stated in the paper, or brute force on tiny inputs.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from paper_2303_08881_gb300 import problems as P

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _csr(mat):
    n, rp, ci, v = mat
    return sp.csr_matrix((v, ci, rp), shape=(n, n))


def _rand_sparse(n, dens, seed, sym_pattern=False, dd=2.0):
    """small random sparse matrix with a stored, dominant diagonal"""
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=dens, random_state=rng, format="csr")
    M.data = rng.standard_normal(M.data.size)
    if sym_pattern:
        M = M + sp.csr_matrix((np.zeros(M.nnz), M.indices, M.indptr), shape=M.shape).T
    M = M.tolil()
    M.setdiag(0.0)
    M = M.tocsr()
    M.eliminate_zeros()
    d = dd * (np.abs(M).sum(axis=1).A.ravel() + 1.0)
    M = (M + sp.diags(d)).tocsr()
    M.sort_indices()
    return M


def _mat_tuple(M):
    M = sp.csr_matrix(M)
    M.sort_indices()
    return (M.shape[0], M.indptr.astype(np.int32), M.indices.astype(np.int32),
            M.data.astype(np.float64))


def _split_lu(n, rp, ci, f):
    F = sp.csr_matrix((f, ci, rp), shape=(n, n))
    L = sp.tril(F, -1) + sp.identity(n)
    U = sp.triu(F)
    return L.tocsr(), U.tocsr()


# --------------------------------------------------------------------------------------
# CSR validation


def test_csr_check_rejects_malformed():
    rp = np.array([0, 2, 4], np.int32)
    assert O.csr_check(2, rp, np.array([0, 1, 0, 1], np.int32)) == O.OK
    assert O.csr_check(2, rp, np.array([1, 0, 0, 1], np.int32)) == O.ERR_CSR   # unsorted
    assert O.csr_check(2, rp, np.array([0, 0, 0, 1], np.int32)) == O.ERR_CSR   # duplicate
    assert O.csr_check(2, rp, np.array([0, 2, 0, 1], np.int32)) == O.ERR_CSR   # out of range
    assert O.csr_check(2, np.array([0, 1, 2], np.int32), np.array([1, 1], np.int32)) == O.ERR_CSR


# --------------------------------------------------------------------------------------
# ILU(0) / MILU(0)


def test_ilu0_milu0_hand_worked_3x3():
    g = json.load(open(os.path.join(GOLD, "milu_3x3.json")))
    f, st, _ = O.ilu0(g["n"], g["rowptr"], g["colind"], g["val"], milu=False)
    assert st == O.OK
    np.testing.assert_allclose(f, g["ilu0"], rtol=0, atol=1e-15)
    f, st, _ = O.ilu0(g["n"], g["rowptr"], g["colind"], g["val"], milu=True)
    np.testing.assert_allclose(f, g["milu0"], rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 17, 200])
def test_ilu0_equals_exact_lu_without_fill(n):
    """Tridiagonal: LU has no fill, so ILU(0) is the exact LU (Doolittle, unit L)."""
    mat = P.tridiag(n, -1.3, 4.0, -0.7)
    f, st, _ = O.ilu0(*mat)
    assert st == O.OK
    L, U = _split_lu(n, mat[1], mat[2], f)
    A = _csr(mat).toarray()
    Pm, Ld, Ud = sla.lu(A)
    assert np.array_equal(Pm, np.eye(n))            # diagonally dominant: no row swaps
    np.testing.assert_allclose(L.toarray(), Ld, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(U.toarray(), Ud, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("milu", [False, True])
def test_ilu0_reproduces_A_on_its_pattern(seed, milu):
    """(LU)_ij = a_ij on the pattern of A (ILU(0)); MILU keeps this off the diagonal and
    moves the dropped fill to the pivot, so row sums of LU equal row sums of A (Sec. 2.3)."""
    M = _rand_sparse(60, 0.08, seed)
    mat = _mat_tuple(M)
    f, st, npert = O.ilu0(*mat, milu=milu)
    assert st == O.OK and npert == 0
    L, U = _split_lu(mat[0], mat[1], mat[2], f)
    LU = (L @ U).toarray()
    A = M.toarray()
    pat = M.copy()
    pat.data[:] = 1.0
    patd = pat.toarray().astype(bool)
    off = patd & ~np.eye(mat[0], dtype=bool)
    scale = np.abs(A).max()
    if not milu:
        np.testing.assert_allclose(LU[patd], A[patd], rtol=0, atol=1e-12 * scale)
    else:
        np.testing.assert_allclose(LU[off], A[off], rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(LU.sum(axis=1), A.sum(axis=1), rtol=0, atol=1e-11 * scale)


def test_ilu0_on_stencil_pattern_property():
    mat = P.aniso2d_9pt(14, 11, 1e-3, math.pi / 4)
    f, st, _ = O.ilu0(*mat)
    L, U = _split_lu(mat[0], mat[1], mat[2], f)
    A = _csr(mat)
    D = (L @ U - A).tocsr()
    # residual restricted to the pattern of A must vanish
    Pat = A.copy()
    Pat.data[:] = 1.0
    assert np.abs(D.multiply(Pat)).max() < 1e-13


def test_pivot_rule():
    """Sec. 4.1.1: tiny pivots are perturbed to eps * max|a_i:| keeping their sign."""
    # row 1 becomes exactly singular: u11 = 1 - 1*1 = 0
    rp = np.array([0, 2, 4], np.int32)
    ci = np.array([0, 1, 0, 1], np.int32)
    v = np.array([1.0, 1.0, 1.0, 1.0])
    f, st, npert = O.ilu0(2, rp, ci, v, pivot_eps=1e-8)
    assert st == O.OK and npert == 1
    assert f[3] == pytest.approx(1e-8)               # sign(0) = +1, eps * max|a_1j| = 1e-8
    f, st, _ = O.ilu0(2, rp, ci, v, pivot_eps=0.0)
    assert st == O.ERR_ZERO_PIVOT
    v2 = np.array([1.0, 1.0, 1.0, 1.0 - 1e-12])        # u11 = -1e-12: negative small pivot
    f, st, npert = O.ilu0(2, rp, ci, v2, pivot_eps=1e-8)
    assert npert == 1 and f[3] == pytest.approx(-1e-8)


# --------------------------------------------------------------------------------------
# ILUT


@pytest.mark.parametrize("seed", range(3))
def test_ilut_without_dropping_is_exact_lu(seed):
    M = _rand_sparse(40, 0.1, seed)
    mat = _mat_tuple(M)
    rp, ci, v = O.ilut(*mat, tau=0.0, p=10**9)
    L, U = _split_lu(mat[0], rp, ci, v)
    np.testing.assert_allclose((L @ U).toarray(), M.toarray(), rtol=0,
                               atol=1e-12 * np.abs(M).max())


def test_ilut_equals_ilu0_when_no_fill_and_no_drop():
    mat = P.tridiag(50, -1.0, 3.0, -1.2)
    rp, ci, v = O.ilut(*mat, tau=1e-12, p=10)
    f, _, _ = O.ilu0(*mat)
    assert np.array_equal(rp, mat[1]) and np.array_equal(ci, mat[2])
    np.testing.assert_allclose(v, f, rtol=1e-15, atol=0)


@pytest.mark.parametrize("tau,pk", [(1e-2, 3), (1e-3, 10), (0.2, 1)])
def test_ilut_dropping_rules(tau, pk):
    """Dual threshold: every kept off-diagonal |l_ij|, |u_ij| >= tau ||a_i||_2 and at most p
    of them in each of the L and U parts of a row; the diagonal is always kept."""
    mat = P.aniso3d_7pt(7, 6, 5, 1.0, 1.0, 1e-3)
    n = mat[0]
    rp, ci, v = O.ilut(*mat, tau=tau, p=pk)
    A = _csr(mat)
    for i in range(n):
        t = tau * np.linalg.norm(A.data[A.indptr[i]:A.indptr[i + 1]])
        cols = ci[rp[i]:rp[i + 1]]
        vals = v[rp[i]:rp[i + 1]]
        assert np.all(np.diff(cols) > 0) and i in cols
        off = cols != i
        assert np.all(np.abs(vals[off]) >= t)
        assert np.sum(cols < i) <= pk and np.sum(cols > i) <= pk


def test_ilut_hand_worked_drop():
    """Hand-worked dual-threshold ILUT on A = [[4,-1,-1],[-1,4,.],[-1,.,4]] ((1,2), (2,1)
    not stored), t_i = tau ||a_i||_2, ||a_1|| = ||a_2|| = sqrt(17):
      row 1: l10 = -1/4; u11 = 4 - 1/4 = 3.75; fill u12 = -(-1/4)(-1) = -1/4.
      row 2: l20 = -1/4; fill w1 = -1/4, u22 = 3.75; then l21 = w1/u11 = -1/15 and
             u22 -= l21 u12 = 3.75 - 1/60.
    tau = 1e-3 keeps everything; tau = 0.05 (t = 0.206) drops l21 = -1/15 before its
    update; tau = 0.07 (t = 0.289) drops l10 and l20 (|1/4| < t)."""
    rp = np.array([0, 3, 5, 7], np.int32)
    ci = np.array([0, 1, 2, 0, 1, 0, 2], np.int32)
    v = np.array([4.0, -1.0, -1.0, -1.0, 4.0, -1.0, 4.0])
    def rows(tau, pk):
        r, c, val = O.ilut(3, rp, ci, v, tau=tau, p=pk)
        return [(list(c[r[i]:r[i + 1]]), list(val[r[i]:r[i + 1]])) for i in range(3)]
    out = rows(1e-3, 10)
    assert out[1] == ([0, 1, 2], [-0.25, 3.75, -0.25])
    assert out[2][0] == [0, 1, 2]
    np.testing.assert_allclose(out[2][1], [-0.25, -1 / 15, 3.75 - 1 / 60], rtol=1e-15)
    out = rows(0.05, 10)
    assert out[1] == ([0, 1, 2], [-0.25, 3.75, -0.25])
    assert out[2] == ([0, 2], [-0.25, 3.75])
    out = rows(0.07, 10)
    assert out[0] == ([0, 1, 2], [4.0, -1.0, -1.0])
    assert out[1] == ([1], [4.0]) and out[2] == ([2], [4.0])
    # p = 1: row 0's two U entries tie at |-1|, the smaller column wins, so u02 is gone;
    # row 1 has no fill, row 2 gets fill w1 = -1/4, l21 = -1/15 (no U-row 1 to apply),
    # u22 stays 4, and the larger of l20, l21 survives.
    out = rows(1e-3, 1)
    assert out[0] == ([0, 1], [4.0, -1.0])
    assert out[1] == ([0, 1], [-0.25, 3.75])
    assert out[2] == ([0, 2], [-0.25, 4.0])


# --------------------------------------------------------------------------------------
# triangular solves, SpMV, levels


def test_trsv_and_spmv_match_scipy():
    M = _rand_sparse(80, 0.06, 7)
    mat = _mat_tuple(M)
    f, _, _ = O.ilu0(*mat)
    L, U = _split_lu(mat[0], mat[1], mat[2], f)
    b = np.random.default_rng(3).standard_normal(mat[0])
    xl = O.trsv_lower_unit(*mat[:3], f, b)
    xu = O.trsv_upper(*mat[:3], f, b)
    np.testing.assert_allclose(xl, spla.spsolve_triangular(L, b, lower=True), rtol=1e-12)
    np.testing.assert_allclose(xu, spla.spsolve_triangular(U, b, lower=False), rtol=1e-12)
    np.testing.assert_allclose(O.spmv(*mat, b), M @ b, rtol=1e-13)


@pytest.mark.parametrize("upper", [False, True])
@pytest.mark.parametrize("seed", range(3))
def test_levels_are_longest_paths(upper, seed):
    """Level scheduling (Sec. 3.1): every dependency of a row sits in an earlier level,
    and a row's level is minimal: level 0 has no dependency, level l > 0 has one at l-1."""
    M = _rand_sparse(120, 0.03, seed)
    mat = _mat_tuple(M)
    lev, nl = O.levels(*mat[:3], upper=upper)
    assert nl == lev.max() + 1
    rp, ci = mat[1], mat[2]
    for i in range(mat[0]):
        deps = [j for j in ci[rp[i]:rp[i + 1]] if (j > i if upper else j < i)]
        for j in deps:
            assert lev[j] < lev[i]
        if lev[i] == 0:
            assert not deps
        else:
            assert any(lev[j] == lev[i] - 1 for j in deps)


def test_levels_of_2d_9pt_grid():
    """Natural ordering of a 9-point grid: row (x,y) depends on (x-1,y) and (x+1,y-1), so
    its lower level is x + 2y; on an m x m grid there are 3(m-1)+1 levels."""
    m = 9
    mat = P.aniso2d_9pt(m, m, 1e-3, 0.3)
    lev, nl = O.levels(*mat[:3], upper=False)
    x = np.arange(m * m) % m
    y = np.arange(m * m) // m
    assert np.array_equal(lev, x + 2 * y) and nl == 3 * (m - 1) + 1


# --------------------------------------------------------------------------------------
# domain decomposition


@pytest.mark.parametrize("seed", range(4))
def test_classification_and_permutation_properties(seed):
    """Sec. 2.2.1: after relabelling interior nodes first, B (interior x interior) is block
    diagonal by subdomain, E and F couple only nodes of one subdomain, each interface node
    has a coupling to another subdomain (in A or A^T), and groups keep ascending order."""
    rng = np.random.default_rng(seed)
    M = _rand_sparse(150, 0.015, seed)
    p = 5
    part = rng.integers(0, p, size=150).astype(np.int32)
    mat = _mat_tuple(M)
    iface = O.classify(mat[0], mat[1], mat[2], part, p)
    perm, iperm, int_ptr, if_ptr, n1 = O.permutation(mat[0], part, p, iface)
    assert np.array_equal(np.sort(perm), np.arange(150)) and np.array_equal(iperm[perm], np.arange(150))
    assert n1 == int((iface == 0).sum())
    Ap = M[perm][:, perm].tocoo()
    for i, j in zip(Ap.row, Ap.col):
        if i < n1 or j < n1:                      # entry of B, E or F
            assert part[perm[i]] == part[perm[j]]
    # each interface node really couples to another subdomain
    Acoo = M.tocoo()
    cross = np.zeros(150, bool)
    m = part[Acoo.row] != part[Acoo.col]
    cross[Acoo.row[m]] = True
    cross[Acoo.col[m]] = True
    assert np.array_equal(cross, iface.astype(bool))
    # groups: interior by subdomain then interface by subdomain, ascending original index
    for s in range(p):
        g = perm[int_ptr[s]:int_ptr[s + 1]]
        assert np.all(part[g] == s) and np.all(np.diff(g) > 0) and not iface[g].any()
        g = perm[n1 + if_ptr[s]:n1 + if_ptr[s + 1]]
        assert np.all(part[g] == s) and np.all(np.diff(g) > 0) and iface[g].all()


def test_structural_counts_of_the_2d_workload():
    """64x64 5-point Poisson on 2x2 boxes: interface = the two grid lines next to each cut
    (each box side has 32 nodes): n2 = 4*2*32 - 4 = 252, n1 = 4096 - 252. Block Jacobi
    factors whole blocks (Sec. 2.1): no interface, no C_off."""
    pr = P.make_workload("poisson2d_64_p4")
    o = O.Oracle.from_problem(pr, variant="schur", factor_B="ilu0", factor_S="milu0")
    s = o.sizes()
    assert (s.n, s.nnz, s.n1, s.n2, s.nnz_coff) == (4096, 20224, 3844, 252, 256)
    s = O.Oracle.from_problem(pr, variant="bj", factor_B="ilu0", factor_S="ilu0").sizes()
    assert (s.n, s.nnz, s.n1, s.n2, s.nnz_coff) == (4096, 20224, 4096, 0, 0)


# --------------------------------------------------------------------------------------
# Schur complement and the exact two-level identities


def _small_dd(kind, seed=0):
    if kind == "aniso2d":
        return P.aniso2d_boxes(10, 2, seed=seed)
    if kind == "conv3d":
        return P.convdiff3d_boxes(6, 2, seed=seed)
    if kind == "rand":
        return P.randsparse(60, 4, mean_k=3.0, seed=seed)
    raise KeyError(kind)


@pytest.mark.parametrize("kind", ["aniso2d", "conv3d", "rand"])
def test_schur_complement_is_inverse_of_A_inverse_block(kind):
    """S = C - E B^{-1} F (Eq. blockldu) satisfies S^{-1} = (A^{-1})_{22} (Eq. blockldusolve)."""
    pr = _small_dd(kind)
    o = O.Oracle.from_problem(pr, factor_B="exact", factor_S="exact")
    pm = o.perm()
    S = o.schur_dense()
    A = pr.scipy().toarray()[np.ix_(pm["perm"], pm["perm"])]
    n1 = pm["n1"]
    Ainv22 = np.linalg.inv(A)[n1:, n1:]
    np.testing.assert_allclose(np.linalg.inv(S), Ainv22, rtol=1e-9, atol=1e-12)
    # and brute force on the permuted dense matrix
    B, F, E, Cc = A[:n1, :n1], A[:n1, n1:], A[n1:, :n1], A[n1:, n1:]
    np.testing.assert_allclose(S, Cc - E @ np.linalg.solve(B, F), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("kind", ["aniso2d", "conv3d", "rand"])
def test_exact_local_factors_give_exact_schur_blocks(kind):
    """Eq. BILU: with an exact LU of A_i the (2,2) factor block is L_S U_S = S_i, and the
    off-diagonal blocks of S are those of C (Sec. 2.2.2), so blockdiag(L_S U_S) + C_off = S."""
    pr = _small_dd(kind)
    o = O.Oracle.from_problem(pr, factor_B="exact", factor_S="exact")
    np.testing.assert_allclose(o.sapprox_dense(), o.schur_dense(), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("kind", ["aniso2d", "conv3d", "rand"])
@pytest.mark.parametrize("form", ["wz", "ef"])
def test_exact_two_level_apply_is_A_inverse(kind, form):
    """Eq. blockldusolve: with exact B and S solves the two-level apply is A^{-1}; inner GMRES
    with as many steps as interface unknowns solves the Schur system exactly."""
    pr = _small_dd(kind)
    n2 = O.Oracle.from_problem(pr).sizes().n2
    o = O.Oracle.from_problem(pr, factor_B="exact", factor_S="exact", form=form,
                              inner_iters=max(n2, 1))
    r = np.random.default_rng(5).standard_normal(pr.n)
    z = o.apply(r)
    np.testing.assert_allclose(z, np.linalg.solve(pr.scipy().toarray(), r), rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("kind", ["aniso2d", "conv3d", "cuts3d"])
def test_pmilu0_is_milu0_of_the_partial_ilu_schur_complement(kind):
    """Sec. 3.2 (partial ILU): the partial ILU(0) of A_i leaves S~ = (C - W Z) on the pattern
    of C, with W = E U_B^{-1} and Z = L_B^{-1} F from the ILU(0) factors (Eq. pILU); factor_S =
    pmilu0 is MILU(0) of that S~. Built here from the ILU(0) factors by a sparse product and
    the separately pinned MILU(0) routine; the interior rows are plain ILU(0)."""
    pr = P.aniso3d_cuts(10, ncuts=(1, 1, 1), seed=3) if kind == "cuts3d" else _small_dd(kind)
    kw = dict(variant="schur", factor_B="ilu0", pivot_eps=0.0)
    o = O.Oracle.from_problem(pr, factor_S="pmilu0", **kw)
    o0 = O.Oracle.from_problem(pr, factor_S="ilu0", **kw)
    pm = o.perm()
    checked = 0
    for sd in range(pr.p):
        ni = int(pm["int_ptr"][sd + 1] - pm["int_ptr"][sd])
        rp, ci, av = o.local_csr(sd)
        m = rp.size - 1
        if ni == m or ni == 0:
            continue
        f1 = o0.local_factor(sd, 1)                 # ILU(0) of A_i
        f2 = o.local_factor(sd, 2)                  # the pmilu0 factorisation
        F1 = sp.csr_matrix((f1, ci, rp), shape=(m, m)).toarray()
        Am = sp.csr_matrix((av, ci, rp), shape=(m, m)).toarray()
        pat = sp.csr_matrix((np.ones(ci.size), ci, rp), shape=(m, m)).toarray() != 0
        W, Z = F1[ni:, :ni], F1[:ni, ni:]
        St = np.where(pat[ni:, ni:], Am[ni:, ni:] - W @ Z, 0.0)
        Sc = sp.csr_matrix(St * pat[ni:, ni:])
        # keep the pattern of C (explicit zeros included)
        Sc = sp.csr_matrix((St[pat[ni:, ni:]], np.nonzero(pat[ni:, ni:])[1],
                            np.r_[0, np.cumsum(pat[ni:, ni:].sum(axis=1))]), shape=(m - ni, m - ni))
        fS, st, _ = O.ilu0(m - ni, Sc.indptr, Sc.indices, Sc.data, milu=True)
        assert st == 0
        F2 = sp.csr_matrix((f2, ci, rp), shape=(m, m)).toarray()
        got = F2[ni:, ni:][pat[ni:, ni:]]
        np.testing.assert_allclose(got, fS, rtol=1e-11, atol=1e-12 * np.abs(fS).max())
        # interior rows: plain ILU(0), identical
        assert np.array_equal(f2[:rp[ni]], f1[:rp[ni]])
        checked += 1
    assert checked > 0
    with pytest.raises(RuntimeError):
        O.Oracle.from_problem(pr, variant="bj", factor_S="pmilu0")


def test_inner_gmres_full_steps_solves_preconditioned_schur_system():
    """Eq. preSS: (I + S~^{-1} C_off) y = S~^{-1} g'  <=>  (blockdiag(L_S U_S) + C_off) y = g'.
    With k = n2 steps inner GMRES returns that solution; residuals shrink with k."""
    pr = P.aniso2d_boxes(12, 3)
    n2 = O.Oracle.from_problem(pr).sizes().n2
    g = np.random.default_rng(2).standard_normal(n2)
    o = O.Oracle.from_problem(pr, inner_iters=n2)
    Sa = o.sapprox_dense()
    np.testing.assert_allclose(o.inner_gmres(g), np.linalg.solve(Sa, g), rtol=1e-8, atol=1e-10)
    prev = np.inf
    for k in range(1, 8):
        ok = O.Oracle.from_problem(pr, inner_iters=k)
        res = np.linalg.norm(Sa @ ok.inner_gmres(g) - g)
        # GMRES minimises the preconditioned residual; check the unpreconditioned one loosely
        assert res <= prev * 1.5 + 1e-14
        prev = min(prev, res)


def test_milu_preserves_constants_through_P():
    """Sec. 3.3 (Eq. iluares..miluwz3): with MILU(0) of A_i and interior rows of zero row
    sum (B1 + F1 = 0), the interpolation keeps constants, P1 = 1 i.e. U_B^{-1} Z 1 = -1, and
    L_S U_S 1 = E 1 + C 1 on every subdomain."""
    rng = np.random.default_rng(11)
    m = 15
    n = m * m
    # weighted graph Laplacian of a periodic 5-point grid (zero row sums everywhere, so no
    # interior row touches a physical boundary); nonsymmetric weights
    rows, cols, vals = [], [], []
    for y in range(m):
        for x in range(m):
            i = x + m * y
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                rows.append(i)
                cols.append((x + dx) % m + m * ((y + dy) % m))
                vals.append(-rng.uniform(0.5, 2.0))
    W = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    Lap = (W - sp.diags(np.asarray(W.sum(axis=1)).ravel())).tocsr()
    Lap.sort_indices()
    part, p = P.box_partition((m, m), (3, 3))
    iface = O.classify(n, *_mat_tuple(Lap)[1:3], part, p)
    shift = np.where(iface == 1, 1.0, 0.0)          # only interface rows lose zero row sum
    A = (Lap + sp.diags(shift)).tocsr()
    A.sort_indices()
    mat = _mat_tuple(A)
    o = O.Oracle(*mat, part, p, variant="schur", factor_B="milu0", factor_S="milu0")
    pm = o.perm()
    n1 = pm["n1"]
    assert 0 < n1 < n
    for s in range(p):
        rp, ci, a = o.local_csr(s)
        f = o.local_factor(s, 1)
        ns = rp.size - 1
        ni = pm["int_ptr"][s + 1] - pm["int_ptr"][s]
        Al = sp.csr_matrix((a, ci, rp), shape=(ns, ns)).toarray()
        Fm = sp.csr_matrix((f, ci, rp), shape=(ns, ns)).toarray()
        L = np.tril(Fm, -1) + np.eye(ns)
        U = np.triu(Fm)
        assert np.allclose(Al[:ni].sum(axis=1), 0.0, atol=1e-12)
        if ni:
            UB, Z = U[:ni, :ni], U[:ni, ni:]
            np.testing.assert_allclose(np.linalg.solve(UB, Z @ np.ones(ns - ni)), -1.0,
                                       rtol=1e-9, atol=1e-9)
        LS, US = L[ni:, ni:], U[ni:, ni:]
        np.testing.assert_allclose(LS @ US @ np.ones(ns - ni), Al[ni:].sum(axis=1),
                                   rtol=1e-9, atol=1e-9)


def test_single_subdomain_two_level_is_global_ilu0():
    """p = 1: no interface, so SCHUR == BJ == global ILU(0) (Sec. 4.1.1, Np=1 rows)."""
    pr = P.aniso2d_boxes(16, 1)
    r = np.random.default_rng(0).standard_normal(pr.n)
    zs = O.Oracle.from_problem(pr, variant="schur").apply(r)
    zb = O.Oracle.from_problem(pr, variant="bj", factor_B="ilu0").apply(r)
    f, _, _ = O.ilu0(pr.n, pr.rowptr, pr.colind, pr.val)
    zg = O.trsv_upper(pr.n, pr.rowptr, pr.colind, f,
                      O.trsv_lower_unit(pr.n, pr.rowptr, pr.colind, f, r))
    assert np.array_equal(zs, zb) and np.array_equal(zb, zg)


def test_bj_apply_is_blockwise_ilu0():
    """Block Jacobi (Sec. 2.1, Algorithm 'Block Jacobi ILU on GPU'): dropping every E_ij the
    apply equals ILU(0) solves of each diagonal block A_i, via scipy on the permuted blocks."""
    pr = P.convdiff3d_boxes(8, 2)
    o = O.Oracle.from_problem(pr, variant="bj", factor_B="ilu0")
    r = np.random.default_rng(4).standard_normal(pr.n)
    z = o.apply(r)
    A = pr.scipy()
    zz = np.zeros(pr.n)
    for s in range(pr.p):
        idx = np.nonzero(pr.part == s)[0]
        # block Jacobi has no interface: the local order is the subdomain's nodes ascending
        Ai = A[idx][:, idx].tocsr()
        Ai.sort_indices()
        f, _, _ = O.ilu0(idx.size, Ai.indptr, Ai.indices, Ai.data)
        L, U = _split_lu(idx.size, Ai.indptr, Ai.indices, f)
        zz[idx] = spla.spsolve_triangular(U, spla.spsolve_triangular(L, r[idx], lower=True),
                                          lower=False)
    np.testing.assert_allclose(z, zz, rtol=1e-12, atol=1e-13)


# --------------------------------------------------------------------------------------
# RCM local order (Sec. 3.1)


def _sym_pattern(n, edges):
    rows = [a for a, b in edges] + [b for a, b in edges]
    cols = [b for a, b in edges] + [a for a, b in edges]
    G = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    G.sum_duplicates()
    G.sort_indices()
    return G


def _random_graph_with_unique_start(n, extra, seed):
    """connected random graph whose every node has degree >= 2, plus one pendant node:
    the pendant is then the unique node of least degree"""
    rng = np.random.default_rng(seed)
    lab = rng.permutation(n)
    edges = [(lab[k], lab[rng.integers(0, k)]) for k in range(1, n)]  # random tree
    edges += [tuple(rng.choice(n, 2, replace=False)) for _ in range(extra)]
    while True:
        deg = np.diff(_sym_pattern(n, edges).indptr)
        low = np.nonzero(deg < 2)[0]
        if low.size == 0:
            break
        for i in low:
            edges.append((int(i), int((i + 1 + rng.integers(0, n - 1)) % n)))
    edges.append((n, int(rng.integers(0, n))))
    return _sym_pattern(n + 1, edges)


@pytest.mark.parametrize("seed", range(5))
def test_rcm_equals_scipy_when_the_start_node_is_unique(seed):
    """scipy.sparse.csgraph.reverse_cuthill_mckee starts each component at a node of least
    degree and appends neighbours by degree, keeping their index order on ties; with a
    unique least-degree node the two orders must agree node for node."""
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    G = _random_graph_with_unique_start(60 + 40 * seed, 30 + 50 * seed, seed)
    deg = np.diff(G.indptr)
    assert np.sum(deg == deg.min()) == 1
    got = O.rcm(G.shape[0], G.indptr, G.indices)
    ref = reverse_cuthill_mckee(G, symmetric_mode=True)
    assert np.array_equal(got, ref)


def test_rcm_of_a_grid_with_a_pendant_equals_scipy_and_is_banded():
    """5-point grid 23 x 9 with one pendant node: same order as scipy, and (Cuthill-McKee
    being a breadth-first search from the start node, which RCM puts last) the graph
    distance from the start never increases along the RCM order."""
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    mx, my = 23, 9
    n, rp, ci, _ = P.poisson2d_5pt(mx, my)
    A = sp.csr_matrix((np.ones(rp[n]), ci, rp), shape=(n, n)).tolil()
    A.resize((n + 1, n + 1))
    A[n, 5 + mx * 4] = 1.0
    A[5 + mx * 4, n] = 1.0
    G = A.tocsr()
    G.setdiag(0)
    G.eliminate_zeros()
    G.sort_indices()
    got = O.rcm(n + 1, G.indptr, G.indices)
    assert np.array_equal(got, reverse_cuthill_mckee(G, symmetric_mode=True))
    from scipy.sparse.csgraph import shortest_path
    assert got[-1] == n  # the pendant, the only node of degree 1
    d = shortest_path(G, unweighted=True, indices=n)
    assert np.all(np.diff(d[got]) <= 0)


def test_rcm_hand_worked_with_ties_and_components():
    """A 12-node pattern worked by hand (tests/golden/rcm_hand.json): degree ties broken by
    index, degree before index among neighbours, three components, entries stored in one
    direction only, duplicates and diagonal entries ignored."""
    g = json.load(open(os.path.join(GOLD, "rcm_hand.json")))
    n = g["n"]
    r = [a for a, b in g["stored"]]
    c = [b for a, b in g["stored"]]
    M = sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(n, n))
    M.sort_indices()
    S = ((M + M.T) > 0).astype(float).tolil()
    S.setdiag(0)
    S = S.tocsr()
    S.eliminate_zeros()
    assert list(np.diff(S.indptr)) == g["degrees"]
    assert list(O.rcm(n, M.indptr, M.indices)) == g["order"]


def test_rcm_depends_only_on_the_symmetrised_graph():
    M = _rand_sparse(80, 0.04, seed=9)
    S = (abs(M) + abs(M).T).tocsr()
    S.sort_indices()
    a = O.rcm(80, M.indptr, M.indices)
    assert np.array_equal(np.sort(a), np.arange(80))
    assert np.array_equal(a, O.rcm(80, S.indptr, S.indices))


def test_bj_rcm_apply_is_blockwise_ilu0_in_rcm_order():
    """Algorithm 'Block Jacobi ILU on GPU': each A_i put in its RCM order, ILU(0) of the
    reordered block, two triangular solves, scattered back (scipy solves)."""
    pr = P.convdiff3d_boxes(8, 2)
    o = O.Oracle.from_problem(pr, variant="bj", factor_B="ilu0", local_order="rcm")
    perm = o.perm()["perm"]
    r = np.random.default_rng(4).standard_normal(pr.n)
    z = o.apply(r)
    A = pr.scipy()
    zz = np.zeros(pr.n)
    at = 0
    for s in range(pr.p):
        nat = np.nonzero(pr.part == s)[0]
        B = A[nat][:, nat].tocsr()
        B.sort_indices()
        idx = nat[O.rcm(nat.size, B.indptr, B.indices)]
        assert np.array_equal(perm[at:at + idx.size], idx)
        at += idx.size
        Ai = A[idx][:, idx].tocsr()
        Ai.sort_indices()
        f, _, _ = O.ilu0(idx.size, Ai.indptr, Ai.indices, Ai.data)
        L, U = _split_lu(idx.size, Ai.indptr, Ai.indices, f)
        zz[idx] = spla.spsolve_triangular(U, spla.spsolve_triangular(L, r[idx], lower=True),
                                          lower=False)
    np.testing.assert_allclose(z, zz, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("kind", ["aniso2d", "conv3d", "rand"])
def test_two_level_rcm_orders_each_group_and_stays_exact(kind):
    """Two-level with the RCM local order: every interior group and every interface group
    is the RCM order of the graph it induces, the split is unchanged, and with exact local
    factors and n2 inner steps the apply is still A^{-1} (Eq. blockldusolve)."""
    pr = _small_dd(kind)
    A = pr.scipy()
    nat = O.Oracle.from_problem(pr).perm()
    o = O.Oracle.from_problem(pr, factor_B="exact", factor_S="exact", local_order="rcm",
                              inner_iters=max(nat["n2"], 1))
    pm = o.perm()
    for k in ("int_ptr", "if_ptr", "iface"):
        assert np.array_equal(pm[k], nat[k])
    n1 = pm["n1"]
    groups = [(pm["int_ptr"][s], pm["int_ptr"][s + 1]) for s in range(pr.p)]
    groups += [(n1 + pm["if_ptr"][s], n1 + pm["if_ptr"][s + 1]) for s in range(pr.p)]
    for a, b in groups:
        g = np.sort(nat["perm"][a:b])
        G = A[g][:, g].tocsr()
        G.sort_indices()
        assert np.array_equal(pm["perm"][a:b], g[O.rcm(g.size, G.indptr, G.indices)])
    assert np.array_equal(pm["iperm"][pm["perm"]], np.arange(pr.n))
    r = np.random.default_rng(5).standard_normal(pr.n)
    np.testing.assert_allclose(o.apply(r), np.linalg.solve(A.toarray(), r), rtol=1e-9, atol=1e-10)


# --------------------------------------------------------------------------------------
# Multicolour local order (Sec. 3.1: fewer levels in the triangular solves)


def test_color_of_grids_is_the_checkerboard():
    """Greedy colouring in natural order: the 5-point grid gets the red-black colouring
    (x + y) mod 2, the 9-point grid the four colours (x mod 2) + 2 (y mod 2)."""
    side = 17
    x, y = np.arange(side * side) % side, np.arange(side * side) // side
    p5 = P.poisson2d_boxes(side, 1, seed=0)
    c5, o5, n5 = O.color(p5.n, p5.rowptr, p5.colind)
    assert n5 == 2 and np.array_equal(c5, (x + y) % 2)
    p9 = P.aniso2d_boxes(side, 1, seed=0)
    c9, o9, n9 = O.color(p9.n, p9.rowptr, p9.colind)
    assert n9 == 4 and np.array_equal(c9, (x % 2) + 2 * (y % 2))
    assert np.array_equal(o9, np.lexsort((np.arange(p9.n), c9)))


@pytest.mark.parametrize("seed", range(6))
def test_color_is_proper_and_first_fit(seed):
    """On random graphs: no edge joins two nodes of one colour, every node of colour c has an
    earlier neighbour of each colour below c (it took the smallest free one), and the order
    lists the nodes by (colour, index)."""
    rng = np.random.default_rng(seed)
    n = 60
    edges = [tuple(rng.choice(n, 2, replace=False)) for _ in range(150)]
    G = _sym_pattern(n, edges)
    col, order, nc = O.color(n, G.indptr, G.indices)
    assert nc == col.max() + 1
    for i in range(n):
        nb = G.indices[G.indptr[i]:G.indptr[i + 1]]
        nb = nb[nb != i]
        assert not np.any(col[nb] == col[i])
        earlier = set(col[nb[nb < i]].tolist())
        assert set(range(col[i])) <= earlier
    assert np.array_equal(order, np.lexsort((np.arange(n), col)))


@pytest.mark.parametrize("kind", ["aniso2d", "conv3d", "rand"])
def test_color_order_gives_one_level_per_colour(kind):
    """Block Jacobi with one subdomain in colour order: the lower factor of ILU(0) (pattern of
    A) has as many levels as colours, the colour classes being independent sets."""
    pr = {"aniso2d": lambda: P.aniso2d_boxes(20, 1, seed=2), "conv3d": lambda: P.convdiff3d_boxes(7, 1, seed=2),
          "rand": lambda: P.randsparse(300, 1, mean_k=4.0, seed=2)}[kind]()
    o = O.Oracle.from_problem(pr, variant="bj", factor_B="ilu0", factor_S="ilu0", local_order="color")
    _, _, nc = O.color(pr.n, pr.rowptr, pr.colind)
    assert o.levels(0)[1] == nc
    perm = o.perm()["perm"]
    col, order, _ = O.color(pr.n, pr.rowptr, pr.colind)
    assert np.array_equal(perm, order)


@pytest.mark.parametrize("kind", ["aniso2d", "conv3d", "rand"])
def test_two_level_color_orders_each_group_and_stays_exact(kind):
    """Two-level with the colour order: each interior and interface group is the colour order
    of the graph it induces, the split is unchanged, and with exact local factors and n2
    inner steps the apply is A^{-1} (Eq. blockldusolve)."""
    pr = _small_dd(kind)
    A = pr.scipy()
    nat = O.Oracle.from_problem(pr).perm()
    o = O.Oracle.from_problem(pr, factor_B="exact", factor_S="exact", local_order="color",
                              inner_iters=max(nat["n2"], 1))
    pm = o.perm()
    for k in ("int_ptr", "if_ptr", "iface"):
        assert np.array_equal(pm[k], nat[k])
    n1 = pm["n1"]
    groups = [(pm["int_ptr"][s], pm["int_ptr"][s + 1]) for s in range(pr.p)]
    groups += [(n1 + pm["if_ptr"][s], n1 + pm["if_ptr"][s + 1]) for s in range(pr.p)]
    for a, b in groups:
        g = np.sort(nat["perm"][a:b])
        G = A[g][:, g].tocsr()
        G.sort_indices()
        assert np.array_equal(pm["perm"][a:b], g[O.color(g.size, G.indptr, G.indices)[1]])
    r = np.random.default_rng(5).standard_normal(pr.n)
    np.testing.assert_allclose(o.apply(r), np.linalg.solve(A.toarray(), r), rtol=1e-9, atol=1e-10)


# --------------------------------------------------------------------------------------
# ILU(k) (level of fill; the paper runs ILU(1) and ILU(2) in Sec. 4.2-4.4)


def _fill_path_levels(M, k):
    """Brute force from the fill-path theorem (Hysom and Pothen): (i, j) has level l iff the
    shortest directed path i -> j in the graph of A whose inner vertices are all below
    min(i, j) has l + 1 edges. Returns the set of positions of level <= k."""
    n = M.shape[0]
    adj = [set(M.indices[M.indptr[i]:M.indptr[i + 1]]) - {i} for i in range(n)]
    keep = set((i, i) for i in range(n))
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            lo = min(i, j)
            dist, frontier, seen = 0, {i}, {i}
            found = None
            while frontier and found is None and dist <= k:
                dist += 1
                nxt = set()
                for u in frontier:
                    for w in adj[u]:
                        if w == j:
                            found = dist
                        elif w < lo and w not in seen:
                            seen.add(w)
                            nxt.add(w)
                frontier = nxt
            if found is not None and found - 1 <= k:
                keep.add((i, j))
    return keep


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_iluk_pattern_is_the_fill_path_closure(seed, k):
    M = _rand_sparse(18, 0.09, seed=40 + seed)
    rp, ci, _ = O.iluk_pattern(18, M.indptr, M.indices, M.data, k)
    got = {(i, int(j)) for i in range(18) for j in ci[rp[i]:rp[i + 1]]}
    assert got == _fill_path_levels(M, k)


def test_iluk_of_the_5pt_grid_adds_the_two_textbook_diagonals():
    """Natural order, 5-point grid nx x ny: ILU(1) adds exactly (i, i - nx + 1) and
    (i, i + nx - 1) where both nodes exist (eliminating the south and west neighbours)."""
    nx, ny = 7, 5
    n, rp, ci, v = P.poisson2d_5pt(nx, ny)
    r1, c1, v1 = O.iluk_pattern(n, rp, ci, v, 1)
    base = {(i, int(j)) for i in range(n) for j in ci[rp[i]:rp[i + 1]]}
    got = {(i, int(j)) for i in range(n) for j in c1[r1[i]:r1[i + 1]]}
    want = set(base)
    for i in range(n):
        x, y = i % nx, i // nx
        if y > 0 and x < nx - 1:
            want.add((i, i - nx + 1))
        if y < ny - 1 and x > 0:
            want.add((i, i + nx - 1))
    assert got == want
    A = sp.csr_matrix((v, ci, rp), shape=(n, n))
    F = sp.csr_matrix((v1, c1, r1), shape=(n, n))
    assert abs(F - A).max() == 0  # A's values, zeros at the fill


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("milu", [False, True])
def test_iluk_factors_match_A_on_their_pattern(k, milu):
    """ILU on a pattern P reproduces A on P: (LU)_ij = a_ij there; MILU(k) instead keeps
    every row sum of A (the dropped updates go to the pivot)."""
    M = _rand_sparse(120, 0.03, seed=3)
    n = 120
    part = np.zeros(n, np.int32)
    kind = "milu0" if milu else "ilu0"
    o = O.Oracle(*_mat_tuple(M), part, 1, variant="bj", factor_B=kind, factor_S=kind, fill_level=k)
    rp, ci, _ = o.local_csr(0)
    f = o.local_factor(0, 1)
    L, U = _split_lu(n, rp, ci, f)
    LU = (L @ U).toarray()
    Ad = M.toarray()
    if milu:
        np.testing.assert_allclose(LU.sum(axis=1), Ad.sum(axis=1), rtol=1e-11, atol=1e-11)
        mask = np.zeros((n, n), bool)
        for i in range(n):
            mask[i, ci[rp[i]:rp[i + 1]]] = True
        np.fill_diagonal(mask, False)
        np.testing.assert_allclose(LU[mask], Ad[mask], rtol=1e-11, atol=1e-11)
    else:
        for i in range(n):
            cols = ci[rp[i]:rp[i + 1]]
            np.testing.assert_allclose(LU[i, cols], Ad[i, cols], rtol=1e-11, atol=1e-11)
    assert rp[-1] > M.nnz  # fill was added


def test_iluk_with_a_large_level_is_exact_lu():
    """With k >= n nothing is dropped: L U = A."""
    M = _rand_sparse(60, 0.06, seed=8)
    o = O.Oracle(*_mat_tuple(M), np.zeros(60, np.int32), 1, variant="bj", factor_B="ilu0",
                 factor_S="ilu0", fill_level=60)
    rp, ci, _ = o.local_csr(0)
    L, U = _split_lu(60, rp, ci, o.local_factor(0, 1))
    np.testing.assert_allclose((L @ U).toarray(), M.toarray(), rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("kind", ["aniso2d", "conv3d", "rand"])
def test_two_level_with_exact_iluk_is_A_inverse(kind):
    """ILU(k) with k >= n is exact on every local block, so with n2 inner steps the
    two-level apply is A^{-1} (Eq. blockldusolve); the same with the RCM order."""
    pr = _small_dd(kind)
    n2 = O.Oracle.from_problem(pr).sizes().n2
    r = np.random.default_rng(5).standard_normal(pr.n)
    x = np.linalg.solve(pr.scipy().toarray(), r)
    for order in ("natural", "rcm"):
        o = O.Oracle.from_problem(pr, factor_B="ilu0", factor_S="ilu0", fill_level=pr.n,
                                  inner_iters=max(n2, 1), local_order=order)
        np.testing.assert_allclose(o.apply(r), x, rtol=1e-9, atol=1e-10)


def test_fill_level_needs_level_based_factors():
    pr = _small_dd("aniso2d")
    with pytest.raises(RuntimeError):
        O.Oracle.from_problem(pr, factor_B="ilut", fill_level=1)
    with pytest.raises(RuntimeError):
        O.Oracle.from_problem(pr, fill_level=-1)


# --------------------------------------------------------------------------------------
# l1 block Jacobi (Sec. 4.3)


def _dense_blocks(o, pr):
    """blockdiag of the oracle's stored local blocks, in the original numbering"""
    n = pr.n
    M = np.zeros((n, n))
    perm = o.perm()["perm"]
    at = 0
    for s in range(pr.p):
        rp, ci, v = o.local_csr(s)
        m = rp.size - 1
        idx = perm[at:at + m]
        for r in range(m):
            M[idx[r], idx[ci[rp[r]:rp[r + 1]]]] = v[rp[r]:rp[r + 1]]
        at += m
    return M


@pytest.mark.parametrize("kind", ["aniso2d", "conv3d"])
def test_l1_block_jacobi_dominates_A(kind):
    """The l1 augmentation makes blockdiag(A_i + D_l1) - A positive semidefinite for
    symmetric A (each off-block pair a_ij = a_ji is covered by |a_ij| on both diagonals,
    Gershgorin on the off-block part); without it blockdiag(A_i) - A is indefinite."""
    pr = P.aniso2d_boxes(12, 3, seed=2) if kind == "aniso2d" else P.convdiff3d_boxes(6, 2, seed=1)
    A = pr.scipy().toarray()
    A = 0.5 * (A + A.T)
    Asym = sp.csr_matrix(A)
    Asym.sort_indices()
    n, rp, ci, v = _mat_tuple(Asym)
    o = O.Oracle(n, rp, ci, v, pr.part, pr.p, variant="bj", factor_B="ilu0", factor_S="ilu0", l1_block=True)
    o0 = O.Oracle(n, rp, ci, v, pr.part, pr.p, variant="bj", factor_B="ilu0", factor_S="ilu0")
    scale = np.abs(A).max()
    assert np.linalg.eigvalsh(_dense_blocks(o, pr) - A).min() >= -1e-12 * scale
    assert np.linalg.eigvalsh(_dense_blocks(o0, pr) - A).min() < -1e-3 * scale
    # the augmentation touches only the diagonal
    D = _dense_blocks(o, pr) - _dense_blocks(o0, pr)
    assert np.count_nonzero(D - np.diag(np.diag(D))) == 0


def test_l1_block_jacobi_apply_is_blockwise_ilu0_of_the_augmented_blocks():
    pr = P.convdiff3d_boxes(8, 2)
    o = O.Oracle.from_problem(pr, variant="bj", factor_B="ilu0", l1_block=True)
    r = np.random.default_rng(4).standard_normal(pr.n)
    A = pr.scipy()
    zz = np.zeros(pr.n)
    for s in range(pr.p):
        idx = np.nonzero(pr.part == s)[0]
        out = np.nonzero(pr.part != s)[0]
        Ai = A[idx][:, idx].tolil()
        Ai.setdiag(Ai.diagonal() + np.asarray(abs(A[idx][:, out]).sum(axis=1)).ravel())
        Ai = Ai.tocsr()
        Ai.sort_indices()
        f, _, _ = O.ilu0(idx.size, Ai.indptr, Ai.indices, Ai.data)
        L, U = _split_lu(idx.size, Ai.indptr, Ai.indices, f)
        zz[idx] = spla.spsolve_triangular(U, spla.spsolve_triangular(L, r[idx], lower=True),
                                          lower=False)
    np.testing.assert_allclose(o.apply(r), zz, rtol=1e-12, atol=1e-13)
    with pytest.raises(RuntimeError):
        O.Oracle.from_problem(pr, variant="schur", l1_block=True)


# --------------------------------------------------------------------------------------
# bfloat16 factor storage


def _bf16_bits(x):
    """Round-to-nearest-even to 8 significant bits on the float64 bit pattern (normal
    bfloat16 range): drop the low 45 significand bits, adding half an ulp minus one plus the
    kept lowest bit first."""
    b = np.asarray(x, dtype=np.float64).view(np.uint64)
    keep = (b >> np.uint64(45)) & np.uint64(1)
    r = (b + np.uint64((1 << 44) - 1) + keep) >> np.uint64(45) << np.uint64(45)
    return r.view(np.float64)


def test_round_bf16_matches_the_bit_level_definition():
    rng = np.random.default_rng(31)
    x = rng.standard_normal(4000) * 10.0 ** rng.uniform(-30, 30, 4000)
    ties = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(2.0 + 2.0 ** -7), 3.0 * 2.0 ** -9])
    for v in np.concatenate([x, ties]):
        assert O.round_bf16(v) == _bf16_bits(v), v
    assert O.round_bf16(1.0 + 2.0 ** -8) == 1.0 and O.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    # below 2^-126 the spacing is 2^-133 (np.round: half to even)
    for v in rng.uniform(-1, 1, 200) * 2.0 ** -126:
        assert O.round_bf16(v) == np.round(v * 2.0 ** 133) * 2.0 ** -133
    assert O.round_bf16(3.4e38) == np.inf and O.round_bf16(3.38e38) < np.inf


@pytest.mark.parametrize("variant", ["bj", "schur", "rap"])
def test_bf16_storage_rounds_the_off_diagonal_factor_entries(variant):
    pr = _small_dd("aniso2d")
    kw = dict(variant=variant, factor_B="ilu0", factor_S="milu0")
    o, ob = O.Oracle.from_problem(pr, **kw), O.Oracle.from_problem(pr, store_bf16=True, **kw)
    facts = [1] if variant == "bj" else [1, 2]
    for sd in range(pr.p):
        rp, ci, _ = o.local_csr(sd)
        diag = np.zeros(ci.size, bool)
        for r in range(rp.size - 1):
            diag[rp[r]:rp[r + 1]] = ci[rp[r]:rp[r + 1]] == r
        for f in facts:
            v, vb = o.local_factor(sd, f), ob.local_factor(sd, f)
            assert np.array_equal(vb[diag], v[diag])
            assert np.array_equal(vb[~diag], _bf16_bits(v[~diag]))


def test_bf16_block_jacobi_apply_uses_the_rounded_factors():
    pr = P.convdiff3d_boxes(8, 2)
    ob = O.Oracle.from_problem(pr, variant="bj", factor_B="ilu0", store_bf16=True)
    r = np.random.default_rng(4).standard_normal(pr.n)
    A = pr.scipy()
    zz = np.zeros(pr.n)
    for sd in range(pr.p):
        idx = np.nonzero(pr.part == sd)[0]
        Ai = A[idx][:, idx].tocsr()
        Ai.sort_indices()
        f, _, _ = O.ilu0(idx.size, Ai.indptr, Ai.indices, Ai.data)
        F = sp.csr_matrix((f, Ai.indices, Ai.indptr), shape=Ai.shape)
        off = F - sp.diags(F.diagonal())
        off.data = _bf16_bits(off.data)
        F = (off + sp.diags(F.diagonal())).tocsr()
        L = (sp.tril(F, -1) + sp.identity(idx.size)).tocsr()
        U = sp.triu(F).tocsr()
        zz[idx] = spla.spsolve_triangular(U, spla.spsolve_triangular(L, r[idx], lower=True), lower=False)
    np.testing.assert_allclose(ob.apply(r), zz, rtol=1e-12, atol=1e-13)
    with pytest.raises(RuntimeError):
        O.Oracle.from_problem(pr, variant="schur", factor_B="ilut", store_bf16=True)


# --------------------------------------------------------------------------------------
# FGMRES


def test_fgmres_full_restart_solves_small_system_exactly():
    """GMRES(n) on an n x n system reaches the exact solution (dense solve) within n steps."""
    pr = P.randsparse(25, 2, mean_k=4.0, seed=3)
    o = O.Oracle.from_problem(pr)
    out = o.fgmres(pr.b, rtol=1e-13, restart=25, maxit=25)
    np.testing.assert_allclose(out["x"], np.linalg.solve(pr.scipy().toarray(), pr.b),
                               rtol=1e-10, atol=1e-10)
    assert out["iters"] <= 25


@pytest.mark.parametrize("variant", ["bj", "schur"])
def test_fgmres_residuals_non_increasing_and_givens_matches_true(variant):
    pr = P.aniso2d_boxes(40, 4, seed=1)
    o = O.Oracle.from_problem(pr, variant=variant)
    out = o.fgmres(pr.b, rtol=1e-10, restart=10, maxit=400, hist_len=1000)
    assert out["status"] == O.OK
    h = out["hist"]
    est = []
    true = []
    prev_true = None
    for v in h:
        if v < 0:
            t = -v
            if prev_true is not None:
                assert t <= prev_true * (1 + 1e-8)
                # Givens estimate at the end of the cycle equals the true residual
                assert abs(est[-1] - t) <= 1e-6 * t + 1e-12 * np.linalg.norm(pr.b)
            prev_true = t
            true.append(t)
            cyc = []
        else:
            est.append(v)
            cyc.append(v)
            assert len(cyc) == 1 or cyc[-1] <= cyc[-2] * (1 + 1e-12)
    x = out["x"]
    assert np.linalg.norm(pr.b - pr.scipy() @ x) <= 1e-10 * np.linalg.norm(pr.b) * 1.0001


def test_fgmres_zero_rhs():
    pr = P.aniso2d_boxes(8, 2)
    o = O.Oracle.from_problem(pr)
    out = o.fgmres(np.zeros(pr.n), x0=np.ones(pr.n))
    assert out["status"] == O.OK and out["iters"] == 0 and not out["x"].any()


def _golden_cases(slow):
    g = json.load(open(os.path.join(GOLD, "paper_iteration_counts.json")))
    return [c for c in g["cases"] if bool(c.get("slow")) == slow]


def _run_paper_case(c):
    if c["problem"] == "poisson2d_5pt":
        mat = P.poisson2d_5pt(*c["grid"])
    elif c["problem"] == "convdiff3d_upwind":
        assert len(set(c["grid"])) == 1 and len(set(c["convection"])) == 1
        # the generator's convection is (pe, pe, pe) / sqrt(3)
        mat = P.convdiff3d_upwind(c["grid"][0], c["convection"][0] * math.sqrt(3.0))
    else:
        mat = P.aniso3d_7pt(*c["grid"], 1.0, 1.0, 1.0)
    n = mat[0]
    part, p = P.contiguous_partition(n, c["p"])
    o = O.Oracle(*mat, part, p, variant=c.get("variant", "bj"), factor_B="ilu0",
                 factor_S=c.get("factor_S", "ilu0"), local_order=c.get("local_order", "natural"),
                 fill_level=c.get("fill_level", 0))
    out = o.fgmres(np.ones(n), rtol=c["rtol"], restart=c["restart"], maxit=20000)
    assert out["status"] == O.OK
    return out["iters"]


@pytest.mark.parametrize("case", _golden_cases(False),
                         ids=lambda c: c["problem"] + "-" + c.get("local_order", "natural"))
def test_paper_iteration_counts(case):
    """The paper's printed FGMRES(50) + ILU(0) iteration counts (tests/golden)."""
    assert _run_paper_case(case) == case["iters"]


@pytest.mark.slow
@pytest.mark.parametrize("case", _golden_cases(True),
                         ids=lambda c: f'{c["problem"]}-p{c["p"]}-{c.get("variant", "bj")}-{c.get("local_order", "natural")}')
def test_paper_iteration_counts_slow(case):
    """Larger printed counts (opt-in): block Jacobi on 2D grids split into 4 and 8 blocks of
    whole grid rows (~80 s, ~3 min); ILU(2) on 3D convection-diffusion 128^3 with
    FGMRES(100) (~75 s); RAP-MILU(0) on 1024 x 2048 in 32 blocks (~7 min); block Jacobi on
    3D 128 x 128 x 256 in 2 blocks (~6 min). The 3D Poisson 128^3 count at Np=1 and the 2D
    block Jacobi count in 2 blocks run by default (about 100 s together)."""
    assert _run_paper_case(case) == case["iters"]


# --------------------------------------------------------------------------------------
# generators (stencil sign conventions)


def test_9pt_stencil_reproduces_second_derivatives():
    """-div(K grad u) = -(a u_xx + 2b u_xy + c u_yy); for u = quadratic the 9-point stencil
    is exact, so A u at an interior node equals -(a*2qa + 2b*qb + c*2qc) (h = 1)."""
    eps, th = 0.01, 0.7
    co = P.aniso2d_9pt_coeffs(eps, th)
    a = math.cos(th) ** 2 + eps * math.sin(th) ** 2
    c = math.sin(th) ** 2 + eps * math.cos(th) ** 2
    b = (1 - eps) * math.cos(th) * math.sin(th)
    qa, qb, qc = 0.3, -1.1, 0.7
    u = lambda x, y: qa * x * x + qb * x * y + qc * y * y + 2 * x - y
    val = sum(w * u(dx, dy) for (dx, dy), w in co.items())
    assert val == pytest.approx(-(a * 2 * qa + 2 * b * qb + c * 2 * qc), abs=1e-12)


def test_upwind_convection_diffusion_row():
    """h^2-scaled -Lap u + beta.grad u: a linear u in x gives beta_x h^2 du/dx exactly."""
    m, pe = 5, 50.0
    n, rp, ci, v = P.convdiff3d_upwind(m, pe)
    h = 1.0 / (m + 1)
    bx = pe / math.sqrt(3.0)
    A = sp.csr_matrix((v, ci, rp), shape=(n, n))
    xs = (np.arange(n) % m + 1) * h
    u = 3.0 * xs
    i = 2 + m * (2 + m * 2)                         # an interior node
    assert (A @ u)[i] == pytest.approx(bx * h * h * 3.0, rel=1e-12)


# --------------------------------------------------------------------------------------
# two-level multiplicative (RAP) preconditioner, Sec. 3.3


def _rap_dense(o, A_orig, n):
    """Dense pieces of the RAP preconditioner in the interior-first order, assembled from
    the oracle's local factors: G = blockdiag((L_A U_A)^{-1}) from F1 (smoother), P and R
    of Eq. wzinmilu and blockdiag(L_S U_S) from F2, and A permuted."""
    pm = o.perm()
    perm, n1 = pm["perm"], pm["n1"]
    n2 = n - n1
    Ap = A_orig.toarray()[np.ix_(perm, perm)]
    G = np.zeros((n, n))
    P_ = np.zeros((n, n2))
    R_ = np.zeros((n2, n))
    M = np.zeros((n2, n2))
    for s in range(o.p):
        rp, ci, a = o.local_csr(s)
        ns = rp.size - 1
        ni = pm["int_ptr"][s + 1] - pm["int_ptr"][s]
        gI = pm["int_ptr"][s] + np.arange(ni)
        gG = n1 + pm["if_ptr"][s] + np.arange(ns - ni)
        glob = np.r_[gI, gG]
        iG = gG - n1
        F1 = sp.csr_matrix((o.local_factor(s, 1), ci, rp), shape=(ns, ns)).toarray()
        F2 = sp.csr_matrix((o.local_factor(s, 2), ci, rp), shape=(ns, ns)).toarray()
        L1, U1 = np.tril(F1, -1) + np.eye(ns), np.triu(F1)
        L2, U2 = np.tril(F2, -1) + np.eye(ns), np.triu(F2)
        G[np.ix_(glob, glob)] = np.linalg.inv(L1 @ U1)
        LB, UB, W, Z = L2[:ni, :ni], U2[:ni, :ni], L2[ni:, :ni], U2[:ni, ni:]
        P_[np.ix_(gG, iG)] = np.eye(ns - ni)
        R_[np.ix_(iG, gG)] = np.eye(ns - ni)
        if ni:
            P_[np.ix_(gI, iG)] = -np.linalg.solve(UB, Z)
            R_[np.ix_(iG, gI)] = -W @ np.linalg.inv(LB)
        M[np.ix_(iG, iG)] = L2[ni:, ni:] @ U2[ni:, ni:]
    return dict(Ap=Ap, G=G, P=P_, R=R_, M=M, perm=perm, n1=n1)


@pytest.mark.parametrize("kind", ["aniso2d", "conv3d", "rand"])
def test_rap_apply_is_the_multiplicative_formula(kind):
    """Algorithm "Two-level multiplicative solve" with the GPU smoother of Algorithm
    "Multiplicative RAP-ILU on GPU": with the coarse GMRES run to n2 steps the apply is
    x = x^ + P (RAP)^{-1} R (b - A x^), x^ = blockdiag(L_A U_A)^{-1} b, built densely here
    from the factors (ILU(0) smoother, MILU(0) for P, R and the coarse preconditioner)."""
    pr = _small_dd(kind, seed=3)
    A = pr.scipy()
    n = pr.n
    o0 = O.Oracle.from_problem(pr, variant="rap", factor_B="ilu0", factor_S="milu0")
    n2 = o0.sizes().n2
    assert n2 > 0
    o = O.Oracle.from_problem(pr, variant="rap", factor_B="ilu0", factor_S="milu0", inner_iters=n2)
    d = _rap_dense(o, A, n)
    b = np.random.default_rng(5).standard_normal(n)
    bn = b[d["perm"]]
    xh = d["G"] @ bn
    S = d["R"] @ d["Ap"] @ d["P"]
    v = np.linalg.solve(S, d["R"] @ (bn - d["Ap"] @ xh))
    xn = xh + d["P"] @ v
    ref = np.empty(n)
    ref[d["perm"]] = xn
    got = o.apply(b)
    np.testing.assert_allclose(got, ref, rtol=1e-8, atol=1e-9 * np.abs(ref).max())


def test_rap_smoother_alone_when_the_coarse_space_is_empty():
    """A single subdomain has no interface, so the two-level multiplicative apply is the
    smoother alone: global ILU(0) (Sec. 3.3, Algorithm "Two-level multiplicative solve"
    with an empty coarse space), checked against scipy triangular solves."""
    pr = P.aniso2d_boxes(12, 1, seed=2)
    o = O.Oracle.from_problem(pr, variant="rap", factor_B="ilu0", factor_S="milu0")
    assert o.sizes().n2 == 0
    b = np.random.default_rng(6).standard_normal(pr.n)
    rp, ci, v = pr.rowptr, pr.colind, pr.val
    f, st, _ = O.ilu0(pr.n, rp, ci, v, milu=False)
    assert st == 0
    L, U = _split_lu(pr.n, rp, ci, f)
    ref = spla.spsolve_triangular(U, spla.spsolve_triangular(L, b, lower=True), lower=False)
    np.testing.assert_allclose(o.apply(b), ref, rtol=1e-12, atol=1e-13)


def test_rap_keeps_constants_with_milu():
    """Sec. 3.3 (Eq. miluwz3): with MILU(0) of A_i and interior rows of zero row sum,
    P 1 = 1 and, subdomain by subdomain, R A_i P 1 = L_S U_S 1 (the coarse preconditioner
    keeps the local operator's action on constants: R L = [0, L_S] and H 1 = 0), on a
    periodic weighted graph Laplacian with 3 x 3 boxes."""
    rng = np.random.default_rng(12)
    m = 15
    n = m * m
    rows, cols, vals = [], [], []
    for y in range(m):
        for x in range(m):
            i = x + m * y
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                rows.append(i)
                cols.append((x + dx) % m + m * ((y + dy) % m))
                vals.append(-rng.uniform(0.5, 2.0))
    W = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A = (W - sp.diags(np.asarray(W.sum(axis=1)).ravel())).tocsr()
    A.sort_indices()
    part, p = P.box_partition((m, m), (3, 3))
    o = O.Oracle(*_mat_tuple(A), part, p, variant="rap", factor_B="ilu0", factor_S="milu0")
    d = _rap_dense(o, A, n)
    n2 = n - d["n1"]
    one = np.ones(n2)
    np.testing.assert_allclose(d["P"] @ one, np.ones(n), rtol=1e-9, atol=1e-9)
    # blockdiag(A_i) in the interior-first order: A without the cross-subdomain couplings
    pm = o.perm()
    Aloc = np.zeros((n, n))
    for s in range(p):
        rp, ci, a = o.local_csr(s)
        ns = rp.size - 1
        ni = pm["int_ptr"][s + 1] - pm["int_ptr"][s]
        glob = np.r_[pm["int_ptr"][s] + np.arange(ni), d["n1"] + pm["if_ptr"][s] + np.arange(ns - ni)]
        Aloc[np.ix_(glob, glob)] = sp.csr_matrix((a, ci, rp), shape=(ns, ns)).toarray()
    S_loc = d["R"] @ Aloc @ d["P"]
    np.testing.assert_allclose(S_loc @ one, d["M"] @ one, rtol=1e-8, atol=1e-8)
    # and the global operator annihilates constants here (zero row sums), unlike M
    np.testing.assert_allclose(d["R"] @ d["Ap"] @ d["P"] @ one, 0.0, atol=1e-8)
