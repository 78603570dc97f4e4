"""Seeded synthetic problem generators: grids, stencils, partitions, right-hand sides.

This module is the only code shared by the CUDA path and the FP64 oracle. It holds
none of the preconditioner's or the solver's arithmetic: it builds a sparse matrix
A (CSR, int32 indices, float64 values, sorted columns, diagonal stored), a
partition ``part[n]`` of the unknowns into ``p`` subdomains, and a right-hand side
``b = A @ x_true`` (scipy's CSR product) from a seeded ``x_true ~ U(-1, 1)``.

The model problems follow the paper's experiments (Sec. 4: Poisson / anisotropic
diffusion and 3D convection-diffusion on structured grids, Eq. (lap) and
Eq. (difconv)); homogeneous Dirichlet nodes are eliminated, only interior grid
nodes are unknowns, and no h^2 scaling is applied (b = A x_true makes the scale
irrelevant). Natural (lexicographic, x fastest) node numbering throughout.

Random streams: ``x_true`` comes from ``numpy.random.default_rng(seed)``; matrix
entries of the random nonsymmetric problem from ``default_rng([seed, 1])``; random
cut planes of the 3D partition from ``default_rng([seed, 2])``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class Problem:
    """A linear system A x = b with a subdomain partition (all host numpy arrays)."""
    name: str
    n: int
    rowptr: np.ndarray          # int32 [n+1]
    colind: np.ndarray          # int32 [nnz]
    val: np.ndarray             # float64 [nnz]
    part: np.ndarray            # int32 [n], values in [0, p)
    p: int
    x_true: np.ndarray          # float64 [n]
    b: np.ndarray               # float64 [n]
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.colind, self.rowptr), shape=(self.n, self.n))


# --------------------------------------------------------------------------------------
# stencil assembly


def _stencil_csr(dims, offsets, coeffs):
    """CSR of a constant-coefficient stencil on a box grid with eliminated Dirichlet
    boundary. ``dims`` = (nx, ny[, nz]); ``offsets`` = list of integer tuples of the
    same rank; ``coeffs`` = matching coefficients. Node id = x + nx*(y + ny*z)."""
    dims = tuple(int(d) for d in dims)
    rank = len(dims)
    n = int(np.prod(dims))
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    lin = [sum(o[k] * strides[k] for k in range(rank)) for o in offsets]
    order = np.argsort(lin, kind="stable")          # ascending column offset = sorted columns
    offsets = [offsets[i] for i in order]
    coeffs = [coeffs[i] for i in order]
    lin = [lin[i] for i in order]
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx
    for d in dims:
        coords.append(rem % d)
        rem = rem // d
    noff = len(offsets)
    mask = np.ones((n, noff), dtype=bool)
    for j, o in enumerate(offsets):
        for k in range(rank):
            if o[k] != 0:
                c = coords[k] + o[k]
                mask[:, j] &= (c >= 0) & (c < dims[k])
    cols = idx[:, None] + np.asarray(lin, dtype=np.int64)[None, :]
    vals = np.broadcast_to(np.asarray(coeffs, dtype=np.float64)[None, :], (n, noff))
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colind = cols[mask].astype(np.int32)
    val = np.ascontiguousarray(vals[mask], dtype=np.float64)
    return n, rowptr.astype(np.int32), colind, val


def poisson2d_5pt(nx: int, ny: int):
    """2D Poisson, 5-point: centre 4, four neighbours -1 (Eq. (lap), 2D)."""
    offs = [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)]
    return _stencil_csr((nx, ny), offs, [4.0, -1.0, -1.0, -1.0, -1.0])


def aniso2d_9pt_coeffs(eps: float, theta: float):
    """Coefficients of -div(K grad u), K = R(theta) diag(1, eps) R(theta)^T, on the
    9-point stencil: a = cos^2+eps sin^2, c = sin^2+eps cos^2, b = (1-eps) cos sin.
    Returns dict offset -> coefficient. The cross term uses the centred difference
    u_xy ~ (u_NE - u_NW - u_SE + u_SW) / 4."""
    ct, st = math.cos(theta), math.sin(theta)
    a = ct * ct + eps * st * st
    c = st * st + eps * ct * ct
    b = (1.0 - eps) * ct * st
    return {
        (0, 0): 2.0 * a + 2.0 * c,
        (-1, 0): -a, (1, 0): -a,
        (0, -1): -c, (0, 1): -c,
        (1, 1): -b / 2.0, (-1, -1): -b / 2.0,
        (-1, 1): b / 2.0, (1, -1): b / 2.0,
    }


def aniso2d_9pt(nx: int, ny: int, eps: float, theta: float):
    co = aniso2d_9pt_coeffs(eps, theta)
    offs = list(co.keys())
    return _stencil_csr((nx, ny), offs, [co[o] for o in offs])


def aniso3d_7pt(nx: int, ny: int, nz: int, cx: float, cy: float, cz: float):
    """3D anisotropic diffusion, 7-point: centre 2(cx+cy+cz), neighbours -c_d."""
    offs = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    co = [2.0 * (cx + cy + cz), -cx, -cx, -cy, -cy, -cz, -cz]
    return _stencil_csr((nx, ny, nz), offs, co)


def convdiff3d_upwind(m: int, pe: float):
    """-Lap u + beta . grad u on [0,1]^3, beta = (pe, pe, pe)/sqrt(3), h = 1/(m+1),
    first-order upwind convection, scaled by h^2 (Eq. (difconv)). Per direction d:
    lower neighbour -1 - beta_d h, upper neighbour -1, centre +2 + beta_d h."""
    h = 1.0 / (m + 1)
    bh = pe / math.sqrt(3.0) * h
    offs = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    co = [6.0 + 3.0 * bh, -1.0 - bh, -1.0, -1.0 - bh, -1.0, -1.0 - bh, -1.0]
    return _stencil_csr((m, m, m), offs, co)


def random_nonsym(n: int, mean_k: float, sigma: float, rng: np.random.Generator,
                  diag_factor: float = 1.1):
    """Random nonsymmetric sparse matrix: row i has k_i = max(1, round(LogNormal(mu,
    sigma))) distinct uniform random off-diagonal columns, mu = ln(mean_k) - sigma^2/2
    (so the distribution mean is mean_k), N(0,1) values, and a_ii = diag_factor *
    sum |off-diagonal of row i|."""
    mu = math.log(mean_k) - 0.5 * sigma * sigma
    k = np.maximum(1, np.rint(rng.lognormal(mu, sigma, size=n))).astype(np.int64)
    k = np.minimum(k, n - 1)
    rows = np.repeat(np.arange(n, dtype=np.int64), k)
    cols = rng.integers(0, n - 1, size=rows.size)
    cols = cols + (cols >= rows)
    # redraw duplicates within a row until all columns of each row are distinct
    for _ in range(100):
        key = rows * n + cols
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.zeros(ks.size, dtype=bool)
        dup[1:] = ks[1:] == ks[:-1]
        if not dup.any():
            break
        bad = order[dup]
        c = rng.integers(0, n - 1, size=bad.size)
        cols[bad] = c + (c >= rows[bad])
    else:  # pragma: no cover
        raise RuntimeError("could not draw distinct columns")
    offv = rng.standard_normal(rows.size)
    absum = np.bincount(rows, weights=np.abs(offv), minlength=n)
    diag = diag_factor * absum
    allr = np.concatenate([rows, np.arange(n, dtype=np.int64)])
    allc = np.concatenate([cols, np.arange(n, dtype=np.int64)])
    allv = np.concatenate([offv, diag])
    order = np.lexsort((allc, allr))
    allr, allc, allv = allr[order], allc[order], allv[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(allr, minlength=n), out=rowptr[1:])
    return n, rowptr.astype(np.int32), allc.astype(np.int32), np.ascontiguousarray(allv)


def tridiag(n: int, lo: float, d: float, up: float):
    """Constant tridiagonal matrix (a 1D three-point stencil)."""
    return _stencil_csr((n,), [(-1,), (0,), (1,)], [lo, d, up])


# --------------------------------------------------------------------------------------
# partitions


def box_partition(dims, boxes):
    """Geometric partition of a box grid into prod(boxes) equal-as-possible boxes.
    part = bx + Bx*(by + By*bz), bx = x * Bx // nx along each axis."""
    dims = tuple(dims)
    n = int(np.prod(dims))
    idx = np.arange(n, dtype=np.int64)
    part = np.zeros(n, dtype=np.int64)
    mult = 1
    rem = idx
    for d, b in zip(dims, boxes):
        c = rem % d
        rem = rem // d
        part += (c * b // d) * mult
        mult *= b
    return part.astype(np.int32), int(mult)


def cut_partition_3d(dims, ncuts, rng: np.random.Generator):
    """Uneven 3D box partition from random cut planes: along axis a, ncuts[a] planes
    drawn without replacement from {2, ..., dims[a]-2} and sorted; a node with
    coordinate c lies in slab #(planes <= c). part = sx + Sx*(sy + Sy*sz)."""
    dims = tuple(dims)
    n = int(np.prod(dims))
    idx = np.arange(n, dtype=np.int64)
    part = np.zeros(n, dtype=np.int64)
    mult = 1
    rem = idx
    cuts = []
    for d, k in zip(dims, ncuts):
        planes = np.sort(rng.choice(np.arange(2, d - 1), size=k, replace=False))
        cuts.append(planes.tolist())
        c = rem % d
        rem = rem // d
        part += np.searchsorted(planes, c, side="right") * mult
        mult *= (k + 1)
    return part.astype(np.int32), int(mult), cuts


def contiguous_partition(n: int, p: int):
    """p contiguous row blocks: part[i] = i * p // n."""
    return (np.arange(n, dtype=np.int64) * p // n).astype(np.int32), p


# --------------------------------------------------------------------------------------
# right-hand side


def make_rhs(n, rowptr, colind, val, seed: int):
    """x_true ~ U(-1, 1) from default_rng(seed); b = A x_true (scipy CSR product)."""
    rng = np.random.default_rng(seed)
    x_true = rng.uniform(-1.0, 1.0, size=n)
    A = sp.csr_matrix((val, colind, rowptr), shape=(n, n))
    b = np.ascontiguousarray(A @ x_true, dtype=np.float64)
    return x_true, b


def _problem(name, mat, part_p, seed, **meta):
    n, rowptr, colind, val = mat
    part, p = part_p[0], part_p[1]
    x_true, b = make_rhs(n, rowptr, colind, val, seed)
    return Problem(name=name, n=n, rowptr=rowptr, colind=colind, val=val,
                   part=part, p=p, x_true=x_true, b=b, meta=meta)


# --------------------------------------------------------------------------------------
# named workloads


def poisson2d_boxes(side: int, boxes: int, seed: int = 0) -> Problem:
    """2D 5-point Poisson on side x side, boxes x boxes geometric subdomains."""
    return _problem(f"poisson2d_{side}_p{boxes*boxes}", poisson2d_5pt(side, side),
                    box_partition((side, side), (boxes, boxes)), seed,
                    grid=(side, side), boxes=(boxes, boxes))


def aniso2d_boxes(side: int, boxes: int, eps: float = 1e-3, theta: float = math.pi / 4,
                  seed: int = 0) -> Problem:
    """2D rotated anisotropic diffusion, 9-point, boxes x boxes subdomains."""
    return _problem(f"aniso2d_{side}_p{boxes*boxes}", aniso2d_9pt(side, side, eps, theta),
                    box_partition((side, side), (boxes, boxes)), seed,
                    grid=(side, side), boxes=(boxes, boxes), eps=eps, theta=theta)


def aniso3d_cuts(side: int, ncuts=(7, 7, 3), coef=(1.0, 1.0, 1e-3), seed: int = 0) -> Problem:
    """3D anisotropic 7-point diffusion with uneven random-cut-plane subdomains."""
    rng = np.random.default_rng([seed, 2])
    part, p, cuts = cut_partition_3d((side, side, side), ncuts, rng)
    return _problem(f"aniso3d_{side}_p{p}", aniso3d_7pt(side, side, side, *coef), (part, p),
                    seed, grid=(side, side, side), cuts=cuts, coef=coef)


def aniso3d_boxes(side: int, boxes: int, coef=(1.0, 1.0, 1e-3), seed: int = 0) -> Problem:
    return _problem(f"aniso3d_{side}_p{boxes**3}", aniso3d_7pt(side, side, side, *coef),
                    box_partition((side,) * 3, (boxes,) * 3), seed,
                    grid=(side,) * 3, coef=coef)


def randsparse(n: int, p: int, mean_k: float = 12.0, sigma: float = 0.6, seed: int = 0) -> Problem:
    """Random nonsymmetric sparse, contiguous row-block subdomains."""
    rng = np.random.default_rng([seed, 1])
    return _problem(f"randsparse_{n}_p{p}", random_nonsym(n, mean_k, sigma, rng),
                    contiguous_partition(n, p), seed, mean_k=mean_k, sigma=sigma)


def convdiff3d_boxes(side: int, boxes: int, pe: float = 50.0, seed: int = 0) -> Problem:
    """3D upwind convection-diffusion, boxes^3 subdomains."""
    return _problem(f"convdiff3d_{side}_p{boxes**3}", convdiff3d_upwind(side, pe),
                    box_partition((side,) * 3, (boxes,) * 3), seed,
                    grid=(side,) * 3, pe=pe)


#: The named workloads at their full sizes (problem, grid or size, subdomains in the name).
WORKLOADS = {
    "poisson2d_64_p4": dict(fn="poisson2d_boxes", side=64, boxes=2),
    "aniso2d_1024_p64": dict(fn="aniso2d_boxes", side=1024, boxes=8),
    "aniso3d_cuts_128_p256": dict(fn="aniso3d_cuts", side=128),
    "randsparse_500k_p64": dict(fn="randsparse", n=500_000, p=64),
    "convdiff3d_96_p64": dict(fn="convdiff3d_boxes", side=96, boxes=4),
}

#: Solver options per workload family (variant, factors, precision, restart).
WORKLOAD_SOLVER = {
    "poisson2d_64_p4": dict(variant="bj", factor_B="ilu0", factor_S="ilu0", prec="fp64", restart=30),
    "aniso2d_1024_p64": dict(variant="schur", factor_B="ilu0", factor_S="milu0", prec="fp32", restart=50),
    "aniso3d_cuts_128_p256": dict(variant="schur", factor_B="ilut", factor_S="milu0", prec="fp32", restart=50,
                                  ilut_tau=1e-3, ilut_p=10),
    "randsparse_500k_p64": dict(variant="schur", factor_B="ilu0", factor_S="milu0", prec="fp32", restart=50),
    "convdiff3d_96_p64": dict(variant="schur", factor_B="ilu0", factor_S="milu0", prec="fp32", restart=50),
}


def make_workload(key: str, seed: int = 0, **override) -> Problem:
    """Build one of the named workloads; keyword overrides shrink it for tests."""
    spec = dict(WORKLOADS[key])
    spec.update(override)
    fn = globals()[spec.pop("fn")]
    return fn(seed=seed, **spec)


# ---------------------------------------------------------------------------------------
# serving trace: a stream of solve requests with Poisson arrivals


@dataclass
class RequestSpec:
    """One request of a serving trace: which matrix (repeats share `key`), which
    right-hand side, and when it arrives (seconds after the trace starts)."""
    rid: int
    arrival: float
    key: str
    kind: str          # "2d" (9-point rotated anisotropic) or "3d" (7-point anisotropic)
    side: int
    eps: float
    theta: float
    boxes: int         # subdomain boxes per axis
    rhs_seed: int


def serving_trace(n_requests: int = 2000, rate: float = 200.0, repeat: float = 0.3, seed: int = 0):
    """Requests for the serving workload: inter-arrival times Exp(1 / rate); half 2D
    9-point rotated anisotropic problems (side log-uniform in [32, 512]), half 3D 7-point
    anisotropic (side log-uniform in [16, 96], coefficients (1, 1, eps)); eps log-uniform
    in [1e-4, 1], theta uniform in [0, pi) (2D only); subdomain boxes of about 64^2 / 16^3
    nodes; a fraction `repeat` of the requests reuse an earlier request's matrix with a
    new right-hand side."""
    rng = np.random.default_rng([seed, 5])
    t = 0.0
    out = []
    for i in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        if out and rng.random() < repeat:
            src = out[int(rng.integers(len(out)))]
            out.append(RequestSpec(i, t, src.key, src.kind, src.side, src.eps, src.theta, src.boxes,
                                   int(rng.integers(1 << 30))))
            continue
        eps = float(10.0 ** rng.uniform(-4.0, 0.0))
        if rng.random() < 0.5:
            side = int(round(2.0 ** rng.uniform(5.0, 9.0)))
            theta = float(rng.uniform(0.0, math.pi))
            kind, boxes = "2d", max(1, side // 64)
        else:
            side = int(round(2.0 ** rng.uniform(4.0, math.log2(96.0))))
            theta = 0.0
            kind, boxes = "3d", max(1, side // 16)
        out.append(RequestSpec(i, t, f"{kind}-{side}-{eps:.6g}-{theta:.6g}", kind, side, eps, theta, boxes,
                               int(rng.integers(1 << 30))))
    return out


def problem_of_request(spec: RequestSpec) -> Problem:
    """The matrix and partition of a request, with its own right-hand side."""
    if spec.kind == "2d":
        return aniso2d_boxes(spec.side, spec.boxes, eps=spec.eps, theta=spec.theta, seed=spec.rhs_seed)
    return aniso3d_boxes(spec.side, spec.boxes, coef=(1.0, 1.0, spec.eps), seed=spec.rhs_seed)
