/*
 * oracle.c -- plain FP64 CPU oracle of the two-level ILU domain-decomposition
 * preconditioner (Xu, Li, Osei-Kuffuor) inside restarted flexible GMRES.
 *
 * TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
 * baseline may load it. It shares no code with the CUDA path.
 *
 * Everything here is sequential and follows the paper's steps in its order:
 *   Sec. 2.2.1  interior / interface classification, interior-first relabelling,
 *               the 2x2 block form (Eq. equ22) and the local blocks (Eq. localA);
 *   Sec. 3.1    ILU(0) in the pattern of the (permuted) local block, with the unit
 *               diagonal of L implicit and L\U stored in the matrix's own pattern;
 *   Sec. 2.3    MILU: the sum of the dropped entries of a row is moved onto its
 *               pivot (Eq. milutithrow, Eq. milutshift);
 *   Sec. 4.1.1  small pivots are perturbed so the factorisation cannot break down;
 *   Sec. 3.2    factor extraction L_B, U_B, L_S, U_S, W = E U_B^{-1}, Z = L_B^{-1} F
 *               (Eq. BILU), the one-L-solve / one-U-solve apply, the block-Jacobi
 *               preconditioned Schur system (Eq. preSS) whose MATVEC is
 *               y + S_i^{-1} sum_j E_ij y_j (Eq. preSMV2), solved by a few GMRES steps;
 *   Algorithm "Additive block ILU solve" (Sec. 2.2.2) for the E/F form;
 *   Algorithm "Block Jacobi ILU on GPU" (Sec. 3.1) for block Jacobi;
 *   Sec. 4.1.1  flexible GMRES(m) outside, because the inner GMRES makes M^{-1}
 *               nonlinear;
 *   Sec. 3.3    the multiplicative two-level variant (RAP) with R and P from MILU(0);
 *   Sec. 3.1    RCM order of the local blocks; Sec. 4.2-4.4 ILU(k) by level of fill;
 *   Sec. 4.3    l1 block Jacobi; Sec. 3.2 MILU(0) of the partial-ILU Schur complement;
 *               bfloat16 storage of the factors (a precision option, not in the paper).
 * Readings where the paper is silent are stated at each function. The test
 * infrastructure pins every function here to facts outside the oracle (the paper's
 * printed counts, closed forms, library routines, brute force).
 */
#include "oracle.h"

#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nr, nc, nnz;
    int* rp;
    int* ci;
    double* v;
} csr_t;

static int csr_init(csr_t* m, int nr, int nc, int nnz) {
    m->nr = nr;
    m->nc = nc;
    m->nnz = nnz;
    m->rp = (int*)calloc((size_t)nr + 1, sizeof(int));
    m->ci = (int*)malloc(((size_t)nnz + 1) * sizeof(int));
    m->v = (double*)malloc(((size_t)nnz + 1) * sizeof(double));
    return (m->rp && m->ci && m->v) ? ORC_OK : ORC_ERR_OOM;
}

static void csr_release(csr_t* m) {
    free(m->rp);
    free(m->ci);
    free(m->v);
    m->rp = NULL;
    m->ci = NULL;
    m->v = NULL;
}

/* ====================================================================================
 * Primitives on one CSR matrix
 * ==================================================================================== */

/* A valid input is square CSR, 0-based, columns strictly increasing in each row, the
   diagonal stored (the ILU pivots live there, Sec. 3.1). */
int orc_csr_check(int n, const int* rp, const int* ci) {
    if (n < 0 || rp[0] != 0) return ORC_ERR_CSR;
    for (int i = 0; i < n; i++) {
        if (rp[i + 1] < rp[i]) return ORC_ERR_CSR;
        int has_diag = 0;
        for (int q = rp[i]; q < rp[i + 1]; q++) {
            if (ci[q] < 0 || ci[q] >= n) return ORC_ERR_CSR;
            if (q > rp[i] && ci[q] <= ci[q - 1]) return ORC_ERR_CSR;
            if (ci[q] == i) has_diag = 1;
        }
        if (!has_diag) return ORC_ERR_CSR;
    }
    return ORC_OK;
}

/* y = A x, each row summed in stored order (Eq. 1-1's A). */
void orc_spmv(int n, const int* rp, const int* ci, const double* v, const double* x,
              double* y) {
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int q = rp[i]; q < rp[i + 1]; q++) s += v[q] * x[ci[q]];
        y[i] = s;
    }
}

static double row_absmax(const int* rp, const double* v, int i) {
    double m = 0.0;
    for (int q = rp[i]; q < rp[i + 1]; q++)
        if (fabs(v[q]) > m) m = fabs(v[q]);
    return m;
}

/* Small-pivot rule (Sec. 4.1.1 says only that small diagonal entries are perturbed;
   the constant is unstated). Reading: if |u_ii| < eps * max_j |a_ij| (the original
   row), u_ii becomes sign(u_ii) * eps * max_j |a_ij| with sign(0) = +1. eps = 0
   disables the rule; a pivot that is still exactly zero is an error. */
static int pivot_rule(double* uii, double rowmax, double eps, int* npert) {
    double thr = eps * rowmax;
    if (eps > 0.0 && fabs(*uii) < thr) {
        *uii = (*uii >= 0.0) ? thr : -thr;
        (*npert)++;
    }
    return (*uii == 0.0) ? ORC_ERR_ZERO_PIVOT : ORC_OK;
}

/* ILU(0) / MILU(0), row-wise IKJ Doolittle in the pattern of A (Sec. 3.1; the L factor
   has a unit diagonal that is not stored). For row i, every stored k < i is taken in
   ascending order: l_ik = w_k / u_kk, then for every stored u_kj with j > k the
   update w_j -= l_ik u_kj is kept if (i,j) is in the pattern of A and dropped
   otherwise. MILU (Sec. 2.3, Eq. milutithrow / milutshift with y = z = 1): the
   dropped entries of row i, H_ij = -l_ik u_kj, are summed into Delta_i and added to
   the pivot, u_ii + Delta_i, so that the row sums of LU equal those of A. */
static int ilu0_factor(int n, const int* rp, const int* ci, const double* a, int milu,
                       int milu_from, double eps, double* f, int* npert) {
    int* pos = (int*)malloc(((size_t)n + 1) * sizeof(int));
    int* dpos = (int*)malloc(((size_t)n + 1) * sizeof(int));
    if (!pos || !dpos) {
        free(pos);
        free(dpos);
        return ORC_ERR_OOM;
    }
    for (int i = 0; i < n; i++) pos[i] = -1;
    for (int i = 0; i < n; i++) {
        dpos[i] = -1;
        for (int q = rp[i]; q < rp[i + 1]; q++)
            if (ci[q] == i) dpos[i] = q;
    }
    memcpy(f, a, (size_t)rp[n] * sizeof(double));
    int st = ORC_OK;
    for (int i = 0; i < n && st == ORC_OK; i++) {
        for (int q = rp[i]; q < rp[i + 1]; q++) pos[ci[q]] = q;
        double delta = 0.0; /* Delta_i = sum of the dropped entries H_ij */
        for (int q = rp[i]; q < rp[i + 1] && ci[q] < i; q++) {
            int k = ci[q];
            f[q] = f[q] / f[dpos[k]];
            double lik = f[q];
            for (int t = dpos[k] + 1; t < rp[k + 1]; t++) {
                int j = ci[t];
                if (pos[j] >= 0)
                    f[pos[j]] -= lik * f[t];
                else if (k >= milu_from) /* only these pivots' drops are compensated */
                    delta -= lik * f[t];
            }
        }
        if (milu) f[dpos[i]] += delta;
        st = pivot_rule(&f[dpos[i]], row_absmax(rp, a, i), eps, npert);
        for (int q = rp[i]; q < rp[i + 1]; q++) pos[ci[q]] = -1;
    }
    free(pos);
    free(dpos);
    return st;
}

int orc_ilu0_csr(int n, const int* rp, const int* ci, const double* val, int milu,
                 double pivot_eps, double* out_val, int* npert) {
    int np = 0;
    int st = ilu0_factor(n, rp, ci, val, milu, 0, pivot_eps, out_val, &np);
    if (npert) *npert = np;
    return st;
}

/* ---- ILUT(tau, p) -----------------------------------------------------------------
   The paper uses ILUT on the CPU (Sec. 4.2) without defining it. Reading: the standard
   dual-threshold ILUT. For row i, t_i = tau * ||a_i,:||_2; IKJ elimination over the
   full working row w with the pivots k < i taken in ascending order, fill allowed;
   after dividing, w_k is dropped (and its update skipped) if |w_k| < t_i; after the
   elimination every off-diagonal w_j with |w_j| < t_i is dropped, then only the p
   largest |w_j| of the L part and the p largest of the U part are kept (ties: larger
   |value| first, then smaller column). The diagonal is always kept and the small-pivot
   rule applies. tau = 0 with p = INT_MAX drops nothing: exact LU without pivoting. */

typedef struct {
    int col;
    double val;
} ent_t;

static int ent_cmp_mag(const void* a, const void* b) {
    const ent_t* x = (const ent_t*)a;
    const ent_t* y = (const ent_t*)b;
    double ax = fabs(x->val), ay = fabs(y->val);
    if (ax > ay) return -1;
    if (ax < ay) return 1;
    return (x->col < y->col) ? -1 : (x->col > y->col);
}

static int ent_cmp_col(const void* a, const void* b) {
    const ent_t* x = (const ent_t*)a;
    const ent_t* y = (const ent_t*)b;
    return (x->col < y->col) ? -1 : (x->col > y->col);
}

static void heap_push(int* h, int* len, int v) {
    int i = (*len)++;
    h[i] = v;
    while (i > 0) {
        int p = (i - 1) / 2;
        if (h[p] <= h[i]) break;
        int t = h[p];
        h[p] = h[i];
        h[i] = t;
        i = p;
    }
}

static int heap_pop(int* h, int* len) {
    int top = h[0];
    h[0] = h[--(*len)];
    int i = 0;
    for (;;) {
        int l = 2 * i + 1, r = l + 1, m = i;
        if (l < *len && h[l] < h[m]) m = l;
        if (r < *len && h[r] < h[m]) m = r;
        if (m == i) break;
        int t = h[m];
        h[m] = h[i];
        h[i] = t;
        i = m;
    }
    return top;
}

typedef struct {
    csr_t f;
    int npert;
} ilut_fact_t;

static int int_cmp(const void* a, const void* b);

/* bfloat16: 1 sign bit, 8 exponent bits (bias 127, like IEEE single), 7 stored significand
   bits. Normal values keep 8 significant bits; below 2^-126 the spacing is 2^-133; at or
   above 2^128 (1 - 2^-9) the value rounds to infinity. nearbyint rounds half to even in
   the default rounding mode. */
double orc_round_bf16(double x) {
    if (x == 0.0 || !isfinite(x)) return x;
    double a = fabs(x), r;
    if (a < ldexp(1.0, -126)) {
        r = ldexp(nearbyint(ldexp(a, 133)), -133);
    } else {
        int e;
        double m = frexp(a, &e);                       /* a = m 2^e, m in [0.5, 1) */
        r = ldexp(nearbyint(ldexp(m, 8)), e - 8);      /* 8 significant bits */
        if (r >= ldexp(1.0, 128)) r = INFINITY;
    }
    return copysign(r, x);
}

/* Level-of-fill pattern of ILU(k) (the paper uses ILU(1) and ILU(2) in Sec. 4.2-4.4 without
   defining them; standard sum rule). Stored entries have level 0. Row i is eliminated with
   its pivots m < i in ascending order, fill included: each entry u_mj (j > m) kept in row m
   gives position (i, j) the level lev(i,m) + lev(m,j) + 1, the smallest such level wins, and
   positions of level <= k are kept. Rows: sorted columns, the diagonal stored. */
static int iluk_symbolic(const csr_t* M, int k, csr_t* out) {
    int n = M->nr, st = ORC_OK;
    int* lev = (int*)malloc(((size_t)n + 1) * sizeof(int));   /* level of (i, j), -1 absent */
    int* cols = (int*)malloc(((size_t)n + 1) * sizeof(int));  /* columns present in row i */
    int* heap = (int*)malloc(((size_t)n + 1) * sizeof(int));  /* pending pivots m < i */
    int* rp = (int*)calloc((size_t)n + 1, sizeof(int));
    int cap = M->nnz + n + 16, nnz = 0;
    int* ci = (int*)malloc((size_t)cap * sizeof(int));
    int* lv = (int*)malloc((size_t)cap * sizeof(int));        /* level of each kept entry */
    int* dg = (int*)malloc(((size_t)n + 1) * sizeof(int));    /* position of each diagonal */
    if (!lev || !cols || !heap || !rp || !ci || !lv || !dg) {
        st = ORC_ERR_OOM;
        goto done;
    }
    for (int j = 0; j < n; j++) lev[j] = -1;
    for (int i = 0; i < n; i++) {
        int nc = 0, hl = 0;
        for (int q = M->rp[i]; q < M->rp[i + 1]; q++) {
            int j = M->ci[q];
            lev[j] = 0;
            cols[nc++] = j;
            if (j < i) heap_push(heap, &hl, j);
        }
        while (hl > 0) {
            int m = heap_pop(heap, &hl);
            int lim = lev[m];
            for (int t = dg[m] + 1; t < rp[m + 1]; t++) {
                int j = ci[t], nl = lim + lv[t] + 1;
                if (nl > k) continue;
                if (lev[j] < 0) {
                    lev[j] = nl;
                    cols[nc++] = j;
                    if (j < i) heap_push(heap, &hl, j);
                } else if (nl < lev[j]) {
                    lev[j] = nl;
                }
            }
        }
        qsort(cols, (size_t)nc, sizeof(int), int_cmp);
        if (nnz + nc > cap) {
            while (nnz + nc > cap) cap *= 2;
            int* c2 = (int*)realloc(ci, (size_t)cap * sizeof(int));
            if (c2) ci = c2;
            int* l2 = (int*)realloc(lv, (size_t)cap * sizeof(int));
            if (l2) lv = l2;
            if (!c2 || !l2) {
                st = ORC_ERR_OOM;
                goto done;
            }
        }
        dg[i] = -1;
        for (int t = 0; t < nc; t++) {
            if (cols[t] == i) dg[i] = nnz;
            ci[nnz] = cols[t];
            lv[nnz++] = lev[cols[t]];
            lev[cols[t]] = -1;
        }
        rp[i + 1] = nnz;
        if (dg[i] < 0) {
            st = ORC_ERR_CSR;
            goto done;
        }
    }
    st = csr_init(out, n, n, nnz);
    if (st) goto done;
    memcpy(out->rp, rp, ((size_t)n + 1) * sizeof(int));
    memcpy(out->ci, ci, (size_t)nnz * sizeof(int));
    for (int i = 0; i < n; i++) { /* A's values, zeros at the fill positions */
        int q = M->rp[i];
        for (int t = rp[i]; t < rp[i + 1]; t++) {
            while (q < M->rp[i + 1] && M->ci[q] < ci[t]) q++;
            out->v[t] = (q < M->rp[i + 1] && M->ci[q] == ci[t]) ? M->v[q] : 0.0;
        }
    }
done:
    free(lev);
    free(cols);
    free(heap);
    free(rp);
    free(ci);
    free(lv);
    free(dg);
    return st;
}

static int ilut_factor(int n, const int* rp, const int* ci, const double* a, double tau,
                       int pkeep, double eps, csr_t* out, int* npert) {
    double* w = (double*)calloc((size_t)n + 1, sizeof(double));
    char* mark = (char*)calloc((size_t)n + 1, 1);
    int* heap = (int*)malloc(((size_t)n + 1) * sizeof(int));
    int* uidx = (int*)malloc(((size_t)n + 1) * sizeof(int));
    int* lkept = (int*)malloc(((size_t)n + 1) * sizeof(int));
    ent_t* tmp = (ent_t*)malloc(((size_t)n + 1) * sizeof(ent_t));
    int* udiag = (int*)malloc(((size_t)n + 1) * sizeof(int)); /* diag position per row */
    int cap = rp[n] > 16 ? 2 * rp[n] : 32;
    int* oci = (int*)malloc((size_t)cap * sizeof(int));
    double* ov = (double*)malloc((size_t)cap * sizeof(double));
    int* orp = (int*)calloc((size_t)n + 1, sizeof(int));
    int st = ORC_OK;
    if (!w || !mark || !heap || !uidx || !lkept || !tmp || !udiag || !oci || !ov || !orp) {
        st = ORC_ERR_OOM;
        goto done;
    }
    int nnz = 0;
    for (int i = 0; i < n && st == ORC_OK; i++) {
        double nrm = 0.0;
        for (int q = rp[i]; q < rp[i + 1]; q++) nrm += a[q] * a[q];
        double ti = tau * sqrt(nrm);
        int hlen = 0, nu = 0, nl = 0;
        w[i] = 0.0;
        mark[i] = 1;
        for (int q = rp[i]; q < rp[i + 1]; q++) {
            int j = ci[q];
            w[j] = a[q];
            if (j == i) continue;
            mark[j] = 1;
            if (j < i)
                heap_push(heap, &hlen, j);
            else
                uidx[nu++] = j;
        }
        while (hlen > 0) {
            int k = heap_pop(heap, &hlen);
            double wk = w[k] / ov[udiag[k]];
            if (fabs(wk) < ti) { /* first dropping rule */
                w[k] = 0.0;
                mark[k] = 0;
                continue;
            }
            w[k] = wk;
            lkept[nl++] = k;
            for (int t = udiag[k] + 1; t < orp[k + 1]; t++) {
                int j = oci[t];
                if (!mark[j]) {
                    mark[j] = 1;
                    w[j] = 0.0;
                    if (j < i)
                        heap_push(heap, &hlen, j);
                    else
                        uidx[nu++] = j;
                }
                w[j] -= wk * ov[t];
            }
        }
        /* second dropping rule, then the p largest of each part */
        int cnt = 0;
        for (int t = 0; t < nl; t++) {
            int j = lkept[t];
            if (fabs(w[j]) >= ti) {
                tmp[cnt].col = j;
                tmp[cnt].val = w[j];
                cnt++;
            }
        }
        qsort(tmp, (size_t)cnt, sizeof(ent_t), ent_cmp_mag);
        int lk = cnt < pkeep ? cnt : pkeep;
        qsort(tmp, (size_t)lk, sizeof(ent_t), ent_cmp_col);
        int ucnt = 0;
        ent_t* ut = tmp + lk;
        for (int t = 0; t < nu; t++) {
            int j = uidx[t];
            if (fabs(w[j]) >= ti) {
                ut[ucnt].col = j;
                ut[ucnt].val = w[j];
                ucnt++;
            }
        }
        qsort(ut, (size_t)ucnt, sizeof(ent_t), ent_cmp_mag);
        int uk = ucnt < pkeep ? ucnt : pkeep;
        qsort(ut, (size_t)uk, sizeof(ent_t), ent_cmp_col);
        double uii = w[i];
        st = pivot_rule(&uii, row_absmax(rp, a, i), eps, npert);
        if (nnz + lk + uk + 1 > cap) {
            int ncap = 2 * cap + lk + uk + 1;
            int* nci = (int*)realloc(oci, (size_t)ncap * sizeof(int));
            double* nv = (double*)realloc(ov, (size_t)ncap * sizeof(double));
            if (!nci || !nv) {
                if (nci) oci = nci;
                if (nv) ov = nv;
                st = ORC_ERR_OOM;
                break;
            }
            oci = nci;
            ov = nv;
            cap = ncap;
        }
        for (int t = 0; t < lk; t++) {
            oci[nnz] = tmp[t].col;
            ov[nnz++] = tmp[t].val;
        }
        udiag[i] = nnz;
        oci[nnz] = i;
        ov[nnz++] = uii;
        for (int t = 0; t < uk; t++) {
            oci[nnz] = ut[t].col;
            ov[nnz++] = ut[t].val;
        }
        orp[i + 1] = nnz;
        /* clear the working row */
        w[i] = 0.0;
        mark[i] = 0;
        for (int t = 0; t < nl; t++) {
            w[lkept[t]] = 0.0;
            mark[lkept[t]] = 0;
        }
        for (int t = 0; t < nu; t++) {
            w[uidx[t]] = 0.0;
            mark[uidx[t]] = 0;
        }
    }
    if (st == ORC_OK) {
        out->nr = n;
        out->nc = n;
        out->nnz = orp[n];
        out->rp = orp;
        out->ci = oci;
        out->v = ov;
        orp = NULL;
        oci = NULL;
        ov = NULL;
    }
done:
    free(w);
    free(mark);
    free(heap);
    free(uidx);
    free(lkept);
    free(tmp);
    free(udiag);
    free(oci);
    free(ov);
    free(orp);
    return st;
}

void* orc_ilut_csr(int n, const int* rp, const int* ci, const double* val, double tau,
                   int p, double pivot_eps, int* status) {
    ilut_fact_t* f = (ilut_fact_t*)calloc(1, sizeof(ilut_fact_t));
    int st = f ? ilut_factor(n, rp, ci, val, tau, p, pivot_eps, &f->f, &f->npert)
               : ORC_ERR_OOM;
    if (status) *status = st;
    if (st != ORC_OK) {
        free(f);
        return NULL;
    }
    return f;
}

void* orc_iluk_pattern(int n, const int* rp, const int* ci, const double* val, int k,
                       int* status) {
    int st = orc_csr_check(n, rp, ci);
    ilut_fact_t* f = NULL;
    if (!st && k < 0) st = ORC_ERR_ARG;
    if (!st) {
        f = (ilut_fact_t*)calloc(1, sizeof(ilut_fact_t));
        if (!f) st = ORC_ERR_OOM;
    }
    if (!st) {
        csr_t M = {n, n, rp[n], (int*)rp, (int*)ci, (double*)val};
        st = iluk_symbolic(&M, k, &f->f);
    }
    if (st && f) {
        csr_release(&f->f);
        free(f);
        f = NULL;
    }
    if (status) *status = st;
    return f;
}

int orc_factor_nnz(void* f) { return ((ilut_fact_t*)f)->f.nnz; }

void orc_factor_get(void* fp, int* rp, int* ci, double* v) {
    ilut_fact_t* f = (ilut_fact_t*)fp;
    memcpy(rp, f->f.rp, ((size_t)f->f.nr + 1) * sizeof(int));
    memcpy(ci, f->f.ci, (size_t)f->f.nnz * sizeof(int));
    memcpy(v, f->f.v, (size_t)f->f.nnz * sizeof(double));
}

void orc_factor_free(void* fp) {
    ilut_fact_t* f = (ilut_fact_t*)fp;
    if (!f) return;
    csr_release(&f->f);
    free(f);
}

/* ---- triangular solves on a row/column window of a combined L\U factor ---------------
   Lower (unit diagonal): x_i = b_i - sum_{c0 <= k < i} l_ik x_k for rows r0..r1-1 in
   increasing order. Upper: x_i = (b_i - sum_{i < j < c1} u_ij x_j) / u_ii for rows
   r1-1..r0. x and b may alias. */
static void lsolve_win(const csr_t* f, int r0, int r1, int c0, const double* b, double* x) {
    for (int i = r0; i < r1; i++) {
        double s = b[i];
        for (int q = f->rp[i]; q < f->rp[i + 1]; q++) {
            int k = f->ci[q];
            if (k >= i) break;
            if (k >= c0) s -= f->v[q] * x[k];
        }
        x[i] = s;
    }
}

static void usolve_win(const csr_t* f, int r0, int r1, int c1, const double* b, double* x) {
    for (int i = r1 - 1; i >= r0; i--) {
        double s = b[i];
        double d = 0.0;
        for (int q = f->rp[i]; q < f->rp[i + 1]; q++) {
            int j = f->ci[q];
            if (j < i) continue;
            if (j == i) {
                d = f->v[q];
                continue;
            }
            if (j < c1) s -= f->v[q] * x[j];
        }
        x[i] = s / d;
    }
}

void orc_trsv_lower_unit(int n, const int* rp, const int* ci, const double* v,
                         const double* b, double* x) {
    csr_t f = {n, n, rp[n], (int*)rp, (int*)ci, (double*)v};
    lsolve_win(&f, 0, n, 0, b, x);
}

void orc_trsv_upper(int n, const int* rp, const int* ci, const double* v, const double* b,
                    double* x) {
    csr_t f = {n, n, rp[n], (int*)rp, (int*)ci, (double*)v};
    usolve_win(&f, 0, n, n, b, x);
}

/* ---- level sets (Sec. 3.1: the level-scheduling analysis) ---------------------------
   Lower: lev(i) = 0 if row i has no stored entry k with c0 <= k < i, else 1 + max lev(k)
   over those. Upper: the same from the bottom over i < j < c1. Returns #levels. */
static int levels_win(const csr_t* f, int r0, int r1, int clo, int chi, int upper,
                      int* lev /* indexed by row */) {
    int nlev = 0;
    if (!upper) {
        for (int i = r0; i < r1; i++) {
            int l = 0;
            for (int q = f->rp[i]; q < f->rp[i + 1]; q++) {
                int k = f->ci[q];
                if (k >= clo && k < i && lev[k] + 1 > l) l = lev[k] + 1;
            }
            lev[i] = l;
            if (l + 1 > nlev) nlev = l + 1;
        }
    } else {
        for (int i = r1 - 1; i >= r0; i--) {
            int l = 0;
            for (int q = f->rp[i]; q < f->rp[i + 1]; q++) {
                int j = f->ci[q];
                if (j > i && j < chi && lev[j] + 1 > l) l = lev[j] + 1;
            }
            lev[i] = l;
            if (l + 1 > nlev) nlev = l + 1;
        }
    }
    return nlev;
}

int orc_levels_csr(int n, const int* rp, const int* ci, int upper, int* lev) {
    csr_t f = {n, n, rp[n], (int*)rp, (int*)ci, NULL};
    return levels_win(&f, 0, n, 0, n, upper, lev);
}

/* ====================================================================================
 * Domain decomposition (Sec. 2.2.1)
 * ==================================================================================== */

/* Interior nodes connect only to nodes of their own subdomain; every other node is an
   exterior (interface) node. Reading for nonsymmetric patterns: node i is interface if
   a stored a_ij OR a stored a_ji couples it to another subdomain (this keeps B, E and F
   block diagonal, Sec. 3.2). Stored explicit zeros count. */
int orc_classify(int n, const int* rp, const int* ci, const int* part, int p, int* iface) {
    for (int i = 0; i < n; i++) {
        if (part[i] < 0 || part[i] >= p) return ORC_ERR_ARG;
        iface[i] = 0;
    }
    for (int i = 0; i < n; i++)
        for (int q = rp[i]; q < rp[i + 1]; q++) {
            int j = ci[q];
            if (part[j] != part[i]) {
                iface[i] = 1;
                iface[j] = 1;
            }
        }
    return ORC_OK;
}

/* Reverse Cuthill-McKee (Sec. 3.1: the local block is put in RCM order before its ILU).
   The graph is that of the pattern made symmetric: i ~ j when a_ij or a_ji is stored and
   i != j; deg(i) = number of distinct neighbours. Cuthill-McKee is a breadth-first search:
   each node taken from the front of the sequence appends its not yet placed neighbours in
   increasing (degree, index). Readings (the paper names the method only): a connected
   component starts at its not yet placed node of smallest (degree, index); the complete
   sequence over all components is reversed at the end. order[k] = node placed k-th. */
typedef struct {
    int deg;
    int idx;
} degidx_t;

static int degidx_cmp(const void* a, const void* b) {
    const degidx_t* x = (const degidx_t*)a;
    const degidx_t* y = (const degidx_t*)b;
    if (x->deg != y->deg) return (x->deg < y->deg) ? -1 : 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

static int int_cmp(const void* a, const void* b) {
    int x = *(const int*)a, y = *(const int*)b;
    return (x < y) ? -1 : (x > y);
}

int orc_rcm(int n, const int* rp, const int* ci, int* order) {
    if (n <= 0) return ORC_OK;
    int st = ORC_OK;
    int* cnt = (int*)calloc((size_t)n + 1, sizeof(int));
    int* deg = (int*)calloc((size_t)n + 1, sizeof(int));
    int* seen = (int*)calloc((size_t)n + 1, sizeof(int));
    int* cm = (int*)malloc(((size_t)n + 1) * sizeof(int));
    degidx_t* start = (degidx_t*)malloc(((size_t)n + 1) * sizeof(degidx_t));
    degidx_t* buf = (degidx_t*)malloc(((size_t)n + 1) * sizeof(degidx_t));
    int* adj = NULL;
    if (!cnt || !deg || !seen || !cm || !start || !buf) {
        st = ORC_ERR_OOM;
        goto done;
    }
    /* adjacency lists of the symmetrised graph: both directions of every stored
       off-diagonal entry, then each list sorted and duplicates removed */
    for (int i = 0; i < n; i++)
        for (int q = rp[i]; q < rp[i + 1]; q++)
            if (ci[q] != i) {
                cnt[i + 1]++;
                cnt[ci[q] + 1]++;
            }
    for (int i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    adj = (int*)malloc(((size_t)cnt[n] + 1) * sizeof(int));
    if (!adj) {
        st = ORC_ERR_OOM;
        goto done;
    }
    for (int i = 0; i < n; i++) deg[i] = cnt[i]; /* fill positions */
    for (int i = 0; i < n; i++)
        for (int q = rp[i]; q < rp[i + 1]; q++)
            if (ci[q] != i) {
                adj[deg[i]++] = ci[q];
                adj[deg[ci[q]]++] = i;
            }
    for (int i = 0; i < n; i++) {
        int a = cnt[i], b = cnt[i + 1], u = a;
        qsort(adj + a, (size_t)(b - a), sizeof(int), int_cmp);
        for (int t = a; t < b; t++)
            if (t == a || adj[t] != adj[t - 1]) adj[u++] = adj[t];
        deg[i] = u - a; /* the distinct neighbours are adj[cnt[i] .. cnt[i] + deg[i]) */
    }
    for (int i = 0; i < n; i++) {
        start[i].deg = deg[i];
        start[i].idx = i;
    }
    qsort(start, (size_t)n, sizeof(degidx_t), degidx_cmp);
    int placed = 0, next_start = 0;
    while (placed < n) {
        while (seen[start[next_start].idx]) next_start++;
        int s = start[next_start].idx;
        seen[s] = 1;
        cm[placed++] = s;
        for (int head = placed - 1; head < placed; head++) {
            int u = cm[head], nb = 0;
            for (int t = cnt[u]; t < cnt[u] + deg[u]; t++) {
                int v = adj[t];
                if (!seen[v]) {
                    seen[v] = 1;
                    buf[nb].deg = deg[v];
                    buf[nb++].idx = v;
                }
            }
            qsort(buf, (size_t)nb, sizeof(degidx_t), degidx_cmp);
            for (int t = 0; t < nb; t++) cm[placed++] = buf[t].idx;
        }
    }
    for (int k = 0; k < n; k++) order[k] = cm[n - 1 - k];
done:
    free(cnt);
    free(deg);
    free(seen);
    free(cm);
    free(start);
    free(buf);
    free(adj);
    return st;
}

/* Sec. 3.1 schedules the triangular solves by levels; listing the nodes of a group colour
   class by colour class, with no edge inside a class, leaves a lower factor in the pattern
   of A one level per colour. The colouring: nodes in ascending index, each taking the
   smallest colour that no neighbour coloured before it has. */
int orc_color(int n, const int* rp, const int* ci, int* color, int* order) {
    if (n <= 0) return 0;
    int* cnt = (int*)calloc((size_t)n + 1, sizeof(int));
    int* pos = (int*)malloc(((size_t)n + 1) * sizeof(int));
    int* used = (int*)malloc(((size_t)n + 1) * sizeof(int));
    int* adj = NULL;
    int ncol = 0;
    if (!cnt || !pos || !used) {
        ncol = ORC_ERR_OOM;
        goto done;
    }
    /* adjacency of the symmetrised graph (duplicates are harmless here) */
    for (int i = 0; i < n; i++)
        for (int q = rp[i]; q < rp[i + 1]; q++)
            if (ci[q] != i) {
                cnt[i + 1]++;
                cnt[ci[q] + 1]++;
            }
    for (int i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    adj = (int*)malloc(((size_t)cnt[n] + 1) * sizeof(int));
    if (!adj) {
        ncol = ORC_ERR_OOM;
        goto done;
    }
    for (int i = 0; i < n; i++) pos[i] = cnt[i];
    for (int i = 0; i < n; i++)
        for (int q = rp[i]; q < rp[i + 1]; q++)
            if (ci[q] != i) {
                adj[pos[i]++] = ci[q];
                adj[pos[ci[q]]++] = i;
            }
    for (int i = 0; i <= n; i++) used[i] = -1;
    for (int i = 0; i < n; i++) {
        /* colours of the neighbours already coloured (index below i) */
        for (int t = cnt[i]; t < cnt[i + 1]; t++)
            if (adj[t] < i) used[color[adj[t]]] = i;
        int c = 0;
        while (used[c] == i) c++;
        color[i] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    /* list by (colour, index): a counting sort, stable in the index */
    {
        int* start = (int*)calloc((size_t)ncol + 1, sizeof(int));
        if (!start) {
            ncol = ORC_ERR_OOM;
            goto done;
        }
        for (int i = 0; i < n; i++) start[color[i] + 1]++;
        for (int c = 0; c < ncol; c++) start[c + 1] += start[c];
        for (int i = 0; i < n; i++) order[start[color[i]]++] = i;
        free(start);
    }
done:
    free(cnt);
    free(pos);
    free(used);
    free(adj);
    return ncol;
}

/* Put the nodes perm[g0 .. g0 + m) of one group in colour order of the graph they induce
   (the pattern of A restricted to the group, with local labels in the current order). */
static int color_group(const csr_t* A, int* perm, int* iperm, int g0, int m, int* lab) {
    if (m <= 1) return ORC_OK;
    int st = ORC_OK;
    int* grp = (int*)malloc((size_t)m * sizeof(int));
    int* srp = (int*)calloc((size_t)m + 1, sizeof(int));
    int* ord = (int*)malloc((size_t)m * sizeof(int));
    int* col = (int*)malloc((size_t)m * sizeof(int));
    int* sci = NULL;
    if (!grp || !srp || !ord || !col) {
        st = ORC_ERR_OOM;
        goto done;
    }
    for (int k = 0; k < m; k++) {
        grp[k] = perm[g0 + k];
        lab[grp[k]] = k;
    }
    for (int k = 0; k < m; k++) {
        int i = grp[k], c = 0;
        for (int q = A->rp[i]; q < A->rp[i + 1]; q++)
            if (lab[A->ci[q]] >= 0) c++;
        srp[k + 1] = srp[k] + c;
    }
    sci = (int*)malloc(((size_t)srp[m] + 1) * sizeof(int));
    if (!sci) {
        st = ORC_ERR_OOM;
        goto done;
    }
    for (int k = 0, at = 0; k < m; k++) {
        int i = grp[k];
        for (int q = A->rp[i]; q < A->rp[i + 1]; q++)
            if (lab[A->ci[q]] >= 0) sci[at++] = lab[A->ci[q]];
    }
    if (orc_color(m, srp, sci, col, ord) < 0) {
        st = ORC_ERR_OOM;
        goto done;
    }
    for (int k = 0; k < m; k++) {
        perm[g0 + k] = grp[ord[k]];
        iperm[grp[ord[k]]] = g0 + k;
    }
done:
    if (grp)
        for (int k = 0; k < m; k++) lab[grp[k]] = -1;
    free(grp);
    free(srp);
    free(ord);
    free(col);
    free(sci);
    return st;
}

/* Put the nodes perm[g0 .. g0 + m) of one group in RCM order of the graph they induce
   (the pattern of A restricted to the group, with local labels in the current order). */
static int rcm_group(const csr_t* A, int* perm, int* iperm, int g0, int m, int* lab) {
    if (m <= 1) return ORC_OK;
    int st = ORC_OK;
    int* grp = (int*)malloc((size_t)m * sizeof(int));
    int* srp = (int*)calloc((size_t)m + 1, sizeof(int));
    int* ord = (int*)malloc((size_t)m * sizeof(int));
    int* sci = NULL;
    if (!grp || !srp || !ord) {
        st = ORC_ERR_OOM;
        goto done;
    }
    for (int k = 0; k < m; k++) {
        grp[k] = perm[g0 + k];
        lab[grp[k]] = k;
    }
    for (int k = 0; k < m; k++) {
        int i = grp[k], c = 0;
        for (int q = A->rp[i]; q < A->rp[i + 1]; q++)
            if (lab[A->ci[q]] >= 0) c++;
        srp[k + 1] = srp[k] + c;
    }
    sci = (int*)malloc(((size_t)srp[m] + 1) * sizeof(int));
    if (!sci) {
        st = ORC_ERR_OOM;
        goto done;
    }
    for (int k = 0, at = 0; k < m; k++) {
        int i = grp[k];
        for (int q = A->rp[i]; q < A->rp[i + 1]; q++)
            if (lab[A->ci[q]] >= 0) sci[at++] = lab[A->ci[q]];
    }
    st = orc_rcm(m, srp, sci, ord);
    if (!st)
        for (int k = 0; k < m; k++) {
            perm[g0 + k] = grp[ord[k]];
            iperm[grp[ord[k]]] = g0 + k;
        }
done:
    if (grp)
        for (int k = 0; k < m; k++) lab[grp[k]] = -1;
    free(grp);
    free(srp);
    free(ord);
    free(sci);
    return st;
}

/* Interior-first relabelling (Fig. DD, Eq. equ22): the new order lists the interior
   nodes grouped by subdomain, then the interface nodes grouped by subdomain, each group
   in ascending original index. perm[new] = old, iperm[old] = new; interior nodes of
   subdomain s are new indices [int_ptr[s], int_ptr[s+1]); its interface nodes are
   n1 + [if_ptr[s], if_ptr[s+1]). Returns n1. */
int orc_permutation(int n, const int* part, int p, const int* iface, int* perm, int* iperm,
                    int* int_ptr, int* if_ptr) {
    for (int s = 0; s <= p; s++) {
        int_ptr[s] = 0;
        if_ptr[s] = 0;
    }
    for (int i = 0; i < n; i++) {
        if (iface[i])
            if_ptr[part[i] + 1]++;
        else
            int_ptr[part[i] + 1]++;
    }
    for (int s = 0; s < p; s++) {
        int_ptr[s + 1] += int_ptr[s];
        if_ptr[s + 1] += if_ptr[s];
    }
    int n1 = int_ptr[p];
    int* ni = (int*)malloc(((size_t)p + 1) * sizeof(int));
    int* nf = (int*)malloc(((size_t)p + 1) * sizeof(int));
    for (int s = 0; s < p; s++) {
        ni[s] = int_ptr[s];
        nf[s] = if_ptr[s];
    }
    for (int i = 0; i < n; i++) {
        int s = part[i];
        int g = iface[i] ? n1 + nf[s]++ : ni[s]++;
        perm[g] = i;
        iperm[i] = g;
    }
    free(ni);
    free(nf);
    return n1;
}

/* ====================================================================================
 * The preconditioner object
 * ==================================================================================== */

typedef struct {
    int n, p, n1, n2, nnzA;
    orc_opts o;
    int form; /* resolved for SCHUR: ORC_FORM_WZ or ORC_FORM_EF */
    csr_t A;
    int *part, *iface, *perm, *iperm, *int_ptr, *if_ptr;
    csr_t* Aloc; /* local blocks A_s, local order [interior; interface] (Eq. localA) */
    csr_t* F1;   /* factor of A_s (or of B_s for ILUT): L_B, U_B (and W, Z, BJ factor) */
    csr_t* F2;   /* factor of A_s whose (2,2) blocks give L_S, U_S (may alias F1) */
    int f2_alias;
    csr_t Coff; /* cross-subdomain couplings, interface x interface (Eq. SS off-diagonal) */
    int npert;
    double* wn; /* work vectors of length n */
    double* wn2;
} orc_t;

void orc_opts_default(orc_opts* o) {
    o->variant = ORC_SCHUR;
    o->factor_B = ORC_ILU0;
    o->factor_S = ORC_MILU0;
    o->form = ORC_FORM_AUTO;
    o->ilut_tau = 1e-3;
    o->ilut_p = 10;
    o->inner_iters = 3;
    o->pivot_eps = 1e-8;
    o->local_order = ORC_ORDER_NATURAL;
    o->fill_level = 0;
    o->l1_block = 0;
    o->store_bf16 = 0;
}

static inline int nint_of(const orc_t* h, int s) { return h->int_ptr[s + 1] - h->int_ptr[s]; }
static inline int nif_of(const orc_t* h, int s) { return h->if_ptr[s + 1] - h->if_ptr[s]; }
/* new global index of local row l of subdomain s */
static inline int glob_of(const orc_t* h, int s, int l) {
    int ni = nint_of(h, s);
    return l < ni ? h->int_ptr[s] + l : h->n1 + h->if_ptr[s] + (l - ni);
}

void orc_free(void* hp) {
    orc_t* h = (orc_t*)hp;
    if (!h) return;
    csr_release(&h->A);
    free(h->part);
    free(h->iface);
    free(h->perm);
    free(h->iperm);
    free(h->int_ptr);
    free(h->if_ptr);
    for (int s = 0; s < h->p; s++) {
        if (h->Aloc) csr_release(&h->Aloc[s]);
        if (h->F1) csr_release(&h->F1[s]);
        if (h->F2 && !h->f2_alias) csr_release(&h->F2[s]);
    }
    free(h->Aloc);
    free(h->F1);
    if (!h->f2_alias) free(h->F2);
    csr_release(&h->Coff);
    free(h->wn);
    free(h->wn2);
    free(h);
}

/* factor one local matrix with the requested kind */
/* ni: interior rows of the local block (where the interface rows begin) */
static int factor_kind(const csr_t* M, int kind, const orc_opts* o, int ni, csr_t* out, int* npert) {
    if (kind == ORC_ILU0 || kind == ORC_MILU0 || kind == ORC_PMILU0) {
        int st = csr_init(out, M->nr, M->nc, M->nnz);
        if (st) return st;
        memcpy(out->rp, M->rp, ((size_t)M->nr + 1) * sizeof(int));
        memcpy(out->ci, M->ci, (size_t)M->nnz * sizeof(int));
        /* PMILU0 (Sec. 3.2, partial ILU): in IKJ order the interior pivots come first, so
           eliminating them with plain dropping and the interface pivots with MILU's
           compensation is the partial ILU(0) of A_i followed by MILU(0) of the Schur
           complement it leaves */
        return ilu0_factor(M->nr, M->rp, M->ci, M->v, kind != ORC_ILU0, kind == ORC_PMILU0 ? ni : 0,
                           o->pivot_eps, out->v, npert);
    }
    if (kind == ORC_ILUT)
        return ilut_factor(M->nr, M->rp, M->ci, M->v, o->ilut_tau, o->ilut_p, o->pivot_eps, out,
                           npert);
    if (kind == ORC_EXACT) return ilut_factor(M->nr, M->rp, M->ci, M->v, 0.0, INT_MAX, 0.0, out, npert);
    return ORC_ERR_ARG;
}

/* (1,1) block B_s of a local matrix (rows and columns [0, ni)) */
static int extract_B(const csr_t* M, int ni, csr_t* B) {
    int cnt = 0;
    for (int i = 0; i < ni; i++)
        for (int q = M->rp[i]; q < M->rp[i + 1]; q++)
            if (M->ci[q] < ni) cnt++;
    int st = csr_init(B, ni, ni, cnt);
    if (st) return st;
    cnt = 0;
    for (int i = 0; i < ni; i++) {
        for (int q = M->rp[i]; q < M->rp[i + 1]; q++)
            if (M->ci[q] < ni) {
                B->ci[cnt] = M->ci[q];
                B->v[cnt++] = M->v[q];
            }
        B->rp[i + 1] = cnt;
    }
    return ORC_OK;
}

void* orc_setup(int n, const int* rp, const int* ci, const double* val, const int* part, int p,
                const orc_opts* oin, int* status) {
    int st = ORC_OK;
    orc_t* h = (orc_t*)calloc(1, sizeof(orc_t));
    if (!h) {
        if (status) *status = ORC_ERR_OOM;
        return NULL;
    }
    if (oin)
        h->o = *oin;
    else
        orc_opts_default(&h->o);
    if (n < 0 || p < 1) {
        st = ORC_ERR_ARG;
        goto fail;
    }
    st = orc_csr_check(n, rp, ci);
    if (st) goto fail;
    h->n = n;
    h->p = p;
    h->nnzA = rp[n];
    st = csr_init(&h->A, n, n, rp[n]);
    if (st) goto fail;
    memcpy(h->A.rp, rp, ((size_t)n + 1) * sizeof(int));
    memcpy(h->A.ci, ci, (size_t)rp[n] * sizeof(int));
    memcpy(h->A.v, val, (size_t)rp[n] * sizeof(double));
    h->part = (int*)malloc(((size_t)n + 1) * sizeof(int));
    h->iface = (int*)malloc(((size_t)n + 1) * sizeof(int));
    h->perm = (int*)malloc(((size_t)n + 1) * sizeof(int));
    h->iperm = (int*)malloc(((size_t)n + 1) * sizeof(int));
    h->int_ptr = (int*)malloc(((size_t)p + 1) * sizeof(int));
    h->if_ptr = (int*)malloc(((size_t)p + 1) * sizeof(int));
    h->wn = (double*)calloc((size_t)n + 1, sizeof(double));
    h->wn2 = (double*)calloc((size_t)n + 1, sizeof(double));
    if (!h->part || !h->iface || !h->perm || !h->iperm || !h->int_ptr || !h->if_ptr || !h->wn ||
        !h->wn2) {
        st = ORC_ERR_OOM;
        goto fail;
    }
    memcpy(h->part, part, (size_t)n * sizeof(int));

    /* Sec. 2.2.1: classify and relabel. Block Jacobi (Sec. 2.1, Algorithm "Block Jacobi
       ILU on GPU") factors the whole A_s: it has no interface, every node of a subdomain
       is in one group. */
    if (h->o.local_order != ORC_ORDER_NATURAL && h->o.local_order != ORC_ORDER_RCM &&
        h->o.local_order != ORC_ORDER_COLOR) {
        st = ORC_ERR_ARG;
        goto fail;
    }
    st = orc_classify(n, rp, ci, part, p, h->iface);
    if (st) goto fail;
    if (h->o.variant == ORC_BJ)
        for (int i = 0; i < n; i++) h->iface[i] = 0;
    h->n1 = orc_permutation(n, part, p, h->iface, h->perm, h->iperm, h->int_ptr, h->if_ptr);
    h->n2 = n - h->n1;
    /* Sec. 3.1: RCM order inside each group (BJ: all of A_s; two-level: the interior
       nodes, then the interface nodes, so that A_s keeps its [B F; E C] form) */
    if (h->o.local_order == ORC_ORDER_RCM || h->o.local_order == ORC_ORDER_COLOR) {
        int* lab = (int*)malloc(((size_t)n + 1) * sizeof(int));
        if (!lab) {
            st = ORC_ERR_OOM;
            goto fail;
        }
        for (int i = 0; i < n; i++) lab[i] = -1;
        int (*reorder)(const csr_t*, int*, int*, int, int, int*) =
            (h->o.local_order == ORC_ORDER_RCM) ? rcm_group : color_group;
        for (int s = 0; s < p && !st; s++) {
            st = reorder(&h->A, h->perm, h->iperm, h->int_ptr[s], nint_of(h, s), lab);
            if (!st) st = reorder(&h->A, h->perm, h->iperm, h->n1 + h->if_ptr[s], nif_of(h, s), lab);
        }
        free(lab);
        if (st) goto fail;
    }

    /* Eq. localA: local blocks A_s = [B_s F_s; E_s C_s], and C_off (Eq. SS) */
    h->Aloc = (csr_t*)calloc((size_t)p, sizeof(csr_t));
    h->F1 = (csr_t*)calloc((size_t)p, sizeof(csr_t));
    if (!h->Aloc || !h->F1) {
        st = ORC_ERR_OOM;
        goto fail;
    }
    {
        int coff_cnt = 0; /* couplings of interface rows (none for block Jacobi) */
        for (int i = 0; i < n; i++)
            if (h->iface[i])
                for (int q = rp[i]; q < rp[i + 1]; q++)
                    if (part[ci[q]] != part[i]) coff_cnt++;
        st = csr_init(&h->Coff, h->n2, h->n2, coff_cnt);
        if (st) goto fail;
        int* cnt = (int*)calloc((size_t)p, sizeof(int));
        for (int i = 0; i < n; i++)
            for (int q = rp[i]; q < rp[i + 1]; q++)
                if (part[ci[q]] == part[i]) cnt[part[i]]++;
        for (int s = 0; s < p; s++) {
            int ns = nint_of(h, s) + nif_of(h, s);
            st = csr_init(&h->Aloc[s], ns, ns, cnt[s]);
            if (st) break;
        }
        free(cnt);
        if (st) goto fail;
        ent_t* row = (ent_t*)malloc(((size_t)n + 1) * sizeof(ent_t));
        int* fill = (int*)calloc((size_t)p, sizeof(int));
        int cpos = 0;
        for (int g = 0; g < n; g++) { /* rows in the new order */
            int i = h->perm[g];
            int s = part[i];
            int base_int = h->int_ptr[s], base_if = h->n1 + h->if_ptr[s], ni = nint_of(h, s);
            int len = 0, clen = 0;
            for (int q = rp[i]; q < rp[i + 1]; q++) {
                int j = ci[q];
                int gj = h->iperm[j];
                if (part[j] == s) {
                    row[len].col = gj < h->n1 ? gj - base_int : ni + (gj - base_if);
                    row[len++].val = val[q];
                }
            }
            qsort(row, (size_t)len, sizeof(ent_t), ent_cmp_col);
            csr_t* M = &h->Aloc[s];
            int l = g < h->n1 ? g - base_int : ni + (g - base_if);
            int at = fill[s];
            for (int t = 0; t < len; t++) {
                M->ci[at + t] = row[t].col;
                M->v[at + t] = row[t].val;
            }
            fill[s] += len;
            M->rp[l + 1] = fill[s];
            if (g >= h->n1) {
                for (int q = rp[i]; q < rp[i + 1]; q++) {
                    int j = ci[q];
                    if (part[j] != s) {
                        row[clen].col = h->iperm[j] - h->n1;
                        row[clen++].val = val[q];
                    }
                }
                qsort(row, (size_t)clen, sizeof(ent_t), ent_cmp_col);
                for (int t = 0; t < clen; t++) {
                    h->Coff.ci[cpos] = row[t].col;
                    h->Coff.v[cpos++] = row[t].val;
                }
                h->Coff.rp[g - h->n1 + 1] = cpos;
            }
        }
        free(row);
        free(fill);
    }

    /* l1-BJ (Sec. 4.3): the diagonal of each row of A_s gains the absolute values of the
       row's entries in the off-diagonal blocks; then the usual factorisation of A_s */
    if (h->o.l1_block != 0 && (h->o.l1_block != 1 || h->o.variant != ORC_BJ)) {
        st = ORC_ERR_ARG;
        goto fail;
    }
    for (int g = 0; g < n && h->o.l1_block; g++) {
        int i = h->perm[g], s = part[i], l = g - h->int_ptr[s];
        double add = 0.0;
        for (int q = rp[i]; q < rp[i + 1]; q++)
            if (part[ci[q]] != s) add += fabs(val[q]);
        csr_t* M = &h->Aloc[s];
        for (int q = M->rp[l]; q < M->rp[l + 1]; q++)
            if (M->ci[q] == l) M->v[q] += add;
    }

    /* ILU(k) / MILU(k): each local block stored in its level-k pattern, so that ILU(0) /
       MILU(0) of the stored block is ILU(k) / MILU(k) of A_s */
    if (h->o.fill_level < 0 ||
        (h->o.fill_level > 0 && (h->o.factor_B > ORC_MILU0 ||
                                 (h->o.factor_S > ORC_MILU0 && h->o.factor_S != ORC_PMILU0)))) {
        st = ORC_ERR_ARG;
        goto fail;
    }
    for (int s = 0; s < p && h->o.fill_level > 0; s++) {
        csr_t X;
        st = iluk_symbolic(&h->Aloc[s], h->o.fill_level, &X);
        if (st) goto fail;
        csr_release(&h->Aloc[s]);
        h->Aloc[s] = X;
    }

    /* factorisations (Sec. 3.1 / 3.2 / 2.3 / 3.3); readings:
       RAP (Sec. 3.3, Algorithm "Multiplicative RAP-ILU on GPU"): F1 = factor_B(A_s), the
         smoother applied on the whole local block (ILU(0) by default); F2 = factor_S(A_s)
         (MILU(0) by default) gives L_B, U_B, W, Z for R and P (Eq. wzinmilu) and L_S, U_S
         for the coarse preconditioner (Eq. miluwz3).
       BJ: F1 = factor_B(A_s), applied as U^{-1} L^{-1} on the whole local block.
       SCHUR with factor_B in {ILU0, MILU0, EXACT}: F1 = factor_B(A_s) gives L_B, U_B and
         W = L(2,1), Z = U(1,2) (Eq. BILU); F2 = factor_S(A_s) gives L_S, U_S; if the two
         kinds agree one factorisation serves both.
       SCHUR with factor_B = ILUT: F1 = ILUT(B_s), and the E/F form is used. */
    {
        int kB = h->o.factor_B, kS = h->o.factor_S;
        if (h->o.variant != ORC_BJ && h->o.variant != ORC_SCHUR && h->o.variant != ORC_RAP) {
            st = ORC_ERR_ARG;
            goto fail;
        }
        if (kB < 0 || kB > 3 || kS < 0 || kS > 4 || kS == ORC_ILUT ||
            (h->o.variant == ORC_RAP && kB == ORC_ILUT) ||
            (kS == ORC_PMILU0 && h->o.variant != ORC_SCHUR)) {
            st = ORC_ERR_ARG;
            goto fail;
        }
        int bonly = (h->o.variant == ORC_SCHUR && kB == ORC_ILUT);
        h->form = ORC_FORM_WZ;
        if (h->o.variant == ORC_SCHUR && (bonly || h->o.form == ORC_FORM_EF)) h->form = ORC_FORM_EF;
        for (int s = 0; s < p && !st; s++) {
            if (bonly) {
                csr_t B;
                st = extract_B(&h->Aloc[s], nint_of(h, s), &B);
                if (!st) st = factor_kind(&B, kB, &h->o, nint_of(h, s), &h->F1[s], &h->npert);
                csr_release(&B);
            } else {
                st = factor_kind(&h->Aloc[s], kB, &h->o, nint_of(h, s), &h->F1[s], &h->npert);
            }
        }
        if (st) goto fail;
        if (h->o.variant != ORC_BJ && !(kS == kB && !bonly)) {
            h->F2 = (csr_t*)calloc((size_t)p, sizeof(csr_t));
            if (!h->F2) {
                st = ORC_ERR_OOM;
                goto fail;
            }
            for (int s = 0; s < p && !st; s++)
                st = factor_kind(&h->Aloc[s], kS, &h->o, nint_of(h, s), &h->F2[s], &h->npert);
            if (st) goto fail;
        } else {
            h->F2 = h->F1;
            h->f2_alias = 1;
        }
    }
    /* bfloat16 storage of the factors the applies read: every off-diagonal entry of F1 and
       F2 (L, U, and the W and Z blocks) rounded, the pivots kept */
    if (h->o.store_bf16) {
        if (h->o.store_bf16 != 1 || h->form != ORC_FORM_WZ || h->o.factor_B > ORC_MILU0) {
            st = ORC_ERR_ARG;
            goto fail;
        }
        for (int pass = 0; pass < (h->f2_alias ? 1 : 2); pass++) {
            csr_t* F = pass ? h->F2 : h->F1;
            for (int s = 0; s < p; s++)
                for (int r = 0; r < F[s].nr; r++)
                    for (int q = F[s].rp[r]; q < F[s].rp[r + 1]; q++)
                        if (F[s].ci[q] != r) F[s].v[q] = orc_round_bf16(F[s].v[q]);
        }
    }
    if (status) *status = ORC_OK;
    return h;
fail:
    orc_free(h);
    if (status) *status = st;
    return NULL;
}

void orc_sizes(void* hp, int* out) {
    orc_t* h = (orc_t*)hp;
    int nlev = 0;
    int* lev = (int*)malloc(((size_t)h->n + 1) * sizeof(int));
    for (int w = 0; w < 6; w++) {
        int l = orc_get_levels(hp, w, lev);
        if (l > nlev) nlev = l;
    }
    free(lev);
    out[0] = h->n;
    out[1] = h->p;
    out[2] = h->n1;
    out[3] = h->n2;
    out[4] = h->Coff.nnz;
    out[5] = h->npert;
    out[6] = h->nnzA;
    out[7] = nlev;
}

void orc_get_perm(void* hp, int* perm, int* iperm, int* int_ptr, int* if_ptr, int* iface) {
    orc_t* h = (orc_t*)hp;
    if (perm) memcpy(perm, h->perm, (size_t)h->n * sizeof(int));
    if (iperm) memcpy(iperm, h->iperm, (size_t)h->n * sizeof(int));
    if (int_ptr) memcpy(int_ptr, h->int_ptr, ((size_t)h->p + 1) * sizeof(int));
    if (if_ptr) memcpy(if_ptr, h->if_ptr, ((size_t)h->p + 1) * sizeof(int));
    if (iface) memcpy(iface, h->iface, (size_t)h->n * sizeof(int));
}

int orc_get_levels(void* hp, int which, int* lev) {
    orc_t* h = (orc_t*)hp;
    for (int g = 0; g < h->n; g++) lev[g] = -1;
    int nlev = 0;
    int* loc = NULL;
    for (int s = 0; s < h->p; s++) {
        int ni = nint_of(h, s), ns = ni + nif_of(h, s);
        free(loc);
        loc = (int*)malloc(((size_t)ns + 1) * sizeof(int));
        const csr_t* f;
        int r0, r1, clo, chi, upper = which & 1;
        switch (which) {
            case 0:
            case 1: /* pattern of A_s (ILU(0)/MILU(0) pattern, BJ factor) */
                f = (h->o.variant == ORC_BJ) ? &h->F1[s] : &h->Aloc[s];
                r0 = 0;
                r1 = ns;
                clo = 0;
                chi = ns;
                break;
            case 2:
            case 3:
                f = &h->F1[s];
                r0 = 0;
                r1 = ni;
                clo = 0;
                chi = ni;
                break;
            case 4:
            case 5:
                f = &h->F2[s];
                r0 = ni;
                r1 = ns;
                clo = ni;
                chi = ns;
                break;
            default:
                free(loc);
                return -1;
        }
        int l = levels_win(f, r0, r1, clo, chi, upper, loc);
        if (l > nlev) nlev = l;
        for (int i = r0; i < r1; i++) lev[glob_of(h, s, i)] = loc[i];
    }
    free(loc);
    return nlev;
}

int orc_local_nnz(void* hp, int s) { return ((orc_t*)hp)->Aloc[s].nnz; }
int orc_local_rows(void* hp, int s) { return ((orc_t*)hp)->Aloc[s].nr; }

void orc_local_csr(void* hp, int s, int* rp, int* ci, double* v) {
    orc_t* h = (orc_t*)hp;
    const csr_t* M = &h->Aloc[s];
    if (rp) memcpy(rp, M->rp, ((size_t)M->nr + 1) * sizeof(int));
    if (ci) memcpy(ci, M->ci, (size_t)M->nnz * sizeof(int));
    if (v) memcpy(v, M->v, (size_t)M->nnz * sizeof(double));
}

int orc_local_factor(void* hp, int s, int fact, double* v) {
    orc_t* h = (orc_t*)hp;
    const csr_t* f = (fact == 1) ? &h->F1[s] : &h->F2[s];
    if (f->nnz != h->Aloc[s].nnz || f->nr != h->Aloc[s].nr) return ORC_ERR_ARG;
    memcpy(v, f->v, (size_t)f->nnz * sizeof(double));
    return ORC_OK;
}

int orc_coff_nnz(void* hp) { return ((orc_t*)hp)->Coff.nnz; }

void orc_coff_csr(void* hp, int* rp, int* ci, double* v) {
    orc_t* h = (orc_t*)hp;
    memcpy(rp, h->Coff.rp, ((size_t)h->n2 + 1) * sizeof(int));
    memcpy(ci, h->Coff.ci, (size_t)h->Coff.nnz * sizeof(int));
    memcpy(v, h->Coff.v, (size_t)h->Coff.nnz * sizeof(double));
}

/* ---- dense helpers (small problems only) ---- */

/* Solve M X = R in place (M n x n row-major, R n x m row-major) by Gaussian elimination
   with partial pivoting. */
static int dense_solve(int n, double* M, int m, double* R) {
    for (int k = 0; k < n; k++) {
        int piv = k;
        for (int i = k + 1; i < n; i++)
            if (fabs(M[(size_t)i * n + k]) > fabs(M[(size_t)piv * n + k])) piv = i;
        if (M[(size_t)piv * n + k] == 0.0) return ORC_ERR_ZERO_PIVOT;
        if (piv != k) {
            for (int j = 0; j < n; j++) {
                double t = M[(size_t)k * n + j];
                M[(size_t)k * n + j] = M[(size_t)piv * n + j];
                M[(size_t)piv * n + j] = t;
            }
            for (int j = 0; j < m; j++) {
                double t = R[(size_t)k * m + j];
                R[(size_t)k * m + j] = R[(size_t)piv * m + j];
                R[(size_t)piv * m + j] = t;
            }
        }
        for (int i = k + 1; i < n; i++) {
            double l = M[(size_t)i * n + k] / M[(size_t)k * n + k];
            if (l == 0.0) continue;
            for (int j = k; j < n; j++) M[(size_t)i * n + j] -= l * M[(size_t)k * n + j];
            for (int j = 0; j < m; j++) R[(size_t)i * m + j] -= l * R[(size_t)k * m + j];
        }
    }
    for (int k = n - 1; k >= 0; k--)
        for (int j = 0; j < m; j++) {
            double s = R[(size_t)k * m + j];
            for (int t = k + 1; t < n; t++) s -= M[(size_t)k * n + t] * R[(size_t)t * m + j];
            R[(size_t)k * m + j] = s / M[(size_t)k * n + k];
        }
    return ORC_OK;
}

/* S = C - E B^{-1} F (Eq. blockldu) from the permuted matrix, by dense elimination. */
int orc_schur_dense(void* hp, double* S) {
    orc_t* h = (orc_t*)hp;
    int n = h->n, n1 = h->n1, n2 = h->n2;
    if (n > 4096) return ORC_ERR_ARG;
    double* Ap = (double*)calloc((size_t)n * n, sizeof(double));
    if (!Ap) return ORC_ERR_OOM;
    for (int i = 0; i < n; i++)
        for (int q = h->A.rp[i]; q < h->A.rp[i + 1]; q++)
            Ap[(size_t)h->iperm[i] * n + h->iperm[h->A.ci[q]]] = h->A.v[q];
    double* B = (double*)malloc((size_t)n1 * n1 * sizeof(double) + 8);
    double* X = (double*)malloc((size_t)n1 * n2 * sizeof(double) + 8); /* F, then B^{-1}F */
    for (int i = 0; i < n1; i++) {
        for (int j = 0; j < n1; j++) B[(size_t)i * n1 + j] = Ap[(size_t)i * n + j];
        for (int j = 0; j < n2; j++) X[(size_t)i * n2 + j] = Ap[(size_t)i * n + n1 + j];
    }
    int st = n1 > 0 ? dense_solve(n1, B, n2, X) : ORC_OK;
    if (st == ORC_OK)
        for (int i = 0; i < n2; i++)
            for (int j = 0; j < n2; j++) {
                double s = Ap[(size_t)(n1 + i) * n + n1 + j];
                for (int k = 0; k < n1; k++) s -= Ap[(size_t)(n1 + i) * n + k] * X[(size_t)k * n2 + j];
                S[(size_t)i * n2 + j] = s;
            }
    free(Ap);
    free(B);
    free(X);
    return st;
}

/* blockdiag(L_S U_S) + C_off (Sec. 3.2: the approximate Schur complement whose block-
   Jacobi part is applied through the (2,2) factor blocks). */
int orc_sapprox_dense(void* hp, double* S) {
    orc_t* h = (orc_t*)hp;
    int n2 = h->n2;
    if (n2 > 4096) return ORC_ERR_ARG;
    memset(S, 0, (size_t)n2 * n2 * sizeof(double));
    for (int s = 0; s < h->p; s++) {
        const csr_t* f = &h->F2[s];
        int ni = nint_of(h, s), nf = nif_of(h, s), b = h->if_ptr[s];
        double* L = (double*)calloc((size_t)nf * nf + 1, sizeof(double));
        double* U = (double*)calloc((size_t)nf * nf + 1, sizeof(double));
        for (int i = 0; i < nf; i++) {
            L[(size_t)i * nf + i] = 1.0;
            for (int q = f->rp[ni + i]; q < f->rp[ni + i + 1]; q++) {
                int j = f->ci[q] - ni;
                if (j < 0) continue;
                if (j < i)
                    L[(size_t)i * nf + j] = f->v[q];
                else
                    U[(size_t)i * nf + j] = f->v[q];
            }
        }
        for (int i = 0; i < nf; i++)
            for (int j = 0; j < nf; j++) {
                double t = 0.0;
                for (int k = 0; k < nf; k++) t += L[(size_t)i * nf + k] * U[(size_t)k * nf + j];
                S[(size_t)(b + i) * n2 + b + j] = t;
            }
        free(L);
        free(U);
    }
    for (int i = 0; i < n2; i++)
        for (int q = h->Coff.rp[i]; q < h->Coff.rp[i + 1]; q++)
            S[(size_t)i * n2 + h->Coff.ci[q]] += h->Coff.v[q];
    return ORC_OK;
}

/* ====================================================================================
 * Apply
 * ==================================================================================== */

/* out = blockdiag(U_S^{-1} L_S^{-1}) in on interface vectors (the local Schur inverse
   approximation of Eq. preSS). in and out may alias. */
static void s_solve(orc_t* h, const double* in, double* out) {
    for (int s = 0; s < h->p; s++) {
        int ni = nint_of(h, s), nf = nif_of(h, s), b = h->if_ptr[s];
        if (nf == 0) continue;
        /* local vector indexed by local row: interface rows live at [ni, ni+nf) */
        double* loc = h->wn2; /* scratch, only [ni, ni+nf) used */
        for (int i = 0; i < nf; i++) loc[ni + i] = in[b + i];
        lsolve_win(&h->F2[s], ni, ni + nf, ni, loc, loc);
        usolve_win(&h->F2[s], ni, ni + nf, ni + nf, loc, loc);
        for (int i = 0; i < nf; i++) out[b + i] = loc[ni + i];
    }
}

/* the preconditioned Schur MATVEC of Eq. preSMV2: out = y + S_i^{-1} sum_j E_ij y_j */
static void schur_op(orc_t* h, const double* y, double* out, double* tmp) {
    orc_spmv(h->n2, h->Coff.rp, h->Coff.ci, h->Coff.v, y, tmp);
    s_solve(h, tmp, tmp);
    for (int i = 0; i < h->n2; i++) out[i] = y[i] + tmp[i];
}

static double dot(int n, const double* a, const double* b) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* Givens rotation that annihilates b in (a, b) */
static void givens(double a, double b, double* c, double* s) {
    double d = sqrt(a * a + b * b);
    if (d == 0.0) {
        *c = 1.0;
        *s = 0.0;
    } else {
        *c = a / d;
        *s = b / d;
    }
}

/* ---- two-level multiplicative (Sec. 3.3) ---- */

static void sub_block_mv(const csr_t* M, int r0, int r1, int c0, int c1, double* loc);

/* full vector in the new order <- local vector of subdomain s (and back) */
static void loc_to_new(orc_t* h, int s, const double* loc, double* xn) {
    int ns = nint_of(h, s) + nif_of(h, s);
    for (int l = 0; l < ns; l++) xn[glob_of(h, s, l)] = loc[l];
}
static void new_to_loc(orc_t* h, int s, const double* xn, double* loc) {
    int ns = nint_of(h, s) + nif_of(h, s);
    for (int l = 0; l < ns; l++) loc[l] = xn[glob_of(h, s, l)];
}

/* P v (Eq. wzinmilu): interior rows -U_B^{-1} Z v, interface rows v, with L_B, U_B, Z
   from F2; out is a full vector in the new order */
static void rap_prolong(orc_t* h, const double* v, double* out, double* loc) {
    for (int s = 0; s < h->p; s++) {
        int ni = nint_of(h, s), ns = ni + nif_of(h, s);
        for (int l = 0; l < ni; l++) loc[l] = 0.0;
        for (int l = ni; l < ns; l++) loc[l] = v[h->if_ptr[s] + (l - ni)];
        sub_block_mv(&h->F2[s], 0, ni, ni, ns, loc); /* 0 - Z v */
        usolve_win(&h->F2[s], 0, ni, ni, loc, loc);  /* U_B^{-1} */
        loc_to_new(h, s, loc, out);
    }
}

/* R u (Eq. wzinmilu): interface rows u_G - W L_B^{-1} u_I per subdomain; u a full vector
   in the new order, out an interface vector */
static void rap_restrict(orc_t* h, const double* u, double* out, double* loc) {
    for (int s = 0; s < h->p; s++) {
        int ni = nint_of(h, s), ns = ni + nif_of(h, s);
        new_to_loc(h, s, u, loc);
        lsolve_win(&h->F2[s], 0, ni, 0, loc, loc);   /* L_B^{-1} u_I */
        sub_block_mv(&h->F2[s], ni, ns, 0, ni, loc); /* u_G - W (.) */
        for (int l = ni; l < ns; l++) out[h->if_ptr[s] + (l - ni)] = loc[l];
    }
}

/* A applied to a vector in the new order (A is stored in the original order) */
static void a_new(orc_t* h, const double* xn, double* yn) {
    int n = h->n;
    double* xo = (double*)malloc(((size_t)n + 1) * sizeof(double));
    double* yo = (double*)malloc(((size_t)n + 1) * sizeof(double));
    for (int g = 0; g < n; g++) xo[h->perm[g]] = xn[g];
    orc_spmv(n, h->A.rp, h->A.ci, h->A.v, xo, yo);
    for (int g = 0; g < n; g++) yn[g] = yo[h->perm[g]];
    free(xo);
    free(yo);
}

/* the preconditioned coarse MATVEC: out = (L_S U_S)^{-1} R A P y (Eq. miluwz3: L_S U_S
   preconditions RAP) */
static void rap_op(orc_t* h, const double* y, double* out) {
    int n = h->n;
    double* pv = (double*)malloc(((size_t)n + 1) * sizeof(double));
    double* apv = (double*)malloc(((size_t)n + 1) * sizeof(double));
    double* loc = (double*)malloc(((size_t)n + 1) * sizeof(double));
    rap_prolong(h, y, pv, loc);
    a_new(h, pv, apv);
    rap_restrict(h, apv, out, loc);
    s_solve(h, out, out);
    free(pv);
    free(apv);
    free(loc);
}

/* Inner Schur solve (Sec. 3.2, Eq. preSS; "a small number of GMRES iterations", three
   in Sec. 4.1.1): GMRES with x0 = 0 and exactly k = inner_iters Arnoldi steps (classical
   Gram-Schmidt with one reorthogonalisation, Givens rotations) on
   (I + S^{-1} C_off) y = S^{-1} g', S^{-1} = blockdiag(U_S^{-1} L_S^{-1}). Reading: a
   step whose new Arnoldi norm is <= 1e-14 ||c|| ends the iteration early (lucky
   breakdown). RAP: the same GMRES on the coarse system left-preconditioned like Eq.
   preSS, S^{-1} R A P y = S^{-1} r (reading: the paper gives only "GMRES on S v = r"
   with L_S U_S as its preconditioner, Sec. 3.3). */
int orc_inner_gmres(void* hp, const double* gp, double* y) {
    orc_t* h = (orc_t*)hp;
    int n2 = h->n2, k = h->o.inner_iters;
    if (n2 == 0) return ORC_OK;
    if (k < 1) k = 1;
    double* V = (double*)calloc((size_t)(k + 1) * n2, sizeof(double));
    double* w = (double*)malloc((size_t)n2 * sizeof(double));
    double* tmp = (double*)malloc((size_t)n2 * sizeof(double));
    double* H = (double*)calloc((size_t)(k + 1) * k, sizeof(double)); /* column-major */
    double* hc = (double*)calloc((size_t)k + 1, sizeof(double));
    double* cs = (double*)calloc((size_t)k, sizeof(double));
    double* sn = (double*)calloc((size_t)k, sizeof(double));
    double* g = (double*)calloc((size_t)k + 1, sizeof(double));
    double* t = (double*)calloc((size_t)k, sizeof(double));
    if (!V || !w || !tmp || !H || !hc || !cs || !sn || !g || !t) return ORC_ERR_OOM;
    s_solve(h, gp, V); /* c = S^{-1} g' */
    double beta = sqrt(dot(n2, V, V));
    for (int i = 0; i < n2; i++) y[i] = 0.0;
    int steps = 0;
    if (beta > 0.0) {
        for (int i = 0; i < n2; i++) V[i] /= beta;
        g[0] = beta;
        for (int j = 0; j < k; j++) {
            double* vj = V + (size_t)j * n2;
            if (h->o.variant == ORC_RAP)
                rap_op(h, vj, w); /* coarse system RAP v = r (Algorithm "Two-level multiplicative solve") */
            else
                schur_op(h, vj, w, tmp);
            for (int i = 0; i <= j; i++) hc[i] = 0.0;
            for (int pass = 0; pass < 2; pass++) { /* CGS2 */
                double hh[64];
                double* hp2 = (j + 1 <= 64) ? hh : (double*)malloc(((size_t)j + 1) * sizeof(double));
                for (int i = 0; i <= j; i++) hp2[i] = dot(n2, V + (size_t)i * n2, w);
                for (int i = 0; i <= j; i++) {
                    const double* vi = V + (size_t)i * n2;
                    for (int r = 0; r < n2; r++) w[r] -= hp2[i] * vi[r];
                    hc[i] += hp2[i];
                }
                if (hp2 != hh) free(hp2);
            }
            double hn = sqrt(dot(n2, w, w));
            for (int i = 0; i <= j; i++) H[(size_t)j * (k + 1) + i] = hc[i];
            H[(size_t)j * (k + 1) + j + 1] = hn;
            double* col = H + (size_t)j * (k + 1);
            for (int i = 0; i < j; i++) {
                double a = cs[i] * col[i] + sn[i] * col[i + 1];
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
                col[i] = a;
            }
            givens(col[j], col[j + 1], &cs[j], &sn[j]);
            col[j] = cs[j] * col[j] + sn[j] * col[j + 1];
            col[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            steps = j + 1;
            if (hn <= 1e-14 * beta) break;
            if (j + 1 < k)
                for (int i = 0; i < n2; i++) V[(size_t)(j + 1) * n2 + i] = w[i] / hn;
        }
        for (int i = steps - 1; i >= 0; i--) {
            double s = g[i];
            for (int l = i + 1; l < steps; l++) s -= H[(size_t)l * (k + 1) + i] * t[l];
            t[i] = s / H[(size_t)i * (k + 1) + i];
        }
        for (int i = 0; i < steps; i++)
            for (int r = 0; r < n2; r++) y[r] += t[i] * V[(size_t)i * n2 + r];
    }
    free(V);
    free(w);
    free(tmp);
    free(H);
    free(hc);
    free(cs);
    free(sn);
    free(g);
    free(t);
    return ORC_OK;
}

/* x <- rows [r0,r1) of local vector minus (rows of M restricted to columns [c0,c1))
   times the same local vector: the E, F, W, Z products of Eq. equ22 / Eq. BILU. */
static void sub_block_mv(const csr_t* M, int r0, int r1, int c0, int c1, double* loc) {
    for (int i = r0; i < r1; i++) {
        double s = loc[i];
        for (int q = M->rp[i]; q < M->rp[i + 1]; q++) {
            int j = M->ci[q];
            if (j >= c0 && j < c1) s -= M->v[q] * loc[j];
        }
        loc[i] = s;
    }
}

/* z = M^{-1} r, in the original ordering.
   BJ (Algorithm "Block Jacobi ILU on GPU"): gather, U^{-1} L^{-1} on every local block,
     scatter.
   SCHUR, W/Z form (Sec. 3.2, the one-L-solve / one-U-solve algorithm and Algorithm
     "Additive SCHUR-ILU on GPU"): f' = L_B^{-1} f; g' = g - W f'; y = inner GMRES on
     Eq. preSS; u = U_B^{-1} (f' - Z y).
   SCHUR, E/F form (Algorithm "Additive block ILU solve"): t = U_B^{-1} L_B^{-1} f;
     g' = g - E t; y = inner GMRES; u = U_B^{-1} L_B^{-1} (f - F y). */
int orc_apply(void* hp, const double* r, double* z) {
    orc_t* h = (orc_t*)hp;
    int n = h->n, n1 = h->n1;
    double* xg = h->wn; /* vector in the new (interior-first) order */
    for (int g = 0; g < n; g++) xg[g] = r[h->perm[g]];
    double* loc = (double*)malloc(((size_t)n + 1) * sizeof(double));
    if (!loc) return ORC_ERR_OOM;
    if (h->o.variant == ORC_BJ) {
        for (int s = 0; s < h->p; s++) {
            int ns = nint_of(h, s) + nif_of(h, s);
            for (int l = 0; l < ns; l++) loc[l] = xg[glob_of(h, s, l)];
            lsolve_win(&h->F1[s], 0, ns, 0, loc, loc);
            usolve_win(&h->F1[s], 0, ns, ns, loc, loc);
            for (int l = 0; l < ns; l++) xg[glob_of(h, s, l)] = loc[l];
        }
    } else if (h->o.variant == ORC_RAP) {
        /* Algorithm "Two-level multiplicative solve" in the GPU form of Algorithm
           "Multiplicative RAP-ILU on GPU": x^ = (L_A U_A)^{-1} b blockwise (F1, the
           smoother); r = R (b - A x^); v = inner GMRES on the coarse system; x = x^ + P v */
        int n2 = h->n2;
        double* xh = (double*)malloc(((size_t)n + 1) * sizeof(double));
        double* res = (double*)malloc(((size_t)n + 1) * sizeof(double));
        double* rc = (double*)malloc(((size_t)n2 + 1) * sizeof(double));
        double* v = (double*)malloc(((size_t)n2 + 1) * sizeof(double));
        for (int s = 0; s < h->p; s++) {
            int ns = nint_of(h, s) + nif_of(h, s);
            new_to_loc(h, s, xg, loc);
            lsolve_win(&h->F1[s], 0, ns, 0, loc, loc);
            usolve_win(&h->F1[s], 0, ns, ns, loc, loc);
            loc_to_new(h, s, loc, xh);
        }
        a_new(h, xh, res);
        for (int g = 0; g < n; g++) res[g] = xg[g] - res[g]; /* b - A x^ */
        rap_restrict(h, res, rc, loc);
        orc_inner_gmres(h, rc, v);
        rap_prolong(h, v, res, loc);                          /* P v */
        for (int g = 0; g < n; g++) xg[g] = xh[g] + res[g];
        free(xh);
        free(res);
        free(rc);
        free(v);
    } else {
        double* gp = (double*)malloc(((size_t)h->n2 + 1) * sizeof(double));
        double* y = (double*)malloc(((size_t)h->n2 + 1) * sizeof(double));
        for (int s = 0; s < h->p; s++) {
            int ni = nint_of(h, s), ns = ni + nif_of(h, s);
            for (int l = 0; l < ns; l++) loc[l] = xg[glob_of(h, s, l)];
            lsolve_win(&h->F1[s], 0, ni, 0, loc, loc); /* f' = L_B^{-1} f (or t, E/F) */
            if (h->form == ORC_FORM_WZ) {
                sub_block_mv(&h->F1[s], ni, ns, 0, ni, loc); /* g' = g - W f' */
            } else {
                usolve_win(&h->F1[s], 0, ni, ni, loc, loc);    /* t = U_B^{-1} L_B^{-1} f */
                sub_block_mv(&h->Aloc[s], ni, ns, 0, ni, loc); /* g' = g - E t */
            }
            for (int l = 0; l < ns; l++) xg[glob_of(h, s, l)] = loc[l];
        }
        for (int i = 0; i < h->n2; i++) gp[i] = xg[n1 + i];
        orc_inner_gmres(h, gp, y);
        for (int s = 0; s < h->p; s++) {
            int ni = nint_of(h, s), ns = ni + nif_of(h, s);
            for (int l = 0; l < ni; l++) loc[l] = xg[glob_of(h, s, l)];
            for (int l = ni; l < ns; l++) loc[l] = y[h->if_ptr[s] + (l - ni)];
            if (h->form == ORC_FORM_WZ) {
                sub_block_mv(&h->F1[s], 0, ni, ni, ns, loc); /* f'' = f' - Z y */
                usolve_win(&h->F1[s], 0, ni, ni, loc, loc);  /* u = U_B^{-1} f'' */
            } else {
                for (int l = 0; l < ni; l++) loc[l] = r[h->perm[h->int_ptr[s] + l]];
                sub_block_mv(&h->Aloc[s], 0, ni, ni, ns, loc); /* f - F y */
                lsolve_win(&h->F1[s], 0, ni, 0, loc, loc);
                usolve_win(&h->F1[s], 0, ni, ni, loc, loc);
            }
            for (int l = 0; l < ns; l++) xg[glob_of(h, s, l)] = loc[l];
        }
        free(gp);
        free(y);
    }
    for (int g = 0; g < n; g++) z[h->perm[g]] = xg[g];
    free(loc);
    return ORC_OK;
}

/* ====================================================================================
 * Flexible GMRES(m) (Sec. 4.1.1: FGMRES because the inner GMRES makes M^{-1} vary)
 * ==================================================================================== */

/* Right-preconditioned flexible Arnoldi: z_j = M^{-1} v_j, w = A z_j, classical
   Gram-Schmidt with one reorthogonalisation, h_{j+1,j} = ||w||, Givens rotations. A
   cycle ends when |g_{j+1}| <= rtol ||b|| or j = m; then x += Z_j y and the true
   residual r = b - A x decides convergence (||r|| <= rtol ||b||) or a restart.
   Iterations = Arnoldi steps over all cycles. ||b|| = 0 gives x = 0. */
int orc_fgmres(void* hp, const double* b, double* x, double rtol, int m, int maxit,
               int* iters, double* relres, double* hist, int hist_len, int* hist_used) {
    orc_t* h = (orc_t*)hp;
    int n = h->n;
    int hu = 0;
    if (m < 1) m = 1;
    double bnorm = sqrt(dot(n, b, b));
    if (iters) *iters = 0;
    if (hist_used) *hist_used = 0;
    if (bnorm == 0.0) {
        for (int i = 0; i < n; i++) x[i] = 0.0;
        if (relres) *relres = 0.0;
        return ORC_OK;
    }
    double* V = (double*)malloc((size_t)(m + 1) * n * sizeof(double));
    double* Z = (double*)malloc((size_t)m * n * sizeof(double));
    double* w = (double*)malloc((size_t)n * sizeof(double));
    double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
    double* hc = (double*)calloc((size_t)m + 1, sizeof(double));
    double* cs = (double*)calloc((size_t)m, sizeof(double));
    double* sn = (double*)calloc((size_t)m, sizeof(double));
    double* g = (double*)calloc((size_t)m + 1, sizeof(double));
    double* yv = (double*)calloc((size_t)m, sizeof(double));
    if (!V || !Z || !w || !H || !hc || !cs || !sn || !g || !yv) return ORC_ERR_OOM;
    int total = 0, st = ORC_ERR_NOT_CONVERGED;
    double target = rtol * bnorm;
    /* r = b - A x */
    orc_spmv(n, h->A.rp, h->A.ci, h->A.v, x, w);
    for (int i = 0; i < n; i++) w[i] = b[i] - w[i];
    double beta = sqrt(dot(n, w, w));
    if (hist && hu < hist_len) hist[hu++] = -beta;
    if (beta <= target) st = ORC_OK;
    while (st != ORC_OK && total < maxit) {
        for (int i = 0; i < n; i++) V[i] = w[i] / beta;
        for (int i = 0; i <= m; i++) g[i] = 0.0;
        g[0] = beta;
        int steps = 0;
        for (int j = 0; j < m && total < maxit; j++) {
            double* vj = V + (size_t)j * n;
            double* zj = Z + (size_t)j * n;
            orc_apply(h, vj, zj);
            orc_spmv(n, h->A.rp, h->A.ci, h->A.v, zj, w);
            for (int i = 0; i <= j; i++) hc[i] = 0.0;
            for (int pass = 0; pass < 2; pass++) {
                for (int i = 0; i <= j; i++) yv[i] = dot(n, V + (size_t)i * n, w);
                for (int i = 0; i <= j; i++) {
                    const double* vi = V + (size_t)i * n;
                    for (int r = 0; r < n; r++) w[r] -= yv[i] * vi[r];
                    hc[i] += yv[i];
                }
            }
            double hn = sqrt(dot(n, w, w));
            double* col = H + (size_t)j * (m + 1);
            for (int i = 0; i <= j; i++) col[i] = hc[i];
            col[j + 1] = hn;
            for (int i = 0; i < j; i++) {
                double a = cs[i] * col[i] + sn[i] * col[i + 1];
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
                col[i] = a;
            }
            givens(col[j], col[j + 1], &cs[j], &sn[j]);
            col[j] = cs[j] * col[j] + sn[j] * col[j + 1];
            col[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            steps = j + 1;
            total++;
            if (hist && hu < hist_len) hist[hu++] = fabs(g[j + 1]);
            if (fabs(g[j + 1]) <= target || hn == 0.0) break;
            double* vn = V + (size_t)(j + 1) * n;
            for (int r = 0; r < n; r++) vn[r] = w[r] / hn;
        }
        /* y = R^{-1} g, x += Z y */
        for (int i = steps - 1; i >= 0; i--) {
            double s = g[i];
            for (int l = i + 1; l < steps; l++) s -= H[(size_t)l * (m + 1) + i] * yv[l];
            yv[i] = s / H[(size_t)i * (m + 1) + i];
        }
        for (int i = 0; i < steps; i++) {
            const double* zi = Z + (size_t)i * n;
            for (int r = 0; r < n; r++) x[r] += yv[i] * zi[r];
        }
        orc_spmv(n, h->A.rp, h->A.ci, h->A.v, x, w);
        for (int i = 0; i < n; i++) w[i] = b[i] - w[i];
        beta = sqrt(dot(n, w, w));
        if (hist && hu < hist_len) hist[hu++] = -beta;
        if (beta <= target) st = ORC_OK;
        if (beta == 0.0) break;
    }
    if (iters) *iters = total;
    if (relres) *relres = beta / bnorm;
    if (hist_used) *hist_used = hu;
    free(V);
    free(Z);
    free(w);
    free(H);
    free(hc);
    free(cs);
    free(sn);
    free(g);
    free(yv);
    return st;
}
