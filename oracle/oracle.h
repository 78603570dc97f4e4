/*
 * oracle.h -- plain FP64 CPU oracle of the two-level ILU domain-decomposition
 * preconditioner inside restarted flexible GMRES.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this library. It shares no code with the CUDA path: no
 * kernels, headers, helpers or tables. It is written for clarity, sequentially,
 * in the order the paper states each step; it is deliberately not optimised.
 *
 * Every function follows one passage of the paper (Xu, Li, Osei-Kuffuor,
 * "A Two-level GPU-Accelerated Incomplete LU Preconditioner for General Sparse
 * Linear Systems"); the passage is cited beside it in oracle.c.
 *
 * Conventions: CSR with 0-based int32 indices, columns sorted and unique in each
 * row, the diagonal stored; all floating point in IEEE double, compiled without
 * floating-point contraction so the results do not depend on the host's FMA.
 */
#ifndef ORC_ORACLE_H
#define ORC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes (same meaning as the library's; defined separately here) */
#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_CSR 2
#define ORC_ERR_OOM 3
#define ORC_ERR_ZERO_PIVOT 4
#define ORC_ERR_NOT_CONVERGED 5

/* factor kinds */
#define ORC_ILU0 0
#define ORC_MILU0 1
#define ORC_ILUT 2
#define ORC_EXACT 3   /* full LU without dropping (ILUT with tau = 0, p = inf); pins only */
#define ORC_PMILU0 4  /* factor_S of SCHUR: partial ILU(0) of A_i (interior pivots, plain
                         dropping), then MILU(0) of the Schur complement it leaves (Sec. 3.2) */

/* variants and forms */
#define ORC_BJ 0
#define ORC_SCHUR 1
#define ORC_RAP 2     /* two-level multiplicative (Algorithm "Two-level multiplicative solve") */
#define ORC_FORM_AUTO 0
#define ORC_FORM_WZ 1
#define ORC_FORM_EF 2
/* local order of each group of a subdomain (Sec. 3.1) */
#define ORC_ORDER_NATURAL 0   /* ascending original index */
#define ORC_ORDER_RCM 1       /* reverse Cuthill-McKee of the group's graph */
#define ORC_ORDER_COLOR 2     /* greedy multicolouring of the group's graph, colour classes
                                 one after the other (Sec. 3.1: fewer levels) */

typedef struct orc_opts {
    int variant;        /* ORC_BJ, ORC_SCHUR or ORC_RAP */
    int factor_B;       /* factor of the interior block (BJ: of the whole local block;
                           RAP: of the whole local block, the smoother) */
    int factor_S;       /* factor whose (2,2) blocks precondition the Schur system
                           (RAP: also the factor that gives R and P) */
    int form;           /* ORC_FORM_*: W/Z (one L_B and one U_B solve) or E/F */
    double ilut_tau;    /* ILUT relative drop tolerance */
    int ilut_p;         /* ILUT: entries kept per row in each of the L and U parts */
    int inner_iters;    /* GMRES steps on the preconditioned Schur system */
    double pivot_eps;   /* small-pivot perturbation, relative to the row's max |a_ij| */
    int local_order;    /* ORC_ORDER_*: order inside each group. Groups: block Jacobi, the
                           whole subdomain (no interior / interface split, Sec. 2.1); the
                           two-level variants, the interior and the interface nodes of each
                           subdomain (Sec. 2.2.1) */
    int fill_level;     /* k >= 0: ILU0 / MILU0 become ILU(k) / MILU(k) (Sec. 4.2-4.4): each
                           local block is stored in its level-k fill pattern, explicit zeros
                           at the fill positions; needs factor_B, factor_S in {ILU0, MILU0} */
    int l1_block;       /* block Jacobi only: 1 = l1-BJ (Sec. 4.3), every diagonal entry of A_s
                           increased by the sum of |a_ij| over the columns of other subdomains */
    int store_bf16;     /* 1: every off-diagonal factor entry rounded to bfloat16 (nearest,
                           ties to even, straight from the double), the pivots u_ii kept;
                           the applies then run in double on those values. W/Z form only */
} orc_opts;

/* ---- primitives on one CSR matrix ---- */
int orc_csr_check(int n, const int* rowptr, const int* colind);
void orc_spmv(int n, const int* rowptr, const int* colind, const double* val,
              const double* x, double* y);
/* ILU(0) (milu = 0) or MILU(0) (milu = 1) in the pattern of A; out_val holds the
   combined factor (strict lower = L without its unit diagonal, rest = U).
   Returns ORC_OK or ORC_ERR_ZERO_PIVOT; *npert = number of perturbed pivots. */
int orc_ilu0_csr(int n, const int* rowptr, const int* colind, const double* val,
                 int milu, double pivot_eps, double* out_val, int* npert);
/* ILUT(tau, p); returns an opaque factor, read back with orc_factor_*(). */
void* orc_ilut_csr(int n, const int* rowptr, const int* colind, const double* val,
                   double tau, int p, double pivot_eps, int* status);
int orc_factor_nnz(void* f);
void orc_factor_get(void* f, int* rowptr, int* colind, double* val);
void orc_factor_free(void* f);
/* x = L^{-1} b (unit lower part of the combined factor) or U^{-1} b */
void orc_trsv_lower_unit(int n, const int* rowptr, const int* colind, const double* val,
                         const double* b, double* x);
void orc_trsv_upper(int n, const int* rowptr, const int* colind, const double* val,
                    const double* b, double* x);
/* level sets: lower (lev(i) = 1 + max lev(k), k < i stored) or upper (from the bottom);
   returns the number of levels */
int orc_levels_csr(int n, const int* rowptr, const int* colind, int upper, int* lev);

/* ---- domain decomposition ---- */
int orc_classify(int n, const int* rowptr, const int* colind, const int* part, int p,
                 int* iface);
/* x rounded to the nearest bfloat16 value (8 significant bits, the exponent range of
   IEEE single), ties to even; zero, infinities and NaN unchanged. */
double orc_round_bf16(double x);
/* Reverse Cuthill-McKee order of the symmetrised graph of a square pattern (i ~ j when
   a_ij or a_ji is stored, i != j): order[k] = the node placed k-th. */
int orc_rcm(int n, const int* rowptr, const int* colind, int* order);
/* Greedy multicolouring of the symmetrised graph of a square pattern (i ~ j when a_ij or
   a_ji is stored, i != j): nodes in ascending index take the smallest colour none of their
   already coloured neighbours has. color[i] = the colour of node i; order[k] = the node
   placed k-th when the nodes are listed by (colour, index). Returns the number of colours
   (negative status on error). */
int orc_color(int n, const int* rowptr, const int* colind, int* color, int* order);
/* Level-k fill pattern of ILU(k) of a square CSR matrix with sorted rows and its diagonal
   stored: returns the pattern as a new CSR (values: the matrix's, 0 at fill positions) via
   orc_factor_* (opaque handle); NULL with *status set on error. */
void* orc_iluk_pattern(int n, const int* rowptr, const int* colind, const double* val, int k,
                       int* status);
/* returns n1 (number of interior unknowns) */
int orc_permutation(int n, const int* part, int p, const int* iface, int* perm, int* iperm,
                    int* int_ptr, int* if_ptr);

/* ---- whole preconditioner ---- */
void orc_opts_default(orc_opts* o);
void* orc_setup(int n, const int* rowptr, const int* colind, const double* val,
                const int* part, int p, const orc_opts* o, int* status);
void orc_free(void* h);
/* out[0..7] = n, p, n1, n2, nnz(Coff), npert, nnz(A), nlev_max */
void orc_sizes(void* h, int* out);
void orc_get_perm(void* h, int* perm, int* iperm, int* int_ptr, int* if_ptr, int* iface);
/* which: 0 = L_A, 1 = U_A (whole local blocks), 2 = L_B, 3 = U_B, 4 = L_S, 5 = U_S.
   lev[n] indexed by permuted global row; rows outside the factor get -1.
   Returns the number of levels (max over subdomains). */
int orc_get_levels(void* h, int which, int* lev);
/* local block A_s (local order: interior then interface, ascending original index) */
int orc_local_nnz(void* h, int s);
int orc_local_rows(void* h, int s);
void orc_local_csr(void* h, int s, int* rowptr, int* colind, double* val);
/* combined factor values of A_s in the pattern of A_s: fact 1 = factor_B's factorization
   (ILU0/MILU0 only), fact 2 = factor_S's factorization */
int orc_local_factor(void* h, int s, int fact, double* val);
/* C_off (n2 x n2, interface numbering) */
int orc_coff_nnz(void* h);
void orc_coff_csr(void* h, int* rowptr, int* colind, double* val);
/* dense n2 x n2 (row-major): S = C - E B^{-1} F computed by dense elimination */
int orc_schur_dense(void* h, double* S);
/* dense n2 x n2: blockdiag(L_S U_S) + C_off, the Schur approximation used inside */
int orc_sapprox_dense(void* h, double* S);

/* z = M^{-1} r, r and z in the original ordering */
int orc_apply(void* h, const double* r, double* z);
/* inner Schur solve alone: gp, y in interface numbering (length n2) */
int orc_inner_gmres(void* h, const double* gp, double* y);
/* FGMRES(m), x in = x0, out = solution; hist (optional, length hist_len) receives the
   Givens residual estimate |g_{j+1}| after every Arnoldi step and the true residual
   norm at every restart, tagged by sign: estimates > 0, true residuals < 0. */
int orc_fgmres(void* h, const double* b, double* x, double rtol, int m, int maxit,
               int* iters, double* relres, double* hist, int hist_len, int* hist_used);

#ifdef __cplusplus
}
#endif
#endif
