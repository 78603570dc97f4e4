/*
 * ilu2l.h -- C ABI of the GB300-native two-level ILU domain-decomposition
 * preconditioner and the flexible GMRES solver around it.
 *
 * Method: Xu, Li, Osei-Kuffuor, "A Two-level GPU-Accelerated Incomplete LU
 * Preconditioner for General Sparse Linear Systems" (arXiv 2303.08881).
 *   - the problem A x = b                                   (Sec. 1, Eq. 1-1)
 *   - p-way domain decomposition, interior nodes first      (Sec. 2.2.1, Eq. equ22)
 *   - block Jacobi ILU                                      (Sec. 2.1, Sec. 3.1)
 *   - additive two-level Schur ILU, E/F form               (Sec. 2.2.2, Algorithm
 *                                                            "Additive block ILU solve")
 *   - the one-L / one-U solve W/Z form and GPU Schur solve  (Sec. 3.2, Eq. preSS,
 *                                                            Eq. preSMV2, Algorithm
 *                                                            "Additive SCHUR-ILU on GPU")
 *   - modified ILU for the Schur factor                     (Sec. 2.3, Sec. 3.3)
 *   - flexible GMRES(m) outside                             (Sec. 4.1.1)
 *
 * All p subdomains live on one GPU and are processed together. Memory layout,
 * ownership and errors are stated per call. Every call returns an ilu_status;
 * nothing is thrown across the ABI. Handles are not thread-safe: one handle is
 * used by one host thread at a time; different handles may run concurrently.
 */
#ifndef ILU2L_H
#define ILU2L_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ILU_OK = 0,
    ILU_ERR_ARG = 1,            /* bad argument: part out of [0,p), NULL, aliasing, bad enum */
    ILU_ERR_CSR = 2,            /* unsorted / duplicate / out-of-range column, missing diagonal */
    ILU_ERR_OOM = 3,            /* a device or host allocation failed */
    ILU_ERR_ZERO_PIVOT = 4,     /* an exactly zero pivot with the perturbation disabled */
    ILU_ERR_NOT_CONVERGED = 5,  /* maxit reached; x holds the last iterate, info is filled */
    ILU_ERR_BREAKDOWN = 6,      /* Arnoldi breakdown without convergence */
    ILU_ERR_TIMEOUT = 7,        /* a bounded device wait gave up */
    ILU_ERR_CUDA = 8,           /* a CUDA runtime call failed */
    ILU_ERR_TOO_LARGE = 9,      /* n or nnz >= 2^31 */
    ILU_ERR_UNSUPPORTED = 10    /* option combination not implemented on the device */
} ilu_status;

/* Square CSR matrix in HOST memory: 0-based int32 indices, columns strictly increasing
   within each row, diagonal stored. The library copies it during ilu_setup. */
typedef struct {
    int32_t n;
    int32_t nnz;
    const int32_t* rowptr; /* n + 1 */
    const int32_t* colind; /* nnz */
    const double* val;     /* nnz */
} ilu_csr;

/* BJ: block Jacobi (Sec. 2.1). SCHUR: additive two-level (Algorithm "Additive SCHUR-ILU on
   GPU"). RAP: multiplicative two-level (Algorithm "Multiplicative RAP-ILU on GPU", Sec. 3.3):
   factor_B is the smoother on each whole local block (ILU(0) or MILU(0)), factor_S gives R,
   P and the coarse preconditioner L_S U_S (MILU(0) in the paper); streamed path only. */
typedef enum { ILU_VARIANT_BJ = 0, ILU_VARIANT_SCHUR = 1, ILU_VARIANT_RAP = 2 } ilu_variant;
/* PMILU0 (factor_S of SCHUR only): the partial ILU(0) of A_i (interior pivots, plain
   dropping) followed by MILU(0) of the Schur complement it leaves (Sec. 3.2, partial ILU),
   computed as one factorisation of A_i whose modification counts only the updates dropped by
   interface pivots. */
typedef enum { ILU_FACT_ILU0 = 0, ILU_FACT_MILU0 = 1, ILU_FACT_ILUT = 2, ILU_FACT_PMILU0 = 3 } ilu_fact;
typedef enum { ILU_FORM_AUTO = 0, ILU_FORM_WZ = 1, ILU_FORM_EF = 2 } ilu_form;
/* FP64, FP32: factors and arithmetic of M^{-1} in that type. BF16_STORE: FP32 arithmetic
   with every off-diagonal factor entry of the level programs stored as bfloat16 (nearest,
   ties to even, from the FP64 factor); pivot inverses and C_off stay FP32. W/Z form on the
   streamed path only (ILU_ERR_UNSUPPORTED with ILUT, the E/F form or kernel_path = 1). */
typedef enum { ILU_PREC_FP64 = 0, ILU_PREC_FP32 = 1, ILU_PREC_BF16_STORE = 2 } ilu_prec;
/* Order inside each group of a subdomain before the factorisation. The groups: block
   Jacobi, the whole subdomain (it has no interface, Sec. 2.1); SCHUR and RAP, the interior
   nodes and the interface nodes of each subdomain (Sec. 2.2.1), so A_i keeps its
   [B F; E C] form. NATURAL: ascending original index. RCM: reverse Cuthill-McKee of the
   graph the group induces in A + A^T (Sec. 3.1, Algorithm "Block Jacobi ILU on GPU"); each
   component starts at its unplaced node of least (degree, index), neighbours are appended
   by (degree, index), the sequence is then reversed. COLOR: greedy multicolouring of that
   graph (nodes in ascending index take the smallest colour none of their earlier neighbours
   has), listed colour by colour, ascending index inside a colour: a lower factor in the
   pattern of A then has one level per colour (Sec. 3.1), at the cost of a weaker ILU. */
typedef enum { ILU_ORDER_NATURAL = 0, ILU_ORDER_RCM = 1, ILU_ORDER_COLOR = 2 } ilu_order;

typedef struct {
    int32_t variant;      /* ilu_variant */
    int32_t factor_B;     /* factor of the interior block B (BJ: of each local block A_i) */
    int32_t factor_S;     /* factorisation of A_i whose (2,2) blocks give L_S, U_S */
    int32_t form;         /* ilu_form; AUTO = W/Z for ILU0/MILU0 B-factors, E/F for ILUT */
    double ilut_tau;      /* ILUT relative drop tolerance (row 2-norm scaled) */
    int32_t ilut_p;       /* ILUT entries kept per row in each of the L and U parts */
    int32_t inner_iters;  /* GMRES steps on the preconditioned Schur system (Eq. preSS) */
    int32_t pc_precision; /* ilu_prec: arithmetic of the factors and of M^{-1} */
    int32_t ordering;     /* ilu_order: order inside each group of a subdomain */
    double pivot_eps;     /* small-pivot perturbation relative to max_j |a_ij| (0 = off) */
    void* stream;         /* cudaStream_t for every device call (NULL = legacy stream) */
    uint64_t spin_limit;  /* iteration bound of every device-side wait (0 = default) */
    int32_t use_graphs;   /* capture one FGMRES cycle as a CUDA graph (1) or launch (0) */
    int32_t block_threads;/* threads per CTA of the per-subdomain kernels (0 = autotune) */
    int32_t analysis_only;/* 1: host analysis only (no device memory, no factorisation);
                             only ilu_get_sizes / _perm / _levels / _local_pattern /
                             _stream / _stream_stats / _times and ilu_free are valid */
    int32_t kernel_path;  /* 0: level programs streamed into shared memory by TMA (falls
                             back to 1 when a row does not fit a chunk);
                             1: generic level kernels reading the programs from global memory */
    int32_t inner_launch; /* streamed path, inner Schur GMRES of the apply: 0 = one
                             cooperative launch for all inner steps when every subdomain's CTA
                             can be resident at once (else as 1; default), 1 = four launches
                             per inner step */
    int32_t fill_level;   /* k >= 0: the ILU0 / MILU0 factor kinds become ILU(k) / MILU(k)
                             (the paper runs ILU(1) and ILU(2), Sec. 4.2-4.4). Each local block
                             is stored in its level-k fill pattern (level of a stored entry 0;
                             eliminating pivot m of row i gives (i, j) the level
                             lev(i,m) + lev(m,j) + 1, the least wins), zeros at the fill, and
                             factorised in it. ILU_ERR_ARG with factor_B = ILUT. Default 0. */
    int32_t l1_block;     /* block Jacobi only (else ILU_ERR_ARG): 1 = l1-BJ (Sec. 4.3), every
                             diagonal entry of A_i increased by the sum of |a_ij| over the columns
                             of other subdomains before the factorisation. Default 0. */
    int32_t chain_sched;  /* streamed path, schedule of the interface rows of each subdomain
                             program (the forward program's W/E, L_S, U_S rows; the local Schur
                             program): 0 = the cheaper of levels and chains by an estimate of
                             consumer cycles (default), 1 = levels only, 2 = chains. Chains run
                             rows that need only the previous row of their chain as warp scans
                             (stream_layout.h); results agree with the level schedule to rounding. */
    int32_t gs_precision; /* gmres_solve, arithmetic of the two classical Gram-Schmidt passes of
                             each Arnoldi step (Sec. 4.1.1): 0 = both in FP64; 1 = the first
                             pass's coefficients h1 = V^T w from FP32 copies of V and w, then
                             w -= V h1 and the second pass in FP64 (the second pass removes the
                             ~6e-8 ||w|| the estimate leaves); 2 = as 1, and the second
                             pass's update w -= V h2 from the FP32 copy of V with FP32 products:
                             h2 is then ~6e-8 ||w||, so the update's error, ~1e-7 ||V h2||, is
                             ~1e-14 ||w||, the size of FP64 rounding in the full update;
                             3 (default) = as 2, and the first update w -= V h1 and the second
                             pass's dots V^T w in double-float arithmetic (pairs of FP32 numbers,
                             ~48 significant bits, error-free products and sums) from a two-term
                             FP32 split of every basis vector kept beside V (4 more bytes per
                             basis entry): no FP64 operation per basis entry, one FP64
                             subtraction per row. In this mode ||w2|| is taken as
                             (||w1||^2 - ||h2||^2)^(1/2), ||w1||^2 summed in double-float beside
                             the dots (w1 = w2 + V h2, V h2 orthogonal to w2), and w2 / ||w2|| is
                             formed in double-float; when the subtraction cancels
                             (||w2||^2 <= 1e-2 ||w1||^2) ||w2|| is formed explicitly.
                             All FP32 forms need the entries of w within the FP32 range. The
                             coefficients H = h1 + h2, w itself, ||w||, the Givens rotations,
                             the solution update and the true residual are FP64 in every mode. */
    int32_t autotune;     /* streamed path: 1 = ilu_setup measures, for each streamed program, the
                             apply time with consumer groups of 32, 64, 96 and 128 threads
                             (CUDA events on opts.stream, the program rebuilt for each) and keeps
                             the fastest; the choice is remembered for the process, keyed by the
                             structure of the problem, so a later setup of the same structure
                             builds it directly. 0 (default) = the level-width rule. Ignored with
                             block_threads != 0. See ilu_get_tuning. */
    int32_t ilut_setup;   /* factor_B = ILUT: 0 (default) = the numeric factorisation on the device
                             (one warp per row, rows handed out in order, each waiting on the
                             rows of its pivots), the host's result bit for bit; the host
                             factorisation when ilut_p > 32, a row touches more columns than
                             the device's per-warp table holds, or the handle is analysis-only.
                             1 = on the host (threads over subdomains). ilu_get_times reports
                             which ran and its time. */
} ilu_opts;

typedef struct {
    int32_t iters;        /* Arnoldi steps over all cycles (the count the paper reports) */
    int32_t restarts;     /* completed cycles */
    double rel_res_true;  /* ||b - A x||_2 / ||b||_2 computed in FP64 at the end */
    double rel_res_est;   /* last Givens residual estimate / ||b|| */
    double setup_ms;      /* wall time of ilu_setup for this handle */
    double solve_ms;      /* wall time of this gmres_solve */
    int32_t status;       /* ilu_status of the solve */
    int32_t npert;        /* pivots perturbed during setup */
} ilu_solve_info;

/* Defaults: SCHUR, B = ILU0, S = MILU0, form AUTO, inner 3 steps, FP32 preconditioner,
   natural ordering, pivot_eps 1e-8, ILUT(1e-3, 10), graphs on, autotuned CTA size. */
void ilu_opts_default(ilu_opts* opts);

/* Setup (Algorithm "Additive SCHUR-ILU on GPU", Setup; Algorithm "Block Jacobi ILU on
   GPU", Setup). A: host CSR; part: host int32[n] with values in [0, p); p >= 1.
   Host side: validation, interior/interface classification (a node is interface if a
   stored a_ij or a_ji couples it to another subdomain), interior-first permutation
   (interior grouped by subdomain, then interface grouped by subdomain; block Jacobi has
   no interface, each subdomain is one group; inside a group the order opts.ordering
   gives), local blocks A_i = [B_i F_i; E_i C_i] (in their level-k pattern with
   fill_level k), level sets, the level programs. Device side: ILU(0)/MILU(0) numeric
   factorisation of every A_i (ILUT is computed on the host), factor extraction and
   packing. ILU_ERR_UNSUPPORTED for option combinations only the streamed path covers
   when it cannot be used (RAP, bfloat16 storage). The library copies A and part; on success
   *h owns all device memory until ilu_free. Errors: ILU_ERR_CSR, ILU_ERR_ARG,
   ILU_ERR_TOO_LARGE, ILU_ERR_OOM, ILU_ERR_ZERO_PIVOT (only with pivot_eps = 0),
   ILU_ERR_UNSUPPORTED, ILU_ERR_CUDA. On error *h is NULL. Synchronises the stream before returning. */
ilu_status ilu_setup(const ilu_csr* A, const int32_t* part, int32_t p, const ilu_opts* opts,
                     void** h);

/* z = M^{-1} r (Algorithm "Additive SCHUR-ILU on GPU", Solve, with the inner GMRES of
   Eq. preSS; or the block Jacobi solve). r, z: DEVICE double[n] in the original
   ordering, caller-owned; z must not alias r. Asynchronous on opts.stream.
   Errors: ILU_ERR_ARG (NULL, aliasing), ILU_ERR_CUDA. */
ilu_status ilu_apply(void* h, const double* r, double* z);

/* Flexible GMRES(restart) with right preconditioning M^{-1} (Sec. 4.1.1), all vectors
   FP64 on the device: b (DEVICE double[n], original ordering) and x (DEVICE double[n],
   in = x0, out = solution), caller-owned. Stops when the true residual
   ||b - A x|| <= rtol ||b|| (checked at the end of every cycle; a cycle ends early when
   the Givens estimate meets the same bound) or after maxit Arnoldi steps.
   Synchronises the stream at every cycle end and fills *info (may be NULL).
   restart in [1, 256] (the Gram-Schmidt kernels keep one coefficient per basis vector in
   shared memory; the paper runs restarts of 50 and 100).
   Returns ILU_OK, ILU_ERR_NOT_CONVERGED (x = last iterate), ILU_ERR_TIMEOUT, ILU_ERR_ARG,
   ILU_ERR_OOM, ILU_ERR_CUDA. ||b|| = 0 gives x = 0. */
ilu_status gmres_solve(void* h, const double* b, double* x, double rtol, int32_t restart,
                       int32_t maxit, ilu_solve_info* info);

/* Releases every resource of the handle (NULL is a no-op). Synchronises the stream. */
ilu_status ilu_free(void* h);

/* Static string for a status code. */
const char* ilu_status_str(ilu_status s);

/* ---------------------------------------------------------------------------------
 * Introspection and single-step entry points (for parity checks and benchmarks).
 * All host outputs are caller-allocated; all device pointers are caller-owned.
 * --------------------------------------------------------------------------------- */

/* out[0..11] = n, p, n1, n2, nnz(A), nnz(C_off), perturbed pivots, max levels over
   subdomains of L_B, U_B, L_S, U_S, max rows of a local block A_i;
   out[12..23] = (scheduled rows, factor entries, levels summed over subdomains) of the
   four level programs the apply runs: block Jacobi L_A+U_A; forward (L_B and W, or L_B,
   U_B and E); local Schur L_S+U_S; backward (Z and U_B, or F, L_B and U_B). */
ilu_status ilu_get_sizes(void* h, int64_t* out);

/* Permutation (host int32 outputs, each may be NULL): perm[new] = old, iperm[old] = new,
   int_ptr[p+1] / if_ptr[p+1]: interior rows of subdomain s are new indices
   [int_ptr[s], int_ptr[s+1]), interface rows n1 + [if_ptr[s], if_ptr[s+1]);
   iface[n] = 1 for interface nodes (original numbering). */
ilu_status ilu_get_perm(void* h, int32_t* perm, int32_t* iperm, int32_t* int_ptr,
                        int32_t* if_ptr, int32_t* iface);

/* Level of every row (host int32[n] indexed by the permuted global row, -1 for rows not
   in the factor) for which = 0 L_A, 1 U_A (pattern of each local block A_i), 2 L_B,
   3 U_B, 4 L_S, 5 U_S (patterns the apply uses); *nlev = max levels over subdomains.
   Level: 0 without dependencies, else 1 + max level of the rows it depends on. */
ilu_status ilu_get_levels(void* h, int32_t which, int32_t* lev, int32_t* nlev);

/* Combined L\U values (host double[nnz of the stored block]) of the device factorisation
   of local block s in the pattern ilu_get_local_pattern returns (local order: the
   subdomain's groups as ilu_setup describes; the level-k pattern with fill_level k):
   fact = 1 the factor giving L_B, U_B, W, Z (block Jacobi: L_A, U_A); fact = 2 the one
   giving L_S, U_S. ILU_ERR_ARG if that factor does not have the stored pattern (ILUT). */
ilu_status ilu_get_local_factor(void* h, int32_t s, int32_t fact, double* val);

/* Pattern of local block s as stored for the factorisation (A_s in the local order; with
   fill_level k > 0 its level-k fill pattern): rowptr (host int32[rows of s + 1], from 0)
   and colind (host int32[*nnz], local column indices, ascending in each row). Either array
   may be NULL; *nnz (required) receives the entry count. Valid on analysis-only handles. */
ilu_status ilu_get_local_pattern(void* h, int32_t s, int32_t* rowptr, int32_t* colind, int32_t* nnz);

/* y = A x with the handle's FP64 CSR SpMV kernel (x, y DEVICE double[n], original
   ordering, no aliasing). Asynchronous on opts.stream. */
ilu_status ilu_spmv(void* h, const double* x, double* y);

/* The inner Schur solve alone (Eq. preSS with inner_iters GMRES steps, x0 = 0):
   gp, y DEVICE double[n2] in interface numbering. Asynchronous. */
ilu_status ilu_inner_solve(void* h, const double* gp, double* y);

/* Device time per kernel class since ilu_profile(h, 1) (which resets the counters):
   names[i] (static strings), ms[i], launches[i] for i < *count (capacity in *count on
   entry; the number of classes on return). Profiling brackets each class's launches
   with CUDA events on opts.stream and disables cycle-graph replay while on; reading
   synchronises on the last event. ilu_profile(h, 0) turns it off. */
ilu_status ilu_profile(void* h, int32_t enable);
ilu_status ilu_profile_read(void* h, const char** names, double* ms, int64_t* launches,
                            int32_t* count);

/* Launch accounting and device status: out[0] = kernels enqueued by this handle so far
   (direct launches plus the kernel nodes of every replayed cycle graph), out[1] =
   cycle-graph replays, out[2] = kernel nodes per cycle graph, out[3] = CTAs of the
   row-partitioned kernels, out[4] = device error word (bit 1: zero pivot, bit 2: a bounded
   device wait timed out; synchronises the stream to read it), out[5] = 1 when the apply
   runs the TMA-streamed level programs, out[6..13] = (entries per row record, consumer
   threads) of the streamed programs block Jacobi, forward, local Schur, backward (0 if
   unused), out[14] = 1 when the apply runs the inner Schur GMRES as one cooperative
   launch, out[15] = device memory the handle holds, in bytes (factors, programs, Krylov
   workspaces; what ilu_free returns). out must hold 16 values. */
ilu_status ilu_get_stats(void* h, int64_t* out);

/* Wall-clock times of a handle, in ms: out[0] = host analysis of ilu_setup (classification,
   ordering, patterns, level programs, streams), out[1] = its device part (uploads, numeric
   factorisation, packing), out[2] = the last gmres_solve, out[3] = the part of it spent
   capturing and instantiating the cycle graph (0 when the handle's graph was reused),
   out[4] = the ILUT factorisation of factor_B = ILUT (part of out[0]; 0 otherwise), out[5] =
   1 when that factorisation ran on the device, 0 when on the host or not ILUT, out[6] = the
   device kernels of it (CUDA events; 0 on the host). out must hold 7 values. Errors: ILU_ERR_ARG for a null pointer. */
ilu_status ilu_get_times(void* h, double* out);

/* The ILUT factor of local block s (factor_B = ILUT): B_s for SCHUR and RAP (the interior rows
   with their interior columns), A_s for block Jacobi, as combined L\U rows in the local order,
   columns ascending, the pivot stored in every row. rowptr: host int32[rows of the block + 1]
   (from 0); colind: host int32[*nnz]; val: host double[*nnz] (FP64, as factorised). Any of the
   three arrays may be NULL; *nnz (required) receives the entry count. On a device handle the
   values are read back from the device (synchronises the stream); on an analysis-only handle
   they are the host factorisation's. Errors: ILU_ERR_ARG (null handle or nnz, s out of
   range, factor_B not ILUT), ILU_ERR_CUDA. */
ilu_status ilu_get_ilut_factor(void* h, int32_t s, int32_t* rowptr, int32_t* colind, double* val,
                               int32_t* nnz);

/* The Krylov basis of the handle's last gmres_solve (its last cycle): which = 0 the
   orthonormal vectors v_0..v_{k-1} (k <= restart + 1), which = 1 the preconditioned
   vectors z_0..z_{k-1} (k <= restart); out: HOST double[k * n], vector i at out + i * n, in
   the original ordering. Vectors past the cycle's last step hold stale values. With
   gs_precision = 3 the basis is kept as two FP32 parts and v = hi + lo is returned.
   Synchronises the stream. Errors: ILU_ERR_ARG (null pointers, which or k out of range, no
   solve yet). */
ilu_status ilu_get_krylov(void* h, int32_t which, int32_t k, double* out);

/* What ilu_setup chose for the streamed programs (0 block Jacobi, 1 forward, 2 local Schur,
   3 backward): nt[i] consumer threads of program i (0 if unused); ms[4 * i + c] the apply
   time measured with candidate c = 0..3 (32, 64, 96, 128 threads; 0 where not measured);
   *state = 0 level-width rule, 1 measured by this setup, 2 taken from an earlier setup of
   the same structure. Host-side only. Errors: ILU_ERR_ARG for a null pointer. */
ilu_status ilu_get_tuning(void* h, int32_t* nt, double* ms, int32_t* state);

/* Shape of one TMA-streamed level program (the level schedule of Sec. 3.1 as the device
   consumes it): program 0 = block Jacobi, 1 = forward (L_B, the W rows and S~), 2 = local
   Schur S~ alone, 3 = backward. out[0] = entries per row record, out[1] = consumer
   threads, out[2] = chunks, out[3] = waves, out[4] = row records including skip records,
   out[5] = skip records, out[6] = group barriers of the longest subdomain program,
   out[7] = levels of the deepest subdomain program (the barriers a plain level schedule
   would need), out[8] = bytes of the shared-memory ring the chunks stream through,
   out[9] = 1 when every subdomain's working vector fits in shared memory beside the ring
   (else the kernels keep it in a global scratch vector; known once the device setup ran,
   0 for analysis-only handles), out[10] = scan waves (chains solved 32 rows per warp and
   wave, stream_layout.h) of the subdomain program with most, out[11] = group barriers plus
   scan waves, largest over the subdomain programs (its dependent steps), out[12] =
   subdomains whose chain section (the interface rows) runs as chains rather than levels.
   A program the handle does not use reports zeros. out must hold 13 values.
   Host-side only: needs no device. Errors: ILU_ERR_ARG for a null pointer or a program
   outside 0..3. */
ilu_status ilu_get_stream_stats(void* h, int32_t program, int64_t* out);

/* Copy of one streamed program as the host built it (values and pivot inverses are
   filled on the device, so the copy holds zeros there): blob = the chunks (layout in the
   comment of csrc/stream_layout.h), ch0 = p+1 chunk offsets per subdomain, meta[0] =
   blob bytes, meta[1] = chunk bytes, meta[2] = entries per record, meta[3] = value bytes,
   meta[4] = consumer threads, meta[5] = working-vector element (and pivot-inverse) bytes;
   meta is int64[6]. Call with blob = ch0 = NULL to read meta first; blob must
   hold meta[0] bytes and ch0 p+1 values. Host-side only. Errors: ILU_ERR_ARG (null
   handle or meta, program outside 0..3), ILU_ERR_UNSUPPORTED (program not built). */
ilu_status ilu_get_stream(void* h, int32_t program, uint8_t* blob, int32_t* ch0, int64_t* meta);

/* ---------------------------------------------------------------------------------
 * Measurement probes (no counterpart in the paper): the denominators the benchmark
 * reports its rooflines against, measured on the current device. Each allocates a few
 * bytes of scratch on `stream` (a cudaStream_t, NULL = legacy stream), synchronises it
 * and frees them. Errors: ILU_ERR_ARG, ILU_ERR_CUDA.
 * --------------------------------------------------------------------------------- */

/* FP64 fused multiply-add throughput: a grid of 8 CTAs of 256 threads per SM, every thread
   running eight independent FMA chains of 2^14 steps, timed with CUDA events after a
   warm-up launch. *tflops = 2 * FMAs / time / 1e12. */
ilu_status ilu_measure_fp64_peak(void* stream, double* tflops);

/* Latency of one dependent level: one CTA of `threads` threads (32..256, a multiple of
   32) runs 4096 levels; in each, every thread reads four values other threads stored in
   the previous level, stores their weighted sum, and the group meets at a barrier
   (bar.sync on the group; __syncwarp for one warp). *cycles_per_level = SM clock cycles
   (clock64) per level: the floor of a level of a level-scheduled triangular solve
   (Sec. 3.1) on this GPU. */
ilu_status ilu_measure_level_latency(void* stream, int32_t threads, double* cycles_per_level);

/* ---------------------------------------------------------------------------------
 * Allocation-free variant (no counterpart in the paper).
 * --------------------------------------------------------------------------------- */

/* The inner Schur solve of ilu_inner_solve, for callers that cannot allocate device
   memory at call time: code that runs on a fixed device-memory budget set aside up front,
   or that must not trigger the implicit synchronisation an allocation can bring.
   Identical inputs, outputs and arithmetic (gp, y: DEVICE double[n2], interface
   numbering), but the Krylov workspace lives in a fixed 8 MiB device array the library
   holds on every GPU that loads it, until the process exits; the call allocates nothing.
   The first call on a device looks up the array's device address (make that first call
   before any stream capture); later calls reuse it, so a cudaDeviceReset after it is not
   supported. Every call shares the array, which keeps the last call's contents; each call
   re-initialises the control state it reads. Calls that overlap on the GPU (other streams
   or host threads) race on it. Needs the default streamed kernels with every subdomain's working vector
   in shared memory (else ILU_ERR_UNSUPPORTED). ILU_ERR_TOO_LARGE when the workspace,
   256-byte aligned pieces of (inner_iters + 4) * n2 vector elements of the
   preconditioner type, 792 * p bytes of partial sums and a 9 KB control block, exceeds
   8 MiB. ILU_ERR_ARG for NULL / aliased vectors, a block Jacobi handle, or a current
   device other than the handle's. Asynchronous on opts.stream. */
ilu_status ilu_inner_solve_noalloc(void* h, const double* gp, double* y);

#ifdef __cplusplus
}
#endif
#endif
