// internal.h -- device data layout and launchers of the ilu2l library (not part of the ABI).
//
// Orderings used inside the library:
//   original   : the caller's row numbering (vectors crossing the ABI);
//   P (global) : interior rows grouped by subdomain, then interface rows grouped by
//                subdomain (Sec. 2.2.1, Eq. equ22); interface numbering = P index - n1;
//   Q (local)  : subdomain-major, inside subdomain s its local order [interior_s;
//                interface_s]; subdomain s owns Q rows [qoff[s], qoff[s+1]).
// Every per-subdomain kernel runs one CTA per subdomain on its Q range and keeps the
// subdomain's working vector in shared memory when it fits (else in a global scratch).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "ilu2l.h"

namespace ilu2l {

constexpr int kMaxInner = 32;   // inner GMRES steps supported on the device
constexpr int kMaxRestart = 400;
constexpr int kMaxRestartGS = 256;  // restart limit of gmres_solve (the Gram-Schmidt kernels' shared arrays)

// ---- a level program: rows of every subdomain scheduled level by level --------------
// Rows of subdomain s are processed in levels [sub_lvl[s], sub_lvl[s+1]); level e covers
// packed rows [lvl_ptr[e], lvl_ptr[e+1]); packed row k updates x[prow[k]] =
// (x[prow[k]] - sum_q pval[q] * x[pcol[q]]) * pdinv[k] over q in [pptr[k], pptr[k+1]).
// Indices are local to the subdomain's working vector (offset by the program's base).
// std::allocator whose value-less construct leaves the element uninitialised: resize()
// then does not write the memory, and the threads that fill a large array fault its pages
// in themselves, in parallel
template <class T>
struct NoInitAlloc : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = NoInitAlloc<U>;
    };
    NoInitAlloc() = default;
    template <class U>
    NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
    template <class U>
    void construct(U* p) noexcept {
        ::new ((void*)p) U;
    }
    template <class U, class... Args>
    void construct(U* p, Args&&... args) {
        ::new ((void*)p) U(std::forward<Args>(args)...);
    }
};
template <class T>
using rawvec = std::vector<T, NoInitAlloc<T>>;

// scan_lvl (optional, one entry per subdomain): the first level of the subdomain's chain
// section -- the levels from there to sub_lvl[s+1] may be scheduled as chains solved by
// warp scans (stream_layout.h); empty when the program has no such section.
struct ProgHost {
    rawvec<int32_t> sub_lvl, lvl_ptr, prow, pptr, pcol, psrc, pdsrc;
    std::vector<int32_t> scan_lvl;
    int32_t max_level_rows = 0, max_levels = 0;
    int64_t nnz() const { return (int64_t)pcol.size(); }
};

template <class T>
struct ProgDev {
    const int32_t* sub_lvl;
    const int32_t* lvl_ptr;
    const int32_t* prow;
    const int32_t* pptr;
    const int32_t* pcol;
    const T* pval;
    const T* pdinv;
};

// ---- per-subdomain geometry ----------------------------------------------------------
struct SubDev {
    const int32_t* qoff;    // p+1
    const int32_t* nint;    // p  : interior rows of s
    const int32_t* if_ptr;  // p+1: interface numbering offsets
    const int32_t* q_orig;  // n  : original index of Q row q
    int32_t p, n, n1, n2;
    int32_t smem_len;       // working-vector capacity in shared memory (elements)
};

// ---- inner (Schur-level) GMRES state, one per apply ----------------------------------
struct InnerCtl {
    double beta;                              // ||c||, c = S~^{-1} g'
    double H[(kMaxInner + 1) * kMaxInner];    // column-major Hessenberg
    int32_t steps;                            // -1 while running, else the steps taken
    int32_t zero;                             // c == 0
    // grid barrier of the single-launch inner solve (cleared by the kernel that starts it)
    uint32_t gbar_count;                      // arrivals at the grid barriers of the current launch
    uint32_t gbar_gen;                        // (unused)
    int32_t gbar_abort;                       // a CTA gave up waiting: the others stop too
};

template <class T>
struct InnerDev {
    const int32_t* coff_rp;  // n2+1
    const int32_t* coff_ci;  // interface numbering
    const T* coff_v;
    T* V;          // (k+1) x n2, normalised Arnoldi vectors
    T* W0;         // unnormalised vector, two buffers (alternating)
    T* W1;
    double* part;  // partial sums: 3 banks x (k+1) x p
    InnerCtl* ctl;
    int32_t k;
};

// ---- outer FGMRES control block -------------------------------------------------------
struct FgCtl {
    double rtol, bnorm, target, beta, est;
    int32_t steps;      // steps in the current cycle
    int32_t cycle_done; // 1 once the current cycle ended (converged estimate / breakdown / maxit)
    int32_t total;      // Arnoldi steps over all cycles
    int32_t maxit;
    int32_t converged;  // true residual met the target
    int32_t breakdown;
    int32_t m;
    uint32_t counter;   // last-CTA-done counter
    int32_t fuse;       // k_fg_cgs_df ended the current step (||w2|| from ||w1||^2 - ||h2||^2)
    double res_true;
    int32_t err;        // host mirror of the device error word (filled by the host copy)
};

struct FgDev {
    double* V;      // (m+1) x ld: basis vector i at V + i * ld
    double* Z;      // m x ld
    double* w;      // n
    double* H;      // (m+1) x m column-major
    double* cs;
    double* sn;
    double* g;      // m+1
    double* h2;     // m+1: reorthogonalisation coefficients of the current step
    double* hnext;  // 2: norm of the next basis vector and its inverse (of beta after k_fg_resid)
    double* y;      // m: the least-squares solution R y = g of the cycle, written when it ends
    double* gpart;  // (m+2) x ng: partial sums of the groups of kRedGroup CTAs
    uint32_t* gcount;  // ng: arrival counters of the groups (zero between launches)
    double* part;   // G x (m+1) partial sums
    FgCtl* ctl;
    float* V32;     // (m+1) x ld: FP32 copy of V for the first Gram-Schmidt pass (null: FP64 pass)
    float* w32;     // n: FP32 copy of w = A z_j for that pass (with Vlo: then hi part of w1)
    float* wlo;     // n: with Vlo, the lo part of w1 (w1 = w32 + wlo to ~48 bits)
    int32_t upd32;  // the second pass's update w -= V h2 from V32 with FP32 products
    float* Vlo;     // (m+1) x ld: V - V32 rounded to FP32, so V32 + Vlo carries ~48 bits of V;
                    // non-null: w -= V h1 and the second pass's dots in double-float arithmetic
    int32_t m, G;
    int64_t ld;     // leading dimension of V and Z: n rounded up to 64 (512-byte rows)
};

// CTAs per first-level group of the two-level reductions of the FGMRES kernels
constexpr int kRedGroup = 32;

struct CsrDev {
    const int32_t* rp;
    const int32_t* ci;
    const double* v;
    int32_t n;
};

// ---- profiling classes ----------------------------------------------------------------
enum ProfClass { PC_APPLY_FWD = 0, PC_INNER, PC_APPLY_BWD, PC_BJ, PC_SPMV_DOT, PC_CGS, PC_NORM,
                 PC_NEXT, PC_UPDATE, PC_RESID, PC_SCALE, PC_COUNT };
extern const char* kProfNames[PC_COUNT];

struct Handle;

// ---- launchers (kernels_*.cu) --------------------------------------------------------
// trsv / apply programs
template <class T>
cudaError_t configure_apply(size_t dyn_bytes);
template <class T>
cudaError_t launch_bj(const Handle& h, const double* r, double* z, const int32_t* done,
                      cudaStream_t st);
template <class T>
cudaError_t launch_schur_fwd(const Handle& h, const double* r, const int32_t* done,
                             cudaStream_t st);
template <class T>
cudaError_t launch_inner(const Handle& h, const int32_t* done, cudaStream_t st);
template <class T>
cudaError_t launch_schur_bwd(const Handle& h, const double* r, double* z, const int32_t* done,
                             cudaStream_t st);
template <class T>
cudaError_t launch_inner_io(const Handle& h, const double* gp, double* y, cudaStream_t st);
template <class T>
cudaError_t launch_inner_bc(const Handle& h, int j, int second, const int32_t* done, cudaStream_t st);
// TMA-streamed level programs (kernels_stream.cu)
struct StreamHost;
template <class T>
cudaError_t configure_stream(const Handle& h, size_t bytes);
template <class T>
cudaError_t launch_pack_stream(const StreamHost& sh, const int64_t* voff, const int32_t* vsrc,
                               const int64_t* doff, const int32_t* dsrc, const double* vals,
                               uint8_t* blob, cudaStream_t st);
template <class T>
cudaError_t launch_bj_s(const Handle& h, const double* r, double* z, const int32_t* done,
                        cudaStream_t st);
template <class T>
cudaError_t launch_fwd_s(const Handle& h, const double* r, const int32_t* done, cudaStream_t st);
template <class T>
cudaError_t launch_inner_s(const Handle& h, const int32_t* done, cudaStream_t st);
template <class T>
cudaError_t launch_bwd_s(const Handle& h, const double* r, double* z, const int32_t* done,
                         cudaStream_t st);
template <class T>
cudaError_t launch_inner_start_s(const Handle& h, const double* gp, cudaStream_t st);
template <class T>
cudaError_t inner_coop_fits(const Handle& h, bool* fits);
// multiplicative two-level variant (kernels_stream.cu, kernels_krylov.cu)
cudaError_t launch_rap_resid(const Handle& h, const double* b, const double* x, double* out, const int32_t* done,
                             cudaStream_t st);
template <class T>
cudaError_t launch_rap_inner_s(const Handle& h, const int32_t* done, cudaStream_t st);
template <class T>
cudaError_t launch_rap_fin_s(const Handle& h, double* z, const int32_t* done, cudaStream_t st);
// inner solve on a caller-provided workspace (allocation-free entry point)
template <class T>
cudaError_t launch_inner_bc_ws(const Handle& h, const InnerDev<T>& in, int j, int second, cudaStream_t st);
template <class T>
cudaError_t launch_inner_finish_ws(const Handle& h, const InnerDev<T>& in, double* y, cudaStream_t st);
template <class T>
cudaError_t launch_inner_io_ws(const Handle& h, const InnerDev<T>& in, T* tbuf, const double* gp, double* y,
                               cudaStream_t st);
// numeric ILU and packing
cudaError_t launch_ilu_numeric(const Handle& h, double* F, int milu, cudaStream_t st);
template <class T>
cudaError_t launch_pack(const ProgHost& ph, const int32_t* d_psrc, const int32_t* d_pdsrc,
                        const double* vals, T* pval, T* pdinv, cudaStream_t st);
// Krylov / SpMV
cudaError_t launch_spmv(const Handle& h, const double* x, double* y, cudaStream_t st);
cudaError_t launch_fg_resid(const Handle& h, const double* b, const double* x, int first, cudaStream_t st);
cudaError_t launch_fg_scale0(const Handle& h, cudaStream_t st);
cudaError_t launch_fg_spmv_dot(const Handle& h, int j, cudaStream_t st);
cudaError_t launch_fg_cgs(const Handle& h, int j, cudaStream_t st);
cudaError_t configure_krylov();
cudaError_t launch_fg_norm(const Handle& h, int j, cudaStream_t st);
cudaError_t launch_fg_next(const Handle& h, int j, cudaStream_t st);
cudaError_t launch_fg_update(const Handle& h, double* x, cudaStream_t st);

}  // namespace ilu2l
