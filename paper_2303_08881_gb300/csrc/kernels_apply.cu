// kernels_apply.cu -- the preconditioner apply z = M^{-1} r on sm_103a.
//
// One CTA per subdomain. A subdomain's working vector lives in shared memory when it
// fits (else in a global scratch slice); its triangular solves run as level programs:
// the rows of one level are independent (Sec. 3.1, level scheduling), so the CTA's
// threads take them in parallel and a CTA barrier separates consecutive levels.
//
//   block Jacobi        (Algorithm "Block Jacobi ILU on GPU", Solve): gather, L_A and
//                        U_A level programs, scatter;                         k_bj
//   two-level, forward   (Algorithm "Additive SCHUR-ILU on GPU", Solve, lines
//                        f' = L_B^{-1} f, g' = g - W f'; or the E/F form of Algorithm
//                        "Additive block ILU solve"), then c = U_S^{-1} L_S^{-1} g';
//                                                                              k_fwd
//   inner GMRES steps    on Eq. preSS, MATVEC y + S~^{-1} sum_j E_ij y_j (Eq. preSMV2),
//                        classical Gram-Schmidt with reorthogonalisation: k_inner_a/b/c
//   backward             least squares, y = V t, f'' = f' - Z y, u = U_B^{-1} f'',
//                        scatter;                                             k_bwd
#include "devutil.cuh"
#include "handle.h"
#include "inner_lsq.cuh"

namespace ilu2l {

// partial-sum banks of the inner GMRES: [bank][i][s]
__device__ __forceinline__ double* ipart(double* base, int bank, int i, int s, int p) {
    return base + ((size_t)(bank * (kMaxInner + 1) + i)) * p + s;
}
constexpr int kBankDot1 = 0, kBankDot2 = 1, kBankNorm = 2;

// Run the levels of program P for subdomain s on the working vector x.
template <class T>
__device__ __forceinline__ void run_prog(const ProgDev<T>& P, int s, T* x) {
    const int e0 = P.sub_lvl[s], e1 = P.sub_lvl[s + 1];
    for (int e = e0; e < e1; e++) {
        const int k0 = P.lvl_ptr[e], k1 = P.lvl_ptr[e + 1];
        for (int k = k0 + (int)threadIdx.x; k < k1; k += blockDim.x) {
            const int r = P.prow[k];
            T acc = x[r];
            const int q1 = P.pptr[k + 1];
            for (int q = P.pptr[k]; q < q1; q++) acc -= P.pval[q] * x[P.pcol[q]];
            x[r] = acc * P.pdinv[k];
        }
        __syncthreads();
    }
}

template <class T>
__device__ __forceinline__ T* work_vec(const SubDev& sd, T* xg, int q0, int ns) {
    extern __shared__ __align__(16) unsigned char smraw[];
    return (ns <= sd.smem_len) ? reinterpret_cast<T*>(smraw) : xg + q0;
}

// ---------------------------------------------------------------------------------------
// block Jacobi: z_i = U_Ai^{-1} L_Ai^{-1} r_i on every subdomain
template <class T>
__global__ void k_bj(SubDev sd, ProgDev<T> P, const double* __restrict__ r, double* __restrict__ z,
                     T* xg, const int32_t* done) {
    if (done && *done) return;
    const int s = blockIdx.x;
    const int q0 = sd.qoff[s], ns = sd.qoff[s + 1] - q0;
    T* x = work_vec<T>(sd, xg, q0, ns);
    for (int l = threadIdx.x; l < ns; l += blockDim.x) x[l] = (T)r[sd.q_orig[q0 + l]];
    __syncthreads();
    run_prog(P, s, x);
    for (int l = threadIdx.x; l < ns; l += blockDim.x) z[sd.q_orig[q0 + l]] = (double)x[l];
}

// ---------------------------------------------------------------------------------------
// two-level forward part: f' (kept in fq) and c = S~^{-1} g' (kept in W0), ||c||^2 partials
template <class T>
__global__ void k_fwd(SubDev sd, ProgDev<T> PF, ProgDev<T> PS, InnerDev<T> in,
                      const double* __restrict__ r, T* __restrict__ fq, T* xg, const int32_t* done) {
    __shared__ double red[32];
    if (done && *done) return;
    const int s = blockIdx.x;
    const int q0 = sd.qoff[s], ns = sd.qoff[s + 1] - q0, ni = sd.nint[s], nf = ns - ni;
    T* x = work_vec<T>(sd, xg, q0, ns);
    for (int l = threadIdx.x; l < ns; l += blockDim.x) x[l] = (T)r[sd.q_orig[q0 + l]];
    __syncthreads();
    run_prog(PF, s, x);
    for (int l = threadIdx.x; l < ni; l += blockDim.x) fq[q0 + l] = x[l];
    run_prog(PS, s, x + ni);
    const int g0 = sd.if_ptr[s];
    T acc = (T)0;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        const T c = x[ni + i];
        in.W0[g0 + i] = c;
        acc += c * c;
    }
    acc = block_sum_t<T>(acc, reinterpret_cast<T*>(red));
    if (threadIdx.x == 0) {
        *ipart(in.part, kBankNorm, 0, s, sd.p) = (double)acc;
        if (s == 0) {
            in.ctl->steps = -1;
            in.ctl->zero = 0;
        }
    }
}

// standalone start of the inner solve: c = S~^{-1} gp for an FP64 interface vector
template <class T>
__global__ void k_inner_start(SubDev sd, ProgDev<T> PS, InnerDev<T> in, const double* __restrict__ gp,
                              T* xg) {
    __shared__ double red[32];
    const int s = blockIdx.x;
    const int q0 = sd.qoff[s], ns = sd.qoff[s + 1] - q0, ni = sd.nint[s], nf = ns - ni;
    T* x = work_vec<T>(sd, xg, q0, ns);
    const int g0 = sd.if_ptr[s];
    for (int i = threadIdx.x; i < nf; i += blockDim.x) x[ni + i] = (T)gp[g0 + i];
    __syncthreads();
    run_prog(PS, s, x + ni);
    T acc = (T)0;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        const T c = x[ni + i];
        in.W0[g0 + i] = c;
        acc += c * c;
    }
    acc = block_sum_t<T>(acc, reinterpret_cast<T*>(red));
    if (threadIdx.x == 0) {
        *ipart(in.part, kBankNorm, 0, s, sd.p) = (double)acc;
        if (s == 0) {
            in.ctl->steps = -1;
            in.ctl->zero = 0;
        }
    }
}

// ---------------------------------------------------------------------------------------
// inner step j, part A: normalise v_j, w = v_j + S~^{-1} (C_off v_j), first CGS dots
template <class T>
__global__ void k_inner_a(SubDev sd, ProgDev<T> PS, InnerDev<T> in, int j, T* xg, const int32_t* done) {
    __shared__ double red[32 * 8];
    if (done && *done) return;
    InnerCtl* ctl = in.ctl;
    if (*((volatile int32_t*)&ctl->steps) >= 0 || *((volatile int32_t*)&ctl->zero)) return;
    const int s = blockIdx.x, p = sd.p, n2 = sd.n2;
    const int q0 = sd.qoff[s], ns = sd.qoff[s + 1] - q0, ni = sd.nint[s], nf = ns - ni;
    // every CTA forms the same norm from the same partials in the same order
    const double nrm = sqrt(warp_allsum_ldcg(ipart(in.part, kBankNorm, 0, 0, p), p));
    if (j == 0) {
        if (s == 0 && threadIdx.x == 0) ctl->beta = nrm;
        if (nrm == 0.0) {
            if (s == 0 && threadIdx.x == 0) ctl->zero = 1;
            return;
        }
    } else {
        const double beta = ctl->beta;
        if (s == 0 && threadIdx.x == 0) ctl->H[(j - 1) * (kMaxInner + 1) + j] = nrm;
        if (nrm <= 1e-14 * beta) {  // lucky breakdown: the Krylov space is exhausted
            if (s == 0 && threadIdx.x == 0) ctl->steps = j;
            return;
        }
    }
    const T inv = (T)(1.0 / nrm);
    const T* __restrict__ Win = (j & 1) ? in.W1 : in.W0;
    T* __restrict__ Wout = (j & 1) ? in.W0 : in.W1;
    T* x = work_vec<T>(sd, xg, q0, ns) + ni;  // interface part only
    const int g0 = sd.if_ptr[s];
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        const int gi = g0 + i;
        T acc = (T)0;
        for (int q = in.coff_rp[gi]; q < in.coff_rp[gi + 1]; q++) acc += in.coff_v[q] * Win[in.coff_ci[q]];
        x[i] = acc * inv;
    }
    __syncthreads();
    run_prog(PS, s, x);
    T* Vj = in.V + (size_t)j * n2;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        const int gi = g0 + i;
        const T v = Win[gi] * inv;
        Vj[gi] = v;
        const T w = v + x[i];
        Wout[gi] = w;
        x[i] = w;
    }
    __syncthreads();
    for (int i0 = 0; i0 <= j; i0 += 8) {
        T acc[8];
#pragma unroll
        for (int u = 0; u < 8; u++) acc[u] = (T)0;
        for (int i = threadIdx.x; i < nf; i += blockDim.x) {
            const T w = x[i];
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (i0 + u <= j) acc[u] += in.V[(size_t)(i0 + u) * n2 + g0 + i] * w;
        }
        block_sum_nt<T, 8>(acc, reinterpret_cast<T*>(red));
        if (threadIdx.x == 0)
            for (int u = 0; u < 8 && i0 + u <= j; u++) *ipart(in.part, kBankDot1, i0 + u, s, p) = (double)acc[u];
    }
}

// inner step j, part B (bank_in = dot1) or C (bank_in = dot2): w -= V h; next partials
template <class T>
__global__ void k_inner_bc(SubDev sd, InnerDev<T> in, int j, int second, const int32_t* done) {
    __shared__ double red[32 * 8];
    __shared__ double hh[kMaxInner + 1];
    if (done && *done) return;
    InnerCtl* ctl = in.ctl;
    if (*((volatile int32_t*)&ctl->steps) >= 0 || *((volatile int32_t*)&ctl->zero)) return;
    const int s = blockIdx.x, p = sd.p, n2 = sd.n2;
    const int ns = sd.qoff[s + 1] - sd.qoff[s], ni = sd.nint[s], nf = ns - ni;
    const int bank = second ? kBankDot2 : kBankDot1;
    {  // warp w sums the partials of coefficients w, w + nwarps, ...
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int i = threadIdx.x >> 5; i <= j; i += nw) {
            const double h = warp_allsum_ldcg(ipart(in.part, bank, i, 0, p), p);
            if (lane == 0) hh[i] = h;
        }
    }
    __syncthreads();
    if (s == 0 && threadIdx.x == 0) {
        for (int i = 0; i <= j; i++) {
            double& H = ctl->H[j * (kMaxInner + 1) + i];
            H = second ? H + hh[i] : hh[i];
        }
    }
    T* __restrict__ W = (j & 1) ? in.W0 : in.W1;
    const int g0 = sd.if_ptr[s];
    T nacc = (T)0;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        T w = W[g0 + i];
        for (int t = 0; t <= j; t++) w -= (T)hh[t] * in.V[(size_t)t * n2 + g0 + i];
        W[g0 + i] = w;
        nacc += w * w;
    }
    if (second) {
        nacc = block_sum_t<T>(nacc, reinterpret_cast<T*>(red));
        if (threadIdx.x == 0) *ipart(in.part, kBankNorm, 0, s, p) = (double)nacc;
        return;
    }
    __syncthreads();
    for (int i0 = 0; i0 <= j; i0 += 8) {
        T acc[8];
#pragma unroll
        for (int u = 0; u < 8; u++) acc[u] = (T)0;
        for (int i = threadIdx.x; i < nf; i += blockDim.x) {
            const T w = W[g0 + i];
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (i0 + u <= j) acc[u] += in.V[(size_t)(i0 + u) * n2 + g0 + i] * w;
        }
        block_sum_nt<T, 8>(acc, reinterpret_cast<T*>(red));
        if (threadIdx.x == 0)
            for (int u = 0; u < 8 && i0 + u <= j; u++) *ipart(in.part, kBankDot2, i0 + u, s, p) = (double)acc[u];
    }
}

// two-level backward part: y = V t; f'' = f' - Z y (or f - F y, L_B); u = U_B^{-1} f''
template <class T>
__global__ void k_bwd(SubDev sd, ProgDev<T> PB, InnerDev<T> in, const double* __restrict__ r,
                      const T* __restrict__ fq, int ef, double* __restrict__ z, T* xg, const int32_t* done) {
    __shared__ double t[kMaxInner];
    if (done && *done) return;
    const int s = blockIdx.x;
    const int q0 = sd.qoff[s], ns = sd.qoff[s + 1] - q0, ni = sd.nint[s], nf = ns - ni;
    const int steps = (sd.n2 > 0) ? inner_lsq<T>(in.ctl, in.part, sd.p, in.k, t) : 0;
    T* x = work_vec<T>(sd, xg, q0, ns);
    if (ef) {
        for (int l = threadIdx.x; l < ni; l += blockDim.x) x[l] = (T)r[sd.q_orig[q0 + l]];
    } else {
        for (int l = threadIdx.x; l < ni; l += blockDim.x) x[l] = fq[q0 + l];
    }
    const int g0 = sd.if_ptr[s];
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        T y = (T)0;
        for (int u = 0; u < steps; u++) y += (T)t[u] * in.V[(size_t)u * sd.n2 + g0 + i];
        x[ni + i] = y;
    }
    __syncthreads();
    run_prog(PB, s, x);
    for (int l = threadIdx.x; l < ns; l += blockDim.x) z[sd.q_orig[q0 + l]] = (double)x[l];
}

// standalone end of the inner solve: y (FP64, interface numbering) = V t
template <class T>
__global__ void k_inner_finish(SubDev sd, InnerDev<T> in, double* __restrict__ y) {
    __shared__ double t[kMaxInner];
    const int s = blockIdx.x;
    const int ns = sd.qoff[s + 1] - sd.qoff[s], ni = sd.nint[s], nf = ns - ni;
    const int steps = inner_lsq<T>(in.ctl, in.part, sd.p, in.k, t);
    const int g0 = sd.if_ptr[s];
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        T acc = (T)0;
        for (int u = 0; u < steps; u++) acc += (T)t[u] * in.V[(size_t)u * sd.n2 + g0 + i];
        y[g0 + i] = (double)acc;
    }
}

// ---------------------------------------------------------------------------------------
// launchers

static size_t smem_bytes(const Handle& h, size_t elt) {
    return (size_t)h.smem_len * elt;
}

template <class T>
cudaError_t launch_inner_bc(const Handle& h, int j, int second, const int32_t* done, cudaStream_t st) {
    k_inner_bc<T><<<h.p, h.threads, 0, st>>>(h.sub(), h.innerdev<T>(), j, second, done);
    return cudaGetLastError();
}

// Per-kernel, process-wide limit: raised to the device maximum, never lowered.
template <class K>
static cudaError_t raise_limit(K kernel) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

template <class T>
cudaError_t configure_apply(size_t dyn_bytes) {
    (void)dyn_bytes;
    cudaError_t e = raise_limit(k_bj<T>);
    if (e == cudaSuccess) e = raise_limit(k_fwd<T>);
    if (e == cudaSuccess) e = raise_limit(k_inner_a<T>);
    if (e == cudaSuccess) e = raise_limit(k_bwd<T>);
    if (e == cudaSuccess) e = raise_limit(k_inner_start<T>);
    return e;
}

template <class T>
cudaError_t launch_bj(const Handle& h, const double* r, double* z, const int32_t* done, cudaStream_t st) {
    k_bj<T><<<h.p, h.threads, smem_bytes(h, sizeof(T)), st>>>(h.sub(), h.progdev<T>(PR_BJ), r, z,
                                                             (T*)h.d_xg, done);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_schur_fwd(const Handle& h, const double* r, const int32_t* done, cudaStream_t st) {
    k_fwd<T><<<h.p, h.threads, smem_bytes(h, sizeof(T)), st>>>(h.sub(), h.progdev<T>(PR_FWD),
                                                               h.progdev<T>(PR_S), h.innerdev<T>(), r,
                                                               (T*)h.d_fq, (T*)h.d_xg, done);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_inner(const Handle& h, const int32_t* done, cudaStream_t st) {
    if (h.n2 == 0) return cudaSuccess;
    for (int j = 0; j < h.inner_k; j++) {
        k_inner_a<T><<<h.p, h.threads, smem_bytes(h, sizeof(T)), st>>>(h.sub(), h.progdev<T>(PR_S),
                                                                       h.innerdev<T>(), j, (T*)h.d_xg, done);
        k_inner_bc<T><<<h.p, h.threads, 0, st>>>(h.sub(), h.innerdev<T>(), j, 0, done);
        k_inner_bc<T><<<h.p, h.threads, 0, st>>>(h.sub(), h.innerdev<T>(), j, 1, done);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_schur_bwd(const Handle& h, const double* r, double* z, const int32_t* done,
                             cudaStream_t st) {
    k_bwd<T><<<h.p, h.threads, smem_bytes(h, sizeof(T)), st>>>(h.sub(), h.progdev<T>(PR_BWD),
                                                               h.innerdev<T>(), r, (const T*)h.d_fq,
                                                               h.form == ILU_FORM_EF ? 1 : 0, z,
                                                               (T*)h.d_xg, done);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_inner_io(const Handle& h, const double* gp, double* y, cudaStream_t st) {
    if (h.n2 == 0) return cudaSuccess;
    cudaError_t e;
    if (h.stream_path) {
        e = launch_inner_start_s<T>(h, gp, st);
        if (e == cudaSuccess) e = launch_inner_s<T>(h, nullptr, st);
    } else {
        k_inner_start<T><<<h.p, h.threads, smem_bytes(h, sizeof(T)), st>>>(h.sub(), h.progdev<T>(PR_S),
                                                                           h.innerdev<T>(), gp, (T*)h.d_xg);
        e = launch_inner<T>(h, nullptr, st);
    }
    if (e != cudaSuccess) return e;
    k_inner_finish<T><<<h.p, h.threads, 0, st>>>(h.sub(), h.innerdev<T>(), y);
    return cudaGetLastError();
}

// Parts B/C and the finish of the inner solve on a caller-provided workspace.
template <class T>
cudaError_t launch_inner_bc_ws(const Handle& h, const InnerDev<T>& in, int j, int second, cudaStream_t st) {
    k_inner_bc<T><<<h.p, h.threads, 0, st>>>(h.sub(), in, j, second, nullptr);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_inner_finish_ws(const Handle& h, const InnerDev<T>& in, double* y, cudaStream_t st) {
    k_inner_finish<T><<<h.p, h.threads, 0, st>>>(h.sub(), in, y);
    return cudaGetLastError();
}

#define ILU2L_INST(T)                                                                              \
    template cudaError_t configure_apply<T>(size_t);                                              \
    template cudaError_t launch_inner_bc_ws<T>(const Handle&, const InnerDev<T>&, int, int, cudaStream_t); \
    template cudaError_t launch_inner_finish_ws<T>(const Handle&, const InnerDev<T>&, double*, cudaStream_t); \
    template cudaError_t launch_inner_bc<T>(const Handle&, int, int, const int32_t*, cudaStream_t);  \
    template cudaError_t launch_bj<T>(const Handle&, const double*, double*, const int32_t*,       \
                                      cudaStream_t);                                              \
    template cudaError_t launch_schur_fwd<T>(const Handle&, const double*, const int32_t*,          \
                                             cudaStream_t);                                         \
    template cudaError_t launch_inner<T>(const Handle&, const int32_t*, cudaStream_t);              \
    template cudaError_t launch_schur_bwd<T>(const Handle&, const double*, double*, const int32_t*, \
                                             cudaStream_t);                                         \
    template cudaError_t launch_inner_io<T>(const Handle&, const double*, double*, cudaStream_t);
ILU2L_INST(float)
ILU2L_INST(double)

}  // namespace ilu2l
