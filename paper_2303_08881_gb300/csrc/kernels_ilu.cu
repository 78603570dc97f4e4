// kernels_ilu.cu -- ILU(0) / MILU(0) numeric factorisation of every local block A_i on
// the device (Sec. 3.1: level-scheduled ILU(0); Sec. 2.3 / Sec. 3.3: MILU, which the
// paper computes on the CPU and calls straightforward to add on the GPU), and the packing
// of factor values into the level programs of the apply.
//
// One CTA per subdomain walks the L levels of A_i; one warp factorises one row with the
// row-wise IKJ update in the pattern of A_i. The arithmetic is ordered exactly like the
// sequential definition (pivots k ascending, each update rounded separately with no
// fused multiply-add, the dropped MILU entries summed in ascending (k, j) order), so the
// device factors are bit-identical to a sequential FP64 factorisation.
#include "devutil.cuh"
#include "handle.h"

namespace ilu2l {

struct NumArgs {
    const int32_t* qoff;
    const int32_t* rp;    // local CSR over Q rows
    const int32_t* ci;    // local column
    const int32_t* dpos;  // diagonal entry per Q row
    const int32_t* sub_lvl;
    const int32_t* lvl_ptr;
    const int32_t* rows;  // local row per level entry
    const double* a;      // original values (pattern of A_i)
    double* f;            // factor values, initialised to a
    double eps;
    int milu;             // 0: ILU(0); 1: MILU(0); 2: MILU only for interface pivots (pmilu0)
    const int32_t* nint;  // interior rows per subdomain (milu = 2)
    int32_t* npert;
    int32_t* err;
};

// position of local column j in the sorted row [b, e) or -1
__device__ __forceinline__ int find_col(const int32_t* __restrict__ ci, int b, int e, int j) {
    while (b < e) {
        const int m = (b + e) >> 1;
        const int c = ci[m];
        if (c == j) return m;
        if (c < j)
            b = m + 1;
        else
            e = m;
    }
    return -1;
}

__global__ void k_ilu_numeric(NumArgs A) {
    const int s = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int q0 = A.qoff[s];
    // pmilu0 (Sec. 3.2, partial ILU): the interior pivots drop plainly, the interface pivots
    // (the Schur complement's own elimination) compensate the diagonal
    const int mfrom = (A.milu == 2) ? A.nint[s] : 0;
    for (int e = A.sub_lvl[s]; e < A.sub_lvl[s + 1]; e++) {
        for (int t = A.lvl_ptr[e] + warp; t < A.lvl_ptr[e + 1]; t += nwarp) {
            const int i = A.rows[t];
            const int q = q0 + i;
            const int rb = A.rp[q], re = A.rp[q + 1], di = A.dpos[q];
            double delta = 0.0;  // MILU: sum of dropped entries (lane 0)
            for (int tk = rb; tk < di; tk++) {
                const int k = A.ci[tk];
                const int qk = q0 + k;
                const double lik = A.f[tk] / A.f[A.dpos[qk]];
                __syncwarp();
                if (lane == 0) A.f[tk] = lik;
                const int ub = A.dpos[qk] + 1, ue = A.rp[qk + 1];
                for (int u0 = ub; u0 < ue; u0 += 32) {
                    const int u = u0 + lane;
                    double prod = 0.0;
                    int pos = -1;
                    const bool act = u < ue;
                    if (act) {
                        const int j = A.ci[u];
                        prod = __dmul_rn(lik, A.f[u]);
                        pos = find_col(A.ci, rb, re, j);
                        if (pos >= 0) A.f[pos] = __dsub_rn(A.f[pos], prod);
                    }
                    unsigned drop = __ballot_sync(kFull, act && pos < 0 && k >= mfrom);
                    while (drop) {  // ascending order of u, like the sequential loop
                        const int b = __ffs(drop) - 1;
                        const double v = __shfl_sync(kFull, prod, b);
                        if (lane == 0) delta = __dsub_rn(delta, v);
                        drop &= drop - 1;
                    }
                }
                __syncwarp();
            }
            double amax = 0.0;
            for (int u = rb + lane; u < re; u += 32) amax = fmax(amax, fabs(A.a[u]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(kFull, amax, o));
            if (lane == 0) {
                double uii = A.f[di];
                if (A.milu) uii = __dadd_rn(uii, delta);
                const double thr = __dmul_rn(A.eps, amax);
                if (A.eps > 0.0 && fabs(uii) < thr) {
                    uii = (uii >= 0.0) ? thr : -thr;
                    atomicAdd(A.npert, 1);
                }
                if (uii == 0.0) atomicOr(A.err, 1);
                A.f[di] = uii;
            }
            __syncwarp();
        }
        __syncthreads();
    }
}

cudaError_t launch_ilu_numeric(const Handle& h, double* F, int milu, cudaStream_t st) {
    NumArgs a;
    a.qoff = h.d_qoff;
    a.rp = h.d_q_rp;
    a.ci = h.d_q_ci;
    a.dpos = h.d_q_dpos;
    a.sub_lvl = h.d_num_sub;
    a.lvl_ptr = h.d_num_lvl;
    a.rows = h.d_num_row;
    a.a = h.d_vals + h.a_base;
    a.f = F;
    a.eps = h.o.pivot_eps;
    a.milu = milu;
    a.nint = h.d_nint;
    a.npert = h.d_npert;
    a.err = h.d_err;
    cudaError_t e = cudaMemcpyAsync(F, a.a, (size_t)h.q_rp[h.n] * sizeof(double),
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    k_ilu_numeric<<<h.p, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// pack: pval[e] = vals[psrc[e]]; pdinv[k] = 1 / vals[pdsrc[k]] (1 for unit rows)
template <class T>
__global__ void k_pack(int64_t nent, int64_t nrow, const int32_t* __restrict__ psrc,
                       const int32_t* __restrict__ pdsrc, const double* __restrict__ vals, T* pval,
                       T* pdinv) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = tid; e < nent; e += stride) pval[e] = (T)vals[psrc[e]];
    for (int64_t k = tid; k < nrow; k += stride) {
        const int32_t d = pdsrc[k];
        pdinv[k] = (d >= 0) ? (T)(1.0 / vals[d]) : (T)1;
    }
}

template <class T>
cudaError_t launch_pack(const ProgHost& ph, const int32_t* d_psrc, const int32_t* d_pdsrc,
                        const double* vals, T* pval, T* pdinv, cudaStream_t st) {
    const int64_t ne = (int64_t)ph.pcol.size(), nr = (int64_t)ph.prow.size();
    if (ne == 0 && nr == 0) return cudaSuccess;
    k_pack<T><<<1024, 256, 0, st>>>(ne, nr, d_psrc, d_pdsrc, vals, pval, pdinv);
    return cudaGetLastError();
}

template cudaError_t launch_pack<float>(const ProgHost&, const int32_t*, const int32_t*, const double*,
                                        float*, float*, cudaStream_t);
template cudaError_t launch_pack<double>(const ProgHost&, const int32_t*, const int32_t*, const double*,
                                         double*, double*, cudaStream_t);

}  // namespace ilu2l
