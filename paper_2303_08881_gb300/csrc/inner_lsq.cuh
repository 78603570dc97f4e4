// inner_lsq.cuh -- least squares of the inner (Schur-level) GMRES, shared by the apply
// kernels: Givens rotations on the small Hessenberg matrix and back substitution,
// computed redundantly by thread 0 of every CTA from the device state the step kernels
// left; the Krylov coefficients t[] end up in shared memory.
#pragma once

#include "devutil.cuh"
#include "internal.h"

namespace ilu2l {

// Least squares of the inner GMRES (Givens rotations, back substitution), computed
// redundantly in every CTA into t[] (shared); returns the step count. The block copies
// the Hessenberg columns and warp 0 forms the last norm; thread 0 then rotates, in the
// arithmetic type A: FP32 for the FP32 preconditioner (the inner GMRES is part of it and
// its vectors carry FP32 accuracy; GB300's FP64 pipe makes each dependent FP64 operation of
// this sequential code cost ~100 cycles), FP64 otherwise.
template <class A>
static __device__ __noinline__ int inner_lsq(const InnerCtl* ctl, const double* part, int p, int k, double* t) {
    __shared__ A Hs[(kMaxInner + 1) * kMaxInner];
    __shared__ A g[kMaxInner + 1], cs[kMaxInner], sn[kMaxInner], ts[kMaxInner];
    __shared__ A last_nrm;
    __shared__ int steps_s;
    for (int i = threadIdx.x; i < (kMaxInner + 1) * k; i += blockDim.x) Hs[i] = (A)ctl->H[i];
    if (threadIdx.x < 32) {
        const double nrm2 = warp_allsum_ldcg(part + ((size_t)(2 * (kMaxInner + 1))) * p, p);
        if (threadIdx.x == 0) last_nrm = sqrt((A)nrm2);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int steps = ctl->steps;
        const int zero = ctl->zero;
        if (zero) {
            steps = 0;
        } else if (steps < 0) {  // ran all k steps: the last norm is still in the partials
            Hs[(k - 1) * (kMaxInner + 1) + k] = last_nrm;
            steps = k;
        }
        for (int i = 0; i <= kMaxInner; i++) g[i] = (A)0;
        g[0] = zero ? (A)0 : (A)ctl->beta;
        for (int j = 0; j < steps; j++) {
            A* col = Hs + j * (kMaxInner + 1);
            for (int i = 0; i < j; i++) {
                const A a = cs[i] * col[i] + sn[i] * col[i + 1];
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
                col[i] = a;
            }
            const A d = sqrt(col[j] * col[j] + col[j + 1] * col[j + 1]);
            if (d == (A)0) {
                cs[j] = (A)1;
                sn[j] = (A)0;
            } else {
                const A rd = (A)1 / d;
                cs[j] = col[j] * rd;
                sn[j] = col[j + 1] * rd;
            }
            col[j] = cs[j] * col[j] + sn[j] * col[j + 1];
            col[j + 1] = (A)0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
        }
        for (int i = steps - 1; i >= 0; i--) {
            A acc = g[i];
            for (int l = i + 1; l < steps; l++) acc -= Hs[l * (kMaxInner + 1) + i] * ts[l];
            ts[i] = acc / Hs[i * (kMaxInner + 1) + i];
        }
        for (int i = 0; i < steps; i++) t[i] = (double)ts[i];
        steps_s = steps;
    }
    __syncthreads();
    return steps_s;
}

}  // namespace ilu2l
