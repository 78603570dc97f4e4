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
// the Hessenberg columns and warp 0 forms the last norm; thread 0 then rotates.
static __device__ __noinline__ int inner_lsq(const InnerCtl* ctl, const double* part, int p, int k, double* t) {
    __shared__ double Hs[(kMaxInner + 1) * kMaxInner];
    __shared__ double g[kMaxInner + 1], cs[kMaxInner], sn[kMaxInner];
    __shared__ double last_nrm;
    __shared__ int steps_s;
    for (int i = threadIdx.x; i < (kMaxInner + 1) * k; i += blockDim.x) Hs[i] = ctl->H[i];
    if (threadIdx.x < 32) {
        const double nrm2 = warp_allsum_ldcg(part + ((size_t)(2 * (kMaxInner + 1))) * p, p);
        if (threadIdx.x == 0) last_nrm = sqrt(nrm2);
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
        for (int i = 0; i <= kMaxInner; i++) g[i] = 0.0;
        g[0] = zero ? 0.0 : ctl->beta;
        for (int j = 0; j < steps; j++) {
            double* col = Hs + j * (kMaxInner + 1);
            for (int i = 0; i < j; i++) {
                const double a = cs[i] * col[i] + sn[i] * col[i + 1];
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
                col[i] = a;
            }
            const double d = sqrt(col[j] * col[j] + col[j + 1] * col[j + 1]);
            if (d == 0.0) {
                cs[j] = 1.0;
                sn[j] = 0.0;
            } else {
                cs[j] = col[j] / d;
                sn[j] = col[j + 1] / d;
            }
            col[j] = cs[j] * col[j] + sn[j] * col[j + 1];
            col[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
        }
        for (int i = steps - 1; i >= 0; i--) {
            double acc = g[i];
            for (int l = i + 1; l < steps; l++) acc -= Hs[l * (kMaxInner + 1) + i] * t[l];
            t[i] = acc / Hs[i * (kMaxInner + 1) + i];
        }
        steps_s = steps;
    }
    __syncthreads();
    return steps_s;
}

}  // namespace ilu2l
