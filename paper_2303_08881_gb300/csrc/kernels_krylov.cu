// kernels_krylov.cu -- FP64 CSR SpMV and the flexible GMRES(m) kernels (Sec. 4.1.1: the
// outer Krylov method is FGMRES because the inner Schur GMRES makes M^{-1} vary).
//
// Every kernel partitions the n rows into G contiguous CTA ranges. Reductions write one
// partial per CTA, combined in a fixed order (by the last CTA to finish, or in two levels
// through groups of CTAs), so every result is independent of timing. The Arnoldi state
// (Hessenberg, Givens rotations, residual estimate, the cycle flag) lives on the device: the
// host reads it once per cycle.
//
// One Arnoldi step j (after z_j = M^{-1} v_j):
//   k_fg_spmv_dot  w = A z_j and the first Gram-Schmidt dots V_{0..j}^T w (FP32 copies
//                  of V and w by default: the second pass corrects their error)
//   k_fg_cgs       w -= V h1 and the reorthogonalisation dots V^T w (FP64), or
//   k_fg_cgs_df    the same in double-float from a two-term FP32 split of V (the default),
//                  with ||w1||^2 and, from ||w1||^2 - ||h2||^2, the new norm
//   k_fg_norm      w -= V h2 (from the FP32 copy of V by default: h2 is then small), ||w||,
//                  Givens rotation, residual estimate, stop decision; with k_fg_cgs_df only
//                  when its norm cancels
//   k_fg_next      v_{j+1} = w / ||w||; after k_fg_cgs_df it forms w = w1 - V h2 itself, and
//                  its CTA 0 takes the Givens rotation, estimate and stop decision
#include <algorithm>

#include "devutil.cuh"
#include "handle.h"

namespace ilu2l {

constexpr int kMaxJ = 255;  // basis vectors a Gram-Schmidt kernel handles (restart <= 256)

// CTA row slices: multiples of 64 rows, so every slice starts 512-byte aligned in a
// basis vector (leading dimension a multiple of 64) and pairs of rows load as 128 bits.
__device__ __forceinline__ void cta_rows(int n, int& r0, int& r1) {
    const int R = ((n + gridDim.x - 1) / gridDim.x + 63) / 64 * 64;
    r0 = min(n, blockIdx.x * R);
    r1 = min(n, r0 + R);
}

__device__ __forceinline__ double2 ld2(const double* p) { return *reinterpret_cast<const double2*>(p); }

// y_r = A_r . x with VL lanes per row; result valid in the row's first lane. Every lane
// of the warp must call it (the shuffles use the full mask); lanes of an out-of-range row
// pass valid = false.
template <int VL>
__device__ __forceinline__ double row_dot(const CsrDev& A, int r, bool valid, const double* __restrict__ x,
                                          int sl) {
    double s = 0.0;
    if (valid) {
        const int e = A.rp[r + 1];
        for (int q = A.rp[r] + sl; q < e; q += VL) s += A.v[q] * x[A.ci[q]];
    }
#pragma unroll
    for (int o = VL / 2; o > 0; o >>= 1) s += __shfl_down_sync(kFull, s, o, VL);
    return s;
}

// Last CTA ticket: returns true in every thread of the last CTA to arrive.
__device__ __forceinline__ bool last_cta(uint32_t* counter) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// In the last CTA: out[i] = sum_c part[i*G + c] for i < m, fixed order. Lane l of the warp
// that takes coefficient i sums partials l, l + 32, ... in groups of eight loads issued
// together (one L2 round trip per group instead of one per partial), then the warp adds its
// lanes. With addto, the sum is also added to addto[i] (by the same lane, in parallel).
__device__ __forceinline__ void reduce_partials(const double* part, int G, int m, double* out,
                                                double* addto = nullptr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < m; i += nw) {
        const double* p = part + (size_t)i * G;
        double s = 0.0;
        for (int c0 = lane; c0 < G; c0 += 256) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; u++) v[u] = (c0 + 32 * u < G) ? __ldcg(p + c0 + 32 * u) : 0.0;
#pragma unroll
            for (int u = 0; u < 8; u++) s += v[u];
        }
        s = warp_sum(s);
        if (lane == 0) {
            out[i] = s;
            if (addto) addto[i] += s;
        }
    }
    __syncthreads();
}

// Two-level form of last_cta + reduce_partials for the Gram-Schmidt kernels. The last CTA to
// arrive in each group of kRedGroup consecutive CTAs sums the group's partials (lane c of the
// warp that takes coefficient i adds CTA c of the group, then the warp's lanes), and the last
// group to finish sums the group sums in group order. GB300 issues FP64 adds at 1/64 of its
// FP32 rate, so one CTA summing every partial (m x G adds on one SM) was the kernels' tail;
// here each level is a few FP64 adds per lane. Returns true in every thread of the CTA that
// holds the final sums (out[i], and addto[i] += out[i] when addto is given); the counters are
// back at zero when the kernel ends.
__device__ __forceinline__ bool reduce_two_level(const FgDev& f, int m, double* out, double* addto = nullptr) {
    const int G = f.G, ng = (G + kRedGroup - 1) / kRedGroup, g = blockIdx.x / kRedGroup;
    const int c0 = g * kRedGroup, cn = min(G, c0 + kRedGroup) - c0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __shared__ bool last_s;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last_s = (atomicAdd(&f.gcount[g], 1u) == (uint32_t)cn - 1);
    __syncthreads();
    if (!last_s) return false;
    __threadfence();
    for (int i = warp; i < m; i += nw) {
        double v = lane < cn ? __ldcg(f.part + (size_t)i * G + c0 + lane) : 0.0;
        v = warp_sum(v);
        if (lane == 0) f.gpart[(size_t)i * ng + g] = v;
    }
    if (threadIdx.x == 0) f.gcount[g] = 0;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last_s = (atomicAdd(&f.ctl->counter, 1u) == (uint32_t)ng - 1);
    __syncthreads();
    if (!last_s) return false;
    __threadfence();
    for (int i = warp; i < m; i += nw) {
        double v = 0.0;
        for (int q = lane; q < ng; q += 32) v += __ldcg(f.gpart + (size_t)i * ng + q);
        v = warp_sum(v);
        if (lane == 0) {
            out[i] = v;
            if (addto) addto[i] += v;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) f.ctl->counter = 0;
    return true;
}

// ---------------------------------------------------------------------------------------
template <int VL>
__global__ void k_spmv(CsrDev A, const double* __restrict__ x, double* __restrict__ y) {
    const int per_block = blockDim.x / VL;  // rows per block per pass (uniform trip count)
    const int sub = threadIdx.x / VL, sl = threadIdx.x & (VL - 1);
    for (int base = blockIdx.x * per_block; base < A.n; base += gridDim.x * per_block) {
        const int r = base + sub;
        const bool valid = r < A.n;
        const double s = row_dot<VL>(A, r, valid, x, sl);
        if (valid && sl == 0) y[r] = s;
    }
}

// r = b - A x into V[0]; ||r||^2 (and ||b||^2 on the first call); cycle set-up
template <int VL>
__global__ void k_fg_resid(CsrDev A, FgDev f, const double* __restrict__ b, const double* __restrict__ x,
                           int first) {
    __shared__ double red[64];
    __shared__ double tot[2];
    int r0, r1;
    cta_rows(A.n, r0, r1);
    const int sl = threadIdx.x & (VL - 1), sub = threadIdx.x / VL, nsub = blockDim.x / VL;
    double rr = 0.0, bb = 0.0;
    for (int base = r0; base < r1; base += nsub) {
        const int r = base + sub;
        const bool valid = r < r1;
        const double ax = row_dot<VL>(A, r, valid, x, sl);
        if (valid && sl == 0) {
            const double rv = b[r] - ax;
            f.V[r] = rv;
            rr += rv * rv;
            bb += b[r] * b[r];
        }
    }
    double v2[2] = {rr, bb};
    block_sum_n<2>(v2, red);
    if (threadIdx.x == 0) {
        f.part[blockIdx.x] = v2[0];
        f.part[(size_t)f.G + blockIdx.x] = v2[1];
    }
    if (!last_cta(&f.ctl->counter)) return;
    reduce_partials(f.part, f.G, 2, tot);
    if (threadIdx.x == 0) {
        FgCtl* c = f.ctl;
        c->counter = 0;
        if (first) {
            c->bnorm = sqrt(tot[1]);
            c->target = c->rtol * c->bnorm;
            c->total = 0;
            c->converged = 0;
            c->breakdown = 0;
        }
        const double beta = sqrt(tot[0]);
        c->beta = beta;
        f.hnext[1] = beta > 0.0 ? 1.0 / beta : 0.0;  // for k_fg_scale0 (one FP64 division)
        c->res_true = beta;
        c->steps = 0;
        c->est = beta;
        if (c->bnorm == 0.0 || beta <= c->target) {
            c->converged = 1;
            c->cycle_done = 1;
        } else if (c->total >= c->maxit) {
            c->cycle_done = 1;
        } else {
            c->cycle_done = 0;
            for (int i = 0; i <= f.m; i++) f.g[i] = 0.0;
            f.g[0] = beta;
        }
    }
}

// ---- double-float arithmetic (Dekker 1971): a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits. Every operation below is
// an explicitly rounded intrinsic, so the compiler cannot contract a product into a sum and
// break the error-free transformations.

// x ~ hi + lo: hi = fl32(x), lo = fl32(x - hi) (x - hi is exact in FP64)
__device__ __forceinline__ void df_split(double x, float& hi, float& lo) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(__dsub_rn(x, (double)hi));
}

// Knuth's TwoSum: s + e = a + b exactly, s = fl(a + b)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// (sh, sl) += (ah + al) * (bh + bl). The leading product ah * bh is split exactly into
// p + e with one FMA (the TwoProduct of Ogita, Rump and Oishi, 2005); the cross terms
// ah * bl + al * bh join e in FP32 (they are 2^-24 of the product, so their rounding is
// 2^-48 of it) and al * bl is below that and left out. p goes into sh by TwoSum; its error
// and e accumulate in sl, which df_renorm folds back from time to time.
__device__ __forceinline__ void df_mac(float& sh, float& sl, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    float t, err;
    two_sum(sh, p, t, err);
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(err, e));
}

// restore |sl| <= ulp(sh) / 2 (TwoSum: no assumption on the sizes)
__device__ __forceinline__ void df_renorm(float& sh, float& sl) {
    float t, e;
    two_sum(sh, sl, t, e);
    sh = t;
    sl = e;
}

// (ah, al) += (bh, bl), both double-float
__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    two_sum(s, e, ah, al);
}

// sum of a double-float value over the 32 lanes of a warp (butterfly: every lane ends with
// the same bits, TwoSum being exact whatever the order of its operands)
__device__ __forceinline__ void df_warp_sum(float& h, float& l) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float bh = __shfl_xor_sync(kFull, h, o), bl = __shfl_xor_sync(kFull, l, o);
        df_add(h, l, bh, bl);
    }
}

// basis entry i (offset into V) in its FP32 forms: the rounded copy V32 and, with the
// double-float second pass, the remainder Vlo
__device__ __forceinline__ void store_basis32(const FgDev& f, size_t i, double v) {
    if (f.Vlo) {
        float hi, lo;
        df_split(v, hi, lo);
        f.V32[i] = hi;
        f.Vlo[i] = lo;
    } else {
        f.V32[i] = (float)v;
    }
}

__global__ void k_fg_scale0(FgDev f, int n) {
    if (f.ctl->cycle_done) return;
    const double inv = __ldcg(f.hnext + 1);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const double v = f.V[r] * inv;
        f.V[r] = v;
        if (f.V32) store_basis32(f, r, v);
    }
}

// Gram-Schmidt kernels. Each CTA owns a row slice (cta_rows). FP64 arithmetic is the
// bound on GB300 (2 fused multiply-adds per SM per clock), so the loops spend as few
// instructions per multiply-add as they can: 128-bit loads of row pairs, long contiguous
// streams per warp, several loads in flight.
//  * Dots V_i . w: tasks (basis vector i, sub-slice) taken by the warps in turn; a warp
//    streams one vector over its sub-slice (four row pairs per lane in flight) and leaves
//    one partial; the sub-slice partials of a vector are added in order.
//  * Updates w -= V h: one row pair per thread, eight basis vectors in flight, the terms
//    subtracted in the order i = 0..j.
// dot tasks per CTA: (j + 1) * max(1, nw / (j + 1)) <= max(j + 1, nw), nw <= 8 warps
constexpr int kMaxTasks = (kMaxJ + 1 > 8) ? kMaxJ + 1 : 8;

// spart[i] (i <= j, shared) = sum over the CTA's rows of V_i[r] w[r]
__device__ __forceinline__ void cta_dots(const double* __restrict__ V, int64_t ld, const double* w, int r0, int r1,
                                         int j, double* spart, double* stask) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nsub = max(1, nw / (j + 1));
    const int len = ((r1 - r0 + nsub - 1) / nsub + 63) / 64 * 64;
    for (int task = warp; task < (j + 1) * nsub; task += nw) {
        const int i = task / nsub, sb = task - i * nsub;
        const int a = min(r1, r0 + sb * len), b = min(r1, a + len);
        const double* __restrict__ v = V + (size_t)i * ld;
        double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        int r = a + 2 * lane;
        for (; r + 193 < b; r += 256) {
            double2 x[4], y[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                x[k] = ld2(v + r + 64 * k);
                y[k] = ld2(w + r + 64 * k);
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                acc[2 * k] += x[k].x * y[k].x;
                acc[2 * k + 1] += x[k].y * y[k].y;
            }
        }
        for (; r + 1 < b; r += 64) {
            const double2 x = ld2(v + r), y = ld2(w + r);
            acc[0] += x.x * y.x;
            acc[1] += x.y * y.y;
        }
        if (r < b) acc[0] += v[r] * w[r];  // the last row of an odd slice
        double t = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
        t = warp_sum(t);
        if (lane == 0) stask[task] = t;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        double t = 0.0;
        for (int sb = 0; sb < nsub; sb++) t += stask[i * nsub + sb];
        spart[i] = t;
    }
    __syncthreads();
}

__device__ __forceinline__ float4 ld4f(const float* p) { return *reinterpret_cast<const float4*>(p); }

// The dots of the first Gram-Schmidt pass from the FP32 copies (FgDev::V32, w32): FP32
// products summed per lane and warp in FP32, the CTA's partial per vector in FP64. The
// second pass, in FP64, removes from w what this estimate leaves (about 6e-8 ||w||), so
// only the coefficients' first ~7 digits matter here. Same task split as cta_dots, four
// rows per lane and load (slices start at multiples of 64 rows: 16-byte aligned).
__device__ __forceinline__ void cta_dots32(const float* __restrict__ V32, int64_t ld, const float* w32, int r0,
                                           int r1, int j, double* spart, double* stask) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nsub = max(1, nw / (j + 1));
    const int len = ((r1 - r0 + nsub - 1) / nsub + 127) / 128 * 128;
    for (int task = warp; task < (j + 1) * nsub; task += nw) {
        const int i = task / nsub, sb = task - i * nsub;
        const int a = min(r1, r0 + sb * len), b = min(r1, a + len);
        const float* __restrict__ v = V32 + (size_t)i * ld;
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int r = a + 4 * lane;
        for (; r + 131 < b; r += 256) {
            const float4 x0 = ld4f(v + r), y0 = ld4f(w32 + r), x1 = ld4f(v + r + 128), y1 = ld4f(w32 + r + 128);
            acc[0] += x0.x * y0.x;
            acc[1] += x0.y * y0.y;
            acc[2] += x0.z * y0.z;
            acc[3] += x0.w * y0.w;
            acc[4] += x1.x * y1.x;
            acc[5] += x1.y * y1.y;
            acc[6] += x1.z * y1.z;
            acc[7] += x1.w * y1.w;
        }
        for (; r + 3 < b; r += 128) {
            const float4 x0 = ld4f(v + r), y0 = ld4f(w32 + r);
            acc[0] += x0.x * y0.x;
            acc[1] += x0.y * y0.y;
            acc[2] += x0.z * y0.z;
            acc[3] += x0.w * y0.w;
        }
        for (int q = r; q < b && q < r + 4; q++) acc[0] += v[q] * w32[q];  // the slice's last rows
        float t = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
        t = warp_sum_t<float>(t);
        if (lane == 0) stask[task] = (double)t;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        double t = 0.0;
        for (int sb = 0; sb < nsub; sb++) t += stask[i * nsub + sb];
        spart[i] = t;
    }
    __syncthreads();
}

// w[r] -= sum_i h[i] V_i[r] over the CTA's rows (i = 0..j in order); optionally the
// partial ||w||^2
__device__ __forceinline__ void cta_update(const double* __restrict__ V, int64_t ld, double* w, const double* hh,
                                           int r0, int r1, int j, double* nrm2) {
    double acc = 0.0;
    for (int r = r0 + 2 * threadIdx.x; r < r1; r += 2 * blockDim.x) {
        const bool pair = r + 1 < r1;
        double2 x = pair ? ld2(w + r) : make_double2(w[r], 0.0);
        int i = 0;
        for (; i + 8 <= j + 1; i += 8) {
            double2 v[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const double* p = V + (size_t)(i + u) * ld + r;
                v[u] = pair ? ld2(p) : make_double2(*p, 0.0);
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                x.x -= hh[i + u] * v[u].x;
                x.y -= hh[i + u] * v[u].y;
            }
        }
        for (; i <= j; i++) {
            const double* p = V + (size_t)i * ld + r;
            const double2 v = pair ? ld2(p) : make_double2(*p, 0.0);
            x.x -= hh[i] * v.x;
            x.y -= hh[i] * v.y;
        }
        if (pair) {
            *reinterpret_cast<double2*>(w + r) = x;
            acc += x.x * x.x + x.y * x.y;
        } else {
            w[r] = x.x;
            acc += x.x * x.x;
        }
    }
    if (nrm2) *nrm2 = acc;
}

// w[r] -= sum_i hf[i] V32_i[r] with FP32 products summed in FP32 (i = 0..j in order), the
// correction subtracted from w in FP64; optionally the partial ||w||^2 in FP64. For the second
// Gram-Schmidt pass only, whose coefficients are ~6e-8 ||w|| after an FP32 first pass: the
// correction's own error, ~1e-7 of it, is then ~1e-14 ||w||. Four rows per thread (float4 of
// the copy, two double2 of w; slices start at multiples of 64 rows).
__device__ __forceinline__ void cta_update32(const float* __restrict__ V32, int64_t ld, double* w, const float* hf,
                                             int r0, int r1, int j, double* nrm2) {
    double acc2 = 0.0;
    for (int r = r0 + 4 * threadIdx.x; r < r1; r += 4 * blockDim.x) {
        if (r + 3 < r1) {
            float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
            int i = 0;
            for (; i + 8 <= j + 1; i += 8) {
                float4 v[8];
#pragma unroll
                for (int u = 0; u < 8; u++) v[u] = ld4f(V32 + (size_t)(i + u) * ld + r);
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const float hv = hf[i + u];
                    c.x += hv * v[u].x;
                    c.y += hv * v[u].y;
                    c.z += hv * v[u].z;
                    c.w += hv * v[u].w;
                }
            }
            for (; i <= j; i++) {
                const float4 v = ld4f(V32 + (size_t)i * ld + r);
                const float hv = hf[i];
                c.x += hv * v.x;
                c.y += hv * v.y;
                c.z += hv * v.z;
                c.w += hv * v.w;
            }
            double2 a = ld2(w + r), b = ld2(w + r + 2);
            a.x -= (double)c.x;
            a.y -= (double)c.y;
            b.x -= (double)c.z;
            b.y -= (double)c.w;
            *reinterpret_cast<double2*>(w + r) = a;
            *reinterpret_cast<double2*>(w + r + 2) = b;
            acc2 += (a.x * a.x + a.y * a.y) + (b.x * b.x + b.y * b.y);
        } else {
            for (int q = r; q < r1; q++) {
                float c = 0.f;
                for (int i = 0; i <= j; i++) c += hf[i] * V32[(size_t)i * ld + q];
                const double x = w[q] - (double)c;
                w[q] = x;
                acc2 += x * x;
            }
        }
    }
    if (nrm2) *nrm2 = acc2;
}

// the CTA's partials of coefficients 0..j into part[u * G + cta]
__device__ __forceinline__ void cta_partials(const double* spart, int j, double* part, int G) {
    for (int u = threadIdx.x; u <= j; u += blockDim.x) part[(size_t)u * G + blockIdx.x] = spart[u];
}

// w = A z_j and the first Gram-Schmidt dots V_{0..j}^T w (from the FP32 copies when they
// exist); the last CTA stores h1 in column j of H
template <int VL>
__global__ void __launch_bounds__(256) k_fg_spmv_dot(CsrDev A, FgDev f, int j) {
    __shared__ double stask[kMaxTasks];
    __shared__ double spart[kMaxJ + 1];
    if (f.ctl->cycle_done) return;
    int r0, r1;
    cta_rows(A.n, r0, r1);
    const double* __restrict__ zj = f.Z + (size_t)j * f.ld;
    const int sl = threadIdx.x & (VL - 1), sub = threadIdx.x / VL, nsub = blockDim.x / VL;
    for (int base = r0; base < r1; base += nsub) {
        const int r = base + sub;
        const bool valid = r < r1;
        const double s = row_dot<VL>(A, r, valid, zj, sl);
        if (valid && sl == 0) {
            f.w[r] = s;
            if (f.w32) f.w32[r] = (float)s;
        }
    }
    __syncthreads();
    if (f.V32)
        cta_dots32(f.V32, f.ld, f.w32, r0, r1, j, spart, stask);
    else
        cta_dots(f.V, f.ld, f.w, r0, r1, j, spart, stask);
    cta_partials(spart, j, f.part, f.G);
    reduce_two_level(f, j + 1, f.H + (size_t)j * (f.m + 1));
}

// w -= V h1 (h1 = column j of H) and the reorthogonalisation dots V^T w; the last CTA
// adds them to column j and keeps them in f.h2 for k_fg_norm
__global__ void __launch_bounds__(256) k_fg_cgs(FgDev f, int n, int j) {
    __shared__ double stask[kMaxTasks];
    __shared__ double spart[kMaxJ + 1];
    __shared__ double hh[kMaxJ + 1];
    if (f.ctl->cycle_done) return;
    int r0, r1;
    cta_rows(n, r0, r1);
    const double* Hj = f.H + (size_t)j * (f.m + 1);
    for (int u = threadIdx.x; u <= j; u += blockDim.x) hh[u] = __ldcg(Hj + u);
    __syncthreads();
    cta_update(f.V, f.ld, f.w, hh, r0, r1, j, nullptr);
    __syncthreads();
    cta_dots(f.V, f.ld, f.w, r0, r1, j, spart, stask);
    cta_partials(spart, j, f.part, f.G);
    reduce_two_level(f, j + 1, f.h2, f.H + (size_t)j * (f.m + 1));
}

// k_fg_cgs in double-float arithmetic from the split basis V32 + Vlo (gs_precision 3):
// w -= V h1 and the reorthogonalisation dots V^T w without FP64 operations per basis entry
// (GB300 issues FP32 at 64 times its FP64 rate, so the kernel is bound by reading the basis
// once, 8 bytes per entry, instead of by FP64 fused multiply-adds). The CTA walks its row
// slice in sub-slices of NT rows:
//  * update: thread t takes row t of the sub-slice, sums h1_i (V32 + Vlo)_ir over i = 0..j
//    in double-float (renormalised every 8 terms; 32 loads in flight per thread), subtracts
//    the sum from w_r in FP64, and leaves w_r split in shared memory;
//  * dots: vector i goes to warp i % (NT / 32); lane l adds the row pairs l, l + 32, ... of
//    the sub-slice into its own double-float accumulator for i (shared memory), renormalised
//    after each sub-slice; a warp takes two vectors per pass. The sub-slice's basis entries
//    are read again here, from L1/L2.
// The dots also accumulate ||w1||^2 (w1 against itself, as coefficient j + 1). At the end
// the 32 lane accumulators of each are added by its warp, and the CTA partials are combined
// in a fixed order (reduce_two_level). The last CTA adds h2 to H and, unless the subtraction
// cancels, takes ||w2||^2 = ||w1||^2 - ||h2||^2: k_fg_norm is then skipped, and k_fg_next
// ends the Arnoldi step (fg_step_tail) and forms w2 = w1 - V h2 as it normalises. Error: every
// operation rounds at 2^-48 instead of FP64's 2^-53, so the update and the dots carry
// errors ~(terms) * 2^-48 of the magnitudes summed: ~1e-13 ||w|| for 50 basis vectors,
// far below the ~6e-8 ||w|| the second pass removes.
// Dynamic shared memory: (j + 2) * 32 float2 accumulators (the last for ||w1||^2).
template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_fg_cgs_df(FgDev f, int n, int j) {
    extern __shared__ float2 sacc[];
    __shared__ __align__(16) float2 hcf[kMaxJ + 2];   // h1_i split: (hi, lo)
    __shared__ __align__(16) float4 wpk[NT / 2];     // w of row pair q: (hi 2q, hi 2q+1, lo 2q, lo 2q+1)
    if (f.ctl->cycle_done) return;
    int r0, r1;
    cta_rows(n, r0, r1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = NT / 32, RP = NT / 64;  // row pairs per lane in the dots
    const double* Hj = f.H + (size_t)j * (f.m + 1);
    for (int u = threadIdx.x; u <= j + 1; u += NT) {
        float a = 0.f, b = 0.f;
        if (u <= j) df_split(__ldcg(Hj + u), a, b);
        hcf[u] = make_float2(a, b);
    }
    for (int u = threadIdx.x; u < (j + 2) * 32; u += NT) sacc[u] = make_float2(0.f, 0.f);
    __syncthreads();
    const float* __restrict__ Vh = f.V32;
    const float* __restrict__ Vl = f.Vlo;
    const int64_t ld = f.ld;
    float* wflat = reinterpret_cast<float*>(wpk);
    for (int base = r0; base < r1; base += NT) {
        const int r = base + threadIdx.x;
        float whi = 0.f, wlo = 0.f;
        if (r < r1) {
            float sh = 0.f, sl = 0.f;
            int i = 0;
            for (; i + 16 <= j + 1; i += 16) {
                float vh[16], vl[16];
#pragma unroll
                for (int u = 0; u < 16; u++) {
                    vh[u] = Vh[(size_t)(i + u) * ld + r];
                    vl[u] = Vl[(size_t)(i + u) * ld + r];
                }
#pragma unroll
                for (int u = 0; u < 16; u += 2) {
                    const float4 c = *reinterpret_cast<const float4*>(&hcf[i + u]);  // two coefficients
                    df_mac(sh, sl, c.x, c.y, vh[u], vl[u]);
                    df_mac(sh, sl, c.z, c.w, vh[u + 1], vl[u + 1]);
                    if (u == 6) df_renorm(sh, sl);
                }
                df_renorm(sh, sl);
            }
            if (i + 8 <= j + 1) {
                float vh[8], vl[8];
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    vh[u] = Vh[(size_t)(i + u) * ld + r];
                    vl[u] = Vl[(size_t)(i + u) * ld + r];
                }
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    const float4 c = *reinterpret_cast<const float4*>(&hcf[i + u]);
                    df_mac(sh, sl, c.x, c.y, vh[u], vl[u]);
                    df_mac(sh, sl, c.z, c.w, vh[u + 1], vl[u + 1]);
                }
                df_renorm(sh, sl);
                i += 8;
            }
            for (; i <= j; i++) {
                const float2 c = hcf[i];
                df_mac(sh, sl, c.x, c.y, Vh[(size_t)i * ld + r], Vl[(size_t)i * ld + r]);
            }
            const double w1 = __dsub_rn(f.w[r], __dadd_rn((double)sh, (double)sl));
            f.w[r] = w1;
            df_split(w1, whi, wlo);
            f.w32[r] = whi;  // w1 split, for k_fg_next
            f.wlo[r] = wlo;
        }
        {
            const int t = threadIdx.x;
            wflat[(t >> 1) * 4 + (t & 1)] = whi;
            wflat[(t >> 1) * 4 + 2 + (t & 1)] = wlo;
        }
        __syncthreads();
        // dots: lane l takes the row pairs l, l + 32, ... of the sub-slice (64-bit loads of
        // two rows' parts); two vectors (i and i + NW) per pass so that twice the loads are in
        // flight. Rows past the slice's end (the last sub-slice) are neither loaded nor used.
        const int cnt = min(NT, r1 - base);
        float4 wq[RP];
#pragma unroll
        for (int k = 0; k < RP; k++) wq[k] = wpk[lane + 32 * k];
        for (int i = warp; i <= j; i += 2 * NW) {
            const int i2 = i + NW;
            const bool two = i2 <= j;
            const float* __restrict__ ph = Vh + (size_t)i * ld + base;
            const float* __restrict__ pl = Vl + (size_t)i * ld + base;
            const float* __restrict__ qh = Vh + (size_t)(two ? i2 : i) * ld + base;
            const float* __restrict__ ql = Vl + (size_t)(two ? i2 : i) * ld + base;
            float2 xh[RP], xl[RP], yh[RP], yl[RP];
            if (cnt == NT) {
#pragma unroll
                for (int k = 0; k < RP; k++) {
                    const int q = 2 * (lane + 32 * k);
                    xh[k] = *reinterpret_cast<const float2*>(ph + q);
                    xl[k] = *reinterpret_cast<const float2*>(pl + q);
                    yh[k] = *reinterpret_cast<const float2*>(qh + q);
                    yl[k] = *reinterpret_cast<const float2*>(ql + q);
                }
            } else {
#pragma unroll
                for (int k = 0; k < RP; k++) {
                    const int q = 2 * (lane + 32 * k);
                    const bool a0 = q < cnt, a1 = q + 1 < cnt;
                    xh[k] = make_float2(a0 ? ph[q] : 0.f, a1 ? ph[q + 1] : 0.f);
                    xl[k] = make_float2(a0 ? pl[q] : 0.f, a1 ? pl[q + 1] : 0.f);
                    yh[k] = make_float2(a0 ? qh[q] : 0.f, a1 ? qh[q + 1] : 0.f);
                    yl[k] = make_float2(a0 ? ql[q] : 0.f, a1 ? ql[q + 1] : 0.f);
                }
            }
            float2 a = sacc[i * 32 + lane];
#pragma unroll
            for (int k = 0; k < RP; k++) {
                df_mac(a.x, a.y, xh[k].x, xl[k].x, wq[k].x, wq[k].z);
                df_mac(a.x, a.y, xh[k].y, xl[k].y, wq[k].y, wq[k].w);
            }
            df_renorm(a.x, a.y);
            sacc[i * 32 + lane] = a;
            if (two) {
                float2 c = sacc[i2 * 32 + lane];
#pragma unroll
                for (int k = 0; k < RP; k++) {
                    df_mac(c.x, c.y, yh[k].x, yl[k].x, wq[k].x, wq[k].z);
                    df_mac(c.x, c.y, yh[k].y, yl[k].y, wq[k].y, wq[k].w);
                }
                df_renorm(c.x, c.y);
                sacc[i2 * 32 + lane] = c;
            }
        }
        if (warp == (j + 1) % NW) {  // ||w1||^2 as accumulator j + 1 (rows past the slice are zero)
            float2 a = sacc[(j + 1) * 32 + lane];
#pragma unroll
            for (int k = 0; k < RP; k++) {
                df_mac(a.x, a.y, wq[k].x, wq[k].z, wq[k].x, wq[k].z);
                df_mac(a.x, a.y, wq[k].y, wq[k].w, wq[k].y, wq[k].w);
            }
            df_renorm(a.x, a.y);
            sacc[(j + 1) * 32 + lane] = a;
        }
        __syncthreads();
    }
    // the lanes' accumulators of a vector summed in double-float by its warp (FP32 shuffles
    // and adds; an FP64 warp sum per vector kept GB300's FP64 pipe a third busy), then one
    // conversion to the FP64 partial
    // (coefficient j + 1: the CTA's ||w1||^2)
    for (int i = warp; i <= j + 1; i += NW) {
        float2 a = sacc[i * 32 + lane];
        df_warp_sum(a.x, a.y);
        if (lane == 0) f.part[(size_t)i * f.G + blockIdx.x] = __dadd_rn((double)a.x, (double)a.y);
    }
    if (!reduce_two_level(f, j + 2, f.h2)) return;
    // the last CTA: h2 into column j of H, and ||w2||^2 = ||w1||^2 - ||h2||^2 (w1 = w2 + V h2,
    // V h2 orthogonal to w2). Without cancellation this ends the step here and k_fg_next forms
    // w2; otherwise k_fg_norm forms w2 and its norm explicitly.
    double* col = f.H + (size_t)j * (f.m + 1);
    for (int i = threadIdx.x; i <= j; i += NT) col[i] += __ldcg(f.h2 + i);
    if (warp == 0) {
        double hs = 0.0;
        for (int i = lane; i <= j; i += 32) {
            const double h = __ldcg(f.h2 + i);
            hs += h * h;
        }
        hs = warp_sum(hs);
        if (lane == 0) {
            const double a = __ldcg(f.h2 + j + 1), d = a - hs;
            const int fu = d > 1e-2 * a;
            f.ctl->fuse = fu;
            if (fu) {  // the norm and its inverse for k_fg_next, whose CTA 0 ends the step
                const double hn = sqrt(d);
                f.hnext[0] = hn;
                f.hnext[1] = 1.0 / hn;
            }
        }
    }
}

constexpr int kCgsDfThreads = 256;

// Back substitution R y = g for the cycle's `steps` coefficients, by the whole CTA (one
// thread per row, steps <= blockDim.x): column i of R (contiguous in H) is applied as soon as
// y_i is known, and every thread prefetches its entry of the next column while the current
// one is applied, so each of the `steps` rounds costs a block barrier, not a global-memory
// round trip. rlast: column steps - 1 (held in shared memory by the caller); g: shared.
__device__ __forceinline__ void solve_upper(const FgDev& f, int steps, const double* rlast, const double* g,
                                            double* ys) {
    const int l = threadIdx.x;
    double gl = (l < steps) ? g[l] : 0.0;
    double rnext = (l < steps) ? rlast[l] : 0.0;
    for (int i = steps - 1; i >= 0; i--) {
        const double rc = rnext;  // R[l][i], the entry of column i in row l
        if (i > 0 && l < i) rnext = __ldcg(f.H + (size_t)(i - 1) * (f.m + 1) + l);
        if (l == i) ys[i] = gl / rc;
        __syncthreads();
        if (l < i) gl -= rc * ys[i];
    }
    __syncthreads();
}

// The end of Arnoldi step j, by the whole last CTA of a kernel, given hn = ||w2|| = h_{j+1,j}:
// the new Hessenberg column, the earlier rotations and g go to shared memory in parallel,
// thread 0 applies the rotations there, the results go back in parallel; then the estimate,
// the stop decision, the norm and its inverse for k_fg_next and, when the cycle ends, R y = g
// for k_fg_update.
__device__ __forceinline__ void fg_step_tail(const FgDev& f, int j, double hn) {
    __shared__ double scol[kMaxJ + 2], scs[kMaxJ + 1], ssn[kMaxJ + 1], sg[kMaxJ + 2];
    __shared__ double ys[kMaxJ + 1];
    __shared__ int done_s;
    const int m1 = f.m + 1;
    double* col = f.H + (size_t)j * m1;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        scol[i] = __ldcg(col + i);
        sg[i] = __ldcg(f.g + i);
        if (i < j) {
            scs[i] = __ldcg(f.cs + i);
            ssn[i] = __ldcg(f.sn + i);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        FgCtl* c = f.ctl;
        scol[j + 1] = hn;
        for (int i = 0; i < j; i++) {
            const double a = scs[i] * scol[i] + ssn[i] * scol[i + 1];
            scol[i + 1] = -ssn[i] * scol[i] + scs[i] * scol[i + 1];
            scol[i] = a;
        }
        const double d = sqrt(scol[j] * scol[j] + scol[j + 1] * scol[j + 1]);
        double cj, sj;
        if (d == 0.0) {
            cj = 1.0;
            sj = 0.0;
        } else {
            cj = scol[j] / d;
            sj = scol[j + 1] / d;
        }
        f.cs[j] = cj;
        f.sn[j] = sj;
        scol[j] = cj * scol[j] + sj * scol[j + 1];
        scol[j + 1] = 0.0;
        sg[j + 1] = -sj * sg[j];
        sg[j] = cj * sg[j];
        f.g[j + 1] = sg[j + 1];
        f.g[j] = sg[j];
        c->total += 1;
        c->steps = j + 1;
        c->est = fabs(sg[j + 1]);
        f.hnext[0] = hn;  // norm of the new basis vector and its inverse, for k_fg_next
        f.hnext[1] = hn > 0.0 ? 1.0 / hn : 0.0;
        int done = 0;
        if (c->est <= c->target || hn == 0.0 || c->total >= c->maxit || j + 1 == f.m) {
            c->cycle_done = 1;
            done = 1;
            if (hn == 0.0) c->breakdown = 1;
        }
        done_s = done;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) col[i] = scol[i];
    if (done_s) {
        solve_upper(f, j + 1, scol, sg, ys);
        for (int i = threadIdx.x; i <= j; i += blockDim.x) f.y[i] = ys[i];
    }
}

// w -= V h2; ||w||; then the step's end (fg_step_tail). With the double-float Gram-Schmidt
// this kernel runs only when k_fg_cgs_df could not take ||w2|| from the Pythagorean relation
// (FgCtl::fuse = 0); otherwise that kernel has ended the step and k_fg_next forms w2 itself.
__global__ void __launch_bounds__(256) k_fg_norm(FgDev f, int n, int j) {
    __shared__ double red[32];
    __shared__ double hh[kMaxJ + 1];
    __shared__ float hf[kMaxJ + 1];
    __shared__ double tot[1];
    if (f.ctl->cycle_done || f.ctl->fuse) return;
    int r0, r1;
    cta_rows(n, r0, r1);
    for (int u = threadIdx.x; u <= j; u += blockDim.x) {
        hh[u] = __ldcg(f.h2 + u);
        hf[u] = (float)hh[u];
    }
    __syncthreads();
    double acc = 0.0;
    if (f.upd32)
        cta_update32(f.V32, f.ld, f.w, hf, r0, r1, j, &acc);
    else
        cta_update(f.V, f.ld, f.w, hh, r0, r1, j, &acc);
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) f.part[blockIdx.x] = acc;
    if (!last_cta(&f.ctl->counter)) return;
    reduce_partials(f.part, f.G, 1, tot);
    if (threadIdx.x == 0) f.ctl->counter = 0;
    fg_step_tail(f, j, sqrt(tot[0]));
}

// (ah, al) * (bh, bl), both double-float: TwoProduct of the high parts by FMA, the cross
// terms in FP32, renormalised by TwoSum
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& h, float& l) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    two_sum(p, e, h, l);
}

// v_{j+1} = w2 / ||w2||. When k_fg_cgs_df ended the step (FgCtl::fuse), this kernel forms
// w2 = w1 - V h2 itself, as k_fg_norm would have (FP32 products of the FP32 basis copy summed
// in FP32), four rows per thread, and the rest in double-float arithmetic: w1 arrives split
// (w32 + wlo), w2 and v = w2 * (1 / ||w2||) are pairs of FP32 numbers, stored as the two FP32
// parts of the basis; the FP64 basis vector, the input of the next preconditioner apply, is
// their sum (one FP64 addition per row instead of the subtraction, product and split).
__global__ void __launch_bounds__(256) k_fg_next(FgDev f, int n, int j) {
    __shared__ float hf[kMaxJ + 1];
    if (f.ctl->cycle_done) return;
    const double inv = __ldcg(f.hnext + 1);
    const size_t off = (size_t)(j + 1) * f.ld;
    if (!f.ctl->fuse) {
        for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
            const double v = f.w[r] * inv;
            f.V[off + r] = v;
            if (f.V32) store_basis32(f, off + r, v);
        }
        return;
    }
    // CTA 0 first ends the Arnoldi step (Givens rotations, estimate, stop decision): a chain
    // of dependent FP64 operations on one thread, hidden behind the other CTAs' rows. If it
    // ends the cycle, CTAs starting later skip their rows; v_{j+1} is then not needed.
    if (blockIdx.x == 0) fg_step_tail(f, j, __ldcg(f.hnext));
    for (int u = threadIdx.x; u <= j; u += blockDim.x) hf[u] = (float)__ldcg(f.h2 + u);
    __syncthreads();
    float ih, il;  // 1 / ||w2|| split
    df_split(inv, ih, il);
    const float* __restrict__ V32 = f.V32;
    const int64_t ld = f.ld;
    const int nth = gridDim.x * blockDim.x;
    // r is a multiple of 4 below n <= ld (a multiple of 64): the four rows' loads stay inside
    // the basis vectors; rows at or past n are not stored
    for (int r = 4 * (blockIdx.x * blockDim.x + threadIdx.x); r < n; r += 4 * nth) {
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        int i = 0;
        for (; i + 8 <= j + 1; i += 8) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; u++) v[u] = ld4f(V32 + (size_t)(i + u) * ld + r);
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const float hv = hf[i + u];
                c.x += hv * v[u].x;
                c.y += hv * v[u].y;
                c.z += hv * v[u].z;
                c.w += hv * v[u].w;
            }
        }
        for (; i <= j; i++) {
            const float4 v = ld4f(V32 + (size_t)i * ld + r);
            const float hv = hf[i];
            c.x += hv * v.x;
            c.y += hv * v.y;
            c.z += hv * v.z;
            c.w += hv * v.w;
        }
        const float cq[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (r + q < n) {
                float sh = f.w32[r + q], sl = f.wlo[r + q], vh, vl;
                df_add(sh, sl, -cq[q], 0.f);
                df_mul(sh, sl, ih, il, vh, vl);
                f.V32[off + r + q] = vh;
                f.Vlo[off + r + q] = vl;
                f.V[off + r + q] = __dadd_rn((double)vh, (double)vl);  // the preconditioner's input
            }
        }
    }
}

// x += Z y on the CTA's rows (y = R^{-1} g, solved by k_fg_norm when the cycle ended)
__global__ void k_fg_update(FgDev f, int n, double* __restrict__ x) {
    __shared__ double y[kMaxRestart];
    const int steps = f.ctl->steps;
    if (steps == 0) return;
    for (int i = threadIdx.x; i < steps; i += blockDim.x) y[i] = __ldcg(f.y + i);
    __syncthreads();
    int r0, r1;
    cta_rows(n, r0, r1);
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        double xv = x[r];
        for (int i = 0; i < steps; i++) xv += y[i] * f.Z[(size_t)i * f.ld + r];
        x[r] = xv;
    }
}

// ---------------------------------------------------------------------------------------
// out = b - A x (b null: out = A x), FP64, rows in the original order; a no-op once the
// FGMRES cycle is done (the multiplicative apply's residual and coarse-operator SpMV)
template <int VL>
__global__ void k_rap_resid(CsrDev A, const double* __restrict__ b, const double* __restrict__ x,
                            double* __restrict__ out, const int32_t* done) {
    if (done && *done) return;
    const int per_block = blockDim.x / VL;
    const int sub = threadIdx.x / VL, sl = threadIdx.x & (VL - 1);
    for (int base = blockIdx.x * per_block; base < A.n; base += gridDim.x * per_block) {
        const int r = base + sub;
        const bool valid = r < A.n;
        const double s = row_dot<VL>(A, r, valid, x, sl);
        if (valid && sl == 0) out[r] = b ? b[r] - s : s;
    }
}

// Lanes per CSR row: every level of the lanes' shuffle reduction is one more FP64 add per
// row, and FP64 issue is the scarce resource on GB300, so short rows get one lane each.
static int pick_vl(const Handle& h) {
    const double avg = h.n ? (double)h.nnz / h.n : 1.0;
    if (avg <= 12) return 1;
    if (avg <= 24) return 2;
    if (avg <= 48) return 4;
    if (avg <= 96) return 8;
    if (avg <= 192) return 16;
    return 32;
}

static CsrDev csr_of(const Handle& h) {
    CsrDev A;
    A.rp = h.d_A_rp;
    A.ci = h.d_A_ci;
    A.v = h.d_A_v;
    A.n = h.n;
    return A;
}

#define ILU2L_VL_SWITCH(vl, CALL) \
    switch (vl) {                 \
        case 1: {                 \
            constexpr int V = 1;  \
            CALL;                 \
        } break;                  \
        case 2: {                 \
            constexpr int V = 2;  \
            CALL;                 \
        } break;                  \
        case 4: {                 \
            constexpr int V = 4;  \
            CALL;                 \
        } break;                  \
        case 8: {                 \
            constexpr int V = 8;  \
            CALL;                 \
        } break;                  \
        case 16: {                \
            constexpr int V = 16; \
            CALL;                 \
        } break;                  \
        default: {                \
            constexpr int V = 32; \
            CALL;                 \
        } break;                  \
    }

cudaError_t launch_spmv(const Handle& h, const double* x, double* y, cudaStream_t st) {
    if (h.n == 0) return cudaSuccess;
    const int vl = pick_vl(h);
    const int blocks = h.sm_count * 8;
    ILU2L_VL_SWITCH(vl, (k_spmv<V><<<blocks, 256, 0, st>>>(csr_of(h), x, y)));
    return cudaGetLastError();
}

cudaError_t launch_rap_resid(const Handle& h, const double* b, const double* x, double* out, const int32_t* done,
                             cudaStream_t st) {
    if (h.n == 0) return cudaSuccess;
    const int vl = pick_vl(h);
    const int blocks = h.sm_count * 8;
    ILU2L_VL_SWITCH(vl, (k_rap_resid<V><<<blocks, 256, 0, st>>>(csr_of(h), b, x, out, done)));
    return cudaGetLastError();
}

cudaError_t launch_fg_resid(const Handle& h, const double* b, const double* x, int first, cudaStream_t st) {
    const int vl = pick_vl(h);
    ILU2L_VL_SWITCH(vl, (k_fg_resid<V><<<h.fg_G, h.fg_threads, 0, st>>>(csr_of(h), h.fg, b, x, first)));
    return cudaGetLastError();
}

cudaError_t launch_fg_scale0(const Handle& h, cudaStream_t st) {
    k_fg_scale0<<<h.sm_count * 4, 256, 0, st>>>(h.fg, h.n);
    return cudaGetLastError();
}

// the double-float k_fg_cgs takes up to (kMaxJ + 1) * 32 float2 of dynamic shared memory
// (set on the current device whenever a handle sizes its FGMRES workspace)
cudaError_t configure_krylov() {
    return cudaFuncSetAttribute(k_fg_cgs_df<kCgsDfThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (kMaxJ + 2) * 32 * (int)sizeof(float2));
}

cudaError_t launch_fg_spmv_dot(const Handle& h, int j, cudaStream_t st) {
    const int vl = pick_vl(h);
    ILU2L_VL_SWITCH(vl, (k_fg_spmv_dot<V><<<h.fg_G, h.fg_threads, 0, st>>>(csr_of(h), h.fg, j)));
    return cudaGetLastError();
}

cudaError_t launch_fg_cgs(const Handle& h, int j, cudaStream_t st) {
    if (h.fg.Vlo)
        k_fg_cgs_df<kCgsDfThreads><<<h.fg_G, kCgsDfThreads, (size_t)(j + 2) * 32 * sizeof(float2), st>>>(h.fg, h.n, j);
    else
        k_fg_cgs<<<h.fg_G, h.fg_threads, 0, st>>>(h.fg, h.n, j);
    return cudaGetLastError();
}

cudaError_t launch_fg_norm(const Handle& h, int j, cudaStream_t st) {
    k_fg_norm<<<h.fg_G, h.fg_threads, 0, st>>>(h.fg, h.n, j);
    return cudaGetLastError();
}

cudaError_t launch_fg_next(const Handle& h, int j, cudaStream_t st) {
    // the double-float form takes four rows per thread: one pass over n
    const int blocks = std::max(h.sm_count * 4, (h.n + 1023) / 1024);
    k_fg_next<<<blocks, 256, 0, st>>>(h.fg, h.n, j);
    return cudaGetLastError();
}

cudaError_t launch_fg_update(const Handle& h, double* x, cudaStream_t st) {
    k_fg_update<<<h.fg_G, h.fg_threads, 0, st>>>(h.fg, h.n, x);
    return cudaGetLastError();
}

}  // namespace ilu2l
