// kernels_ilut.cu -- the ILUT(tau, p) numeric factorisation of the local blocks on the GPU.
// The paper factorises with ILUT on the CPU (Sec. 4.2); the dual-threshold rule is the
// standard one, as the host factorisation in setup_host.cpp states it, and this kernel gives
// its result bit for bit.
//
// ILUT's fill is decided row by row, so its rows cannot be level-scheduled in advance. Every
// row of every local block is a work item; items are handed out to persistent warps by an
// atomic counter in a fixed order -- round robin over the blocks by local row index, so all
// blocks advance together. A row eliminates its pivots k < i in ascending order exactly as
// the sequential definition does; before it reads row k's U part it waits for row k's done
// flag. A row only waits on rows handed out before it, and those are held by running warps
// that only wait on rows before them, so the waits end; they are bounded all the same (a
// wait that runs out sets the error word). A row that fails (full table, zero pivot, a wait
// that ran out, a failed pivot row) still releases its flag, marked failed, so no row waits
// on it for long, and once the error word is set the remaining rows are skipped.
//
// Per row, in one warp:
//   * the working row w is an open-addressing table in shared memory (column -> slot, linear
//     probing), each slot with its value and state, plus a list of the occupied slots so that
//     every scan costs the row's entries, not the table's size;
//   * lane 0 sums the row's squares in CSR order; t_i = tau * ||a_i||_2;
//   * the smallest pending pivot comes from a warp-wide minimum over the list; l_ik =
//     w_k / u_kk; |l_ik| < t_i drops it, otherwise each lane merges one entry of row k's U part,
//     w_j -= l_ik * u_kj, product and difference rounded separately (the host code is compiled
//     without contraction), so each w_j sees the same operations in the same order;
//   * the p largest kept L entries and the p largest U entries with |w_j| >= t_i (ties: the
//     smaller column) are picked by rounds of a warp-wide arg-max, pick j in lane j, and
//     written at their rank by column;
//   * a pivot below eps * max_j |a_ij| is set to that bound with its sign (a zero pivot with
//     eps = 0 is an error).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "devutil.cuh"
#include "handle.h"

namespace ilu2l {

namespace {

constexpr uint8_t kFree = 0, kPend = 1, kKeptL = 2, kDropL = 3, kUpper = 4, kTaken = 5;
constexpr int32_t kErrIlutWait = 2, kErrIlutTable = 8, kErrIlutZero = 16;
constexpr int32_t kRowDone = 1, kRowFailed = 2;

struct IlutArgs {
    const int32_t* rp;     // rows of all blocks, block-local column indices < the block's size
    const int32_t* ci;
    const double* v;
    const int32_t* row0;   // per row: index of its block's first row
    const int32_t* order;  // hand-out order of the rows
    int32_t nrows;
    int32_t W;             // output slots per row: 2p + 1
    int32_t hmask;         // table slots - 1 (a power of two minus one)
    int32_t warps;         // warps per CTA
    double tau, eps;
    int32_t pkeep;         // p <= 32
    int32_t* out_ci;       // nrows x W, block-local columns, the row's entries by column
    double* out_v;
    int32_t* out_cnt;      // entries of each row
    int32_t* out_dpos;     // position of the pivot in the row
    int32_t* done;         // per row: 0, kRowDone or kRowFailed
    uint32_t* queue;       // next hand-out position
    int32_t* npert;        // perturbed pivots
    int32_t* err;          // error word
    uint64_t spin;
};

__device__ __forceinline__ int32_t ld_acquire(const int32_t* p) {
    int32_t v;
    asm volatile("ld.acquire.gpu.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int32_t* p, int32_t v) {
    asm volatile("st.release.gpu.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int32_t ld_volatile(const int32_t* p) { return *(const volatile int32_t*)p; }

struct Table {
    double* val;
    int32_t* key;
    int32_t* list;
    int32_t* cnt;
    uint8_t* st;
    uint32_t mask;

    // slot of column c, inserting it when absent (*fresh = true, the slot listed); -1 when
    // the table is full. Lanes of one call insert distinct columns.
    __device__ __forceinline__ int find_or_insert(int32_t c, bool* fresh) const {
        uint32_t h = ((uint32_t)c * 2654435761u) & mask;
        for (uint32_t probe = 0; probe <= mask; probe++) {
            const int32_t k = ((volatile int32_t*)key)[h];
            if (k == c) {
                *fresh = false;
                return (int)h;
            }
            if (k == -1) {
                const int32_t old = atomicCAS(&key[h], -1, c);
                if (old == -1) {
                    *fresh = true;
                    list[atomicAdd(cnt, 1)] = (int32_t)h;
                    return (int)h;
                }
                if (old == c) {
                    *fresh = false;
                    return (int)h;
                }
            }
            h = (h + 1) & mask;
        }
        return -1;
    }
};

// warp-wide arg-max of (|value|, then the smaller column): the winner's (magnitude, column, slot)
__device__ __forceinline__ void warp_best(double& bm, int32_t& bc, int& bh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double mo = __shfl_xor_sync(kFull, bm, o);
        const int32_t co = __shfl_xor_sync(kFull, bc, o);
        const int ho = __shfl_xor_sync(kFull, bh, o);
        if (mo > bm || (mo == bm && co < bc)) {
            bm = mo;
            bc = co;
            bh = ho;
        }
    }
}

__global__ void k_ilut(IlutArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t H = (size_t)A.hmask + 1, NW = (size_t)A.warps;
    Table T;
    T.val = reinterpret_cast<double*>(smem) + wid * H;
    T.key = reinterpret_cast<int32_t*>(smem + NW * H * 8) + wid * H;
    T.list = reinterpret_cast<int32_t*>(smem + NW * H * 12) + wid * H;
    T.cnt = reinterpret_cast<int32_t*>(smem + NW * H * 16) + wid;
    T.st = smem + NW * H * 16 + NW * 4 + wid * H;
    T.mask = (uint32_t)A.hmask;
    for (size_t h = lane; h < H; h += 32) {
        T.key[h] = -1;
        T.st[h] = kFree;
    }
    if (lane == 0) *T.cnt = 0;
    __syncwarp();
    for (;;) {
        int32_t t = 0, abort = 0;
        if (lane == 0) {
            t = (int32_t)atomicAdd(A.queue, 1u);
            abort = ld_volatile(A.err);
        }
        t = __shfl_sync(kFull, t, 0);
        if (t >= A.nrows) break;
        const int32_t r = A.order[t];
        if (__shfl_sync(kFull, abort, 0)) {  // an earlier row failed: the result is discarded
            if (lane == 0) st_release(A.done + r, kRowFailed);
            continue;
        }
        const int32_t g0 = A.row0[r];  // the block's first row
        const int32_t i = r - g0;      // local row index
        const int32_t qa = A.rp[r], qb = A.rp[r + 1];
        double nrm2 = 0.0, amax = 0.0;
        if (lane == 0)
            for (int32_t q = qa; q < qb; q++) {
                const double a = A.v[q];
                nrm2 = __dadd_rn(nrm2, __dmul_rn(a, a));
                amax = fmax(amax, fabs(a));
            }
        nrm2 = __shfl_sync(kFull, nrm2, 0);
        amax = __shfl_sync(kFull, amax, 0);
        const double ti = __dmul_rn(A.tau, __dsqrt_rn(nrm2));
        bool bad = false;
        int32_t fail = 0;  // error bits of this row (-1: a pivot row failed, its bits are set)
        // the row into the table; the pivot's slot exists even when a_ii is not stored
        int hpiv = -1;
        if (lane == 0) {
            bool fresh;
            hpiv = T.find_or_insert(i, &fresh);
            if (hpiv >= 0) {
                T.val[hpiv] = 0.0;
                T.st[hpiv] = kUpper;
            }
        }
        hpiv = __shfl_sync(kFull, hpiv, 0);
        for (int32_t q = qa + lane; q < qb; q += 32) {
            const int32_t c = A.ci[q];
            bool fresh;
            const int h = T.find_or_insert(c, &fresh);
            if (h < 0) {
                bad = true;
                continue;
            }
            T.val[h] = A.v[q];
            if (c != i) T.st[h] = (c < i) ? kPend : kUpper;
        }
        if (__any_sync(kFull, bad) || hpiv < 0) fail = kErrIlutTable;
        __syncwarp();
        // pivots in ascending order
        while (!fail) {
            const int32_t n = ld_volatile(T.cnt);
            int32_t kmin = INT32_MAX;
            int hmin = -1;
            for (int32_t e = lane; e < n; e += 32) {
                const int h = T.list[e];
                if (T.st[h] == kPend && T.key[h] < kmin) {
                    kmin = T.key[h];
                    hmin = h;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const int32_t ko = __shfl_xor_sync(kFull, kmin, o);
                const int ho = __shfl_xor_sync(kFull, hmin, o);
                if (ko < kmin) {
                    kmin = ko;
                    hmin = ho;
                }
            }
            if (kmin == INT32_MAX) break;
            const int32_t rk = g0 + kmin;  // the pivot's row, handed out before this one
            int32_t d = 0;
            double wk = 0.0;
            if (lane == 0) {
                for (uint64_t s = 0; s < A.spin && d == 0; s++) d = ld_acquire(A.done + rk);
                wk = T.val[hmin];
            }
            d = __shfl_sync(kFull, d, 0);
            wk = __shfl_sync(kFull, wk, 0);
            if (d != kRowDone) {
                fail = (d == 0) ? kErrIlutWait : -1;
                break;
            }
            (void)ld_acquire(A.done + rk);  // every lane reads row k after observing its release
            const int32_t kd = __ldcg(A.out_dpos + rk), kc = __ldcg(A.out_cnt + rk);
            const double lik = __ddiv_rn(wk, __ldcg(A.out_v + (size_t)rk * A.W + kd));
            if (fabs(lik) < ti) {  // dropped: no update from row k
                if (lane == 0) {
                    T.val[hmin] = 0.0;
                    T.st[hmin] = kDropL;
                }
                __syncwarp();
                continue;
            }
            if (lane == 0) {
                T.val[hmin] = lik;
                T.st[hmin] = kKeptL;
            }
            for (int32_t u = kd + 1 + lane; u < kc; u += 32) {
                const int32_t j = __ldcg(A.out_ci + (size_t)rk * A.W + u);
                const double ukj = __ldcg(A.out_v + (size_t)rk * A.W + u);
                bool fresh;
                const int h = T.find_or_insert(j, &fresh);
                if (h < 0) {
                    bad = true;
                    continue;
                }
                const double w0 = fresh ? 0.0 : T.val[h];
                if (fresh) T.st[h] = (j < i) ? kPend : kUpper;
                T.val[h] = __dsub_rn(w0, __dmul_rn(lik, ukj));
            }
            __syncwarp();
            if (__any_sync(kFull, bad)) fail = kErrIlutTable;
        }
        __syncwarp();
        // the p largest of each part, pick j in lane j; then each pick's rank by column
        int32_t pc[2] = {INT32_MAX, INT32_MAX}, npk[2] = {0, 0};
        double pv[2] = {0.0, 0.0};
        const int32_t n = ld_volatile(T.cnt);
        for (int part = 0; part < 2 && !fail; part++) {
            const uint8_t want = part == 0 ? kKeptL : kUpper;
            for (int round = 0; round < A.pkeep; round++) {
                double bm = -1.0;
                int32_t bc = INT32_MAX;
                int bh = -1;
                for (int32_t e = lane; e < n; e += 32) {
                    const int h = T.list[e];
                    if (T.st[h] != want || h == hpiv) continue;
                    const double m = fabs(T.val[h]);
                    if (!(m >= ti)) continue;
                    const int32_t c = T.key[h];
                    if (m > bm || (m == bm && c < bc)) {
                        bm = m;
                        bc = c;
                        bh = h;
                    }
                }
                warp_best(bm, bc, bh);
                if (bh < 0) break;
                if (lane == round) {
                    pc[part] = bc;
                    pv[part] = T.val[bh];
                }
                __syncwarp();
                if (lane == 0) T.st[bh] = kTaken;
                __syncwarp();
                npk[part]++;
            }
        }
        int32_t* oci = A.out_ci + (size_t)r * A.W;
        double* ov = A.out_v + (size_t)r * A.W;
        if (!fail) {
            double uii = T.val[hpiv];
            const double thr = __dmul_rn(A.eps, amax);
            if (A.eps > 0.0 && fabs(uii) < thr) {
                uii = (uii >= 0.0) ? thr : -thr;
                if (lane == 0) atomicAdd(A.npert, 1);
            }
            if (uii == 0.0) {
                fail = kErrIlutZero;
            } else {
                const int32_t nl = npk[0], nu = npk[1];
                int32_t rank[2] = {0, 0};
                for (int part = 0; part < 2; part++)
                    for (int l = 0; l < npk[part]; l++)
                        if (__shfl_sync(kFull, pc[part], l) < pc[part]) rank[part]++;
                if (lane < nl) {
                    oci[rank[0]] = pc[0];
                    ov[rank[0]] = pv[0];
                }
                if (lane < nu) {
                    oci[nl + 1 + rank[1]] = pc[1];
                    ov[nl + 1 + rank[1]] = pv[1];
                }
                if (lane == 0) {
                    oci[nl] = i;
                    ov[nl] = uii;
                    A.out_dpos[r] = nl;
                    A.out_cnt[r] = nl + 1 + nu;
                }
            }
        }
        // clear the table through its list
        for (int32_t e = lane; e < n; e += 32) {
            const int h = T.list[e];
            T.key[h] = -1;
            T.st[h] = kFree;
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            *T.cnt = 0;
            if (fail > 0) atomicOr(A.err, fail);
            st_release(A.done + r, fail ? kRowFailed : kRowDone);
        }
        __syncwarp();
    }
}

}  // namespace

// ILUT of the interior blocks B_s (two-level) or of the whole local blocks A_s (block
// Jacobi) -- each block's rows with their local columns below the block's size -- on the
// device; fills h.f1_rp / f1_ci / f1_dpos / f1_host_vals exactly as the host factorisation
// does. Returns ILU_ERR_UNSUPPORTED when p > 32 or a row touches more columns than the
// largest table holds (the caller then factorises on the host), ILU_ERR_ZERO_PIVOT,
// ILU_ERR_TIMEOUT, ILU_ERR_OOM or ILU_ERR_CUDA. Synchronises h.st.
ilu_status device_ilut(Handle& h) {
    const bool schur = (h.variant != ILU_VARIANT_BJ);
    const int32_t p = h.p, n = h.n, pk = h.o.ilut_p;
    if (pk < 0 || pk > 32) return ILU_ERR_UNSUPPORTED;
    std::vector<int32_t> rp(1, 0), ci, row0, blk0(p + 1, 0);
    std::vector<double> v;
    int32_t mmax = 0;
    for (int32_t s = 0; s < p; s++) {
        const int32_t q0 = h.qoff[s];
        const int32_t m = schur ? h.nint[s] : (h.qoff[s + 1] - q0);
        blk0[s + 1] = blk0[s] + m;
        mmax = std::max(mmax, m);
        for (int32_t r = 0; r < m; r++) {
            for (int32_t k = h.q_rp[q0 + r]; k < h.q_rp[q0 + r + 1]; k++)
                if (h.q_ci[k] < m) {
                    ci.push_back(h.q_ci[k]);
                    v.push_back(h.q_v[k]);
                }
            rp.push_back((int32_t)ci.size());
            row0.push_back(blk0[s]);
        }
    }
    const int32_t R = blk0[p];
    h.f1_rp.assign(n + 1, 0);
    h.f1_dpos.assign(n, -1);
    h.f1_ci.clear();
    h.f1_host_vals.clear();
    if (R == 0) return ILU_OK;
    // hand-out order: local row 0 of every block, then local row 1, ...
    std::vector<int32_t> order;
    order.reserve(R);
    for (int32_t t = 0; t < mmax; t++)
        for (int32_t s = 0; s < p; s++)
            if (t < blk0[s + 1] - blk0[s]) order.push_back(blk0[s] + t);
    const int32_t W = 2 * pk + 1;
    int dev = 0, sms = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return ILU_ERR_CUDA;
    int32_t* d_rp = h.alloc<int32_t>(rp.size(), &e);
    int32_t* d_ci = h.alloc<int32_t>(std::max<size_t>(ci.size(), 1), &e);
    double* d_v = h.alloc<double>(std::max<size_t>(v.size(), 1), &e);
    int32_t* d_row0 = h.alloc<int32_t>(R, &e);
    int32_t* d_order = h.alloc<int32_t>(R, &e);
    int32_t* d_oci = h.alloc<int32_t>((size_t)R * W, &e);
    double* d_ov = h.alloc<double>((size_t)R * W, &e);
    int32_t* d_cnt = h.alloc<int32_t>(R, &e);
    int32_t* d_dpos = h.alloc<int32_t>(R, &e);
    int32_t* d_done = h.alloc<int32_t>(R, &e);
    int32_t* d_misc = h.alloc<int32_t>(4, &e);  // queue, npert, err
    auto release_all = [&] {
        for (void* q : {(void*)d_rp, (void*)d_ci, (void*)d_v, (void*)d_row0, (void*)d_order, (void*)d_oci,
                        (void*)d_ov, (void*)d_cnt, (void*)d_dpos, (void*)d_done, (void*)d_misc})
            if (q) h.release(q);
    };
    auto ck = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    if (e == cudaSuccess) {
        ck(cudaMemcpyAsync(d_rp, rp.data(), rp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h.st));
        if (!ci.empty()) {
            ck(cudaMemcpyAsync(d_ci, ci.data(), ci.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h.st));
            ck(cudaMemcpyAsync(d_v, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice, h.st));
        }
        ck(cudaMemcpyAsync(d_row0, row0.data(), (size_t)R * sizeof(int32_t), cudaMemcpyHostToDevice, h.st));
        ck(cudaMemcpyAsync(d_order, order.data(), (size_t)R * sizeof(int32_t), cudaMemcpyHostToDevice, h.st));
    }
    IlutArgs a{};
    a.rp = d_rp;
    a.ci = d_ci;
    a.v = d_v;
    a.row0 = d_row0;
    a.order = d_order;
    a.nrows = R;
    a.W = W;
    a.tau = h.o.ilut_tau;
    a.eps = h.o.pivot_eps;
    a.pkeep = pk;
    a.out_ci = d_oci;
    a.out_v = d_ov;
    a.out_cnt = d_cnt;
    a.out_dpos = d_dpos;
    a.done = d_done;
    a.queue = reinterpret_cast<uint32_t*>(d_misc);
    a.npert = d_misc + 1;
    a.err = d_misc + 2;
    a.spin = h.o.spin_limit ? h.o.spin_limit : (1ull << 22);
    // first a 512-slot table per warp, four warps per CTA; when a row fills it, once more
    // with one warp per CTA and the largest table the shared memory holds
    std::vector<int32_t> misc(4, 0);
    for (int attempt = 0; attempt < 2 && e == cudaSuccess; attempt++) {
        int hbits = 9, warps = 4;
        if (attempt == 1) {
            warps = 1;
            while (hbits < 16 && 17 * ((size_t)2 << hbits) + 4 <= (size_t)optin) hbits++;
        }
        a.hmask = (1 << hbits) - 1;
        a.warps = warps;
        const size_t smem = (size_t)warps * (17 * ((size_t)1 << hbits) + 4);
        ck(cudaFuncSetAttribute(k_ilut, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ck(cudaMemsetAsync(d_done, 0, (size_t)R * sizeof(int32_t), h.st));
        ck(cudaMemsetAsync(d_misc, 0, 4 * sizeof(int32_t), h.st));
        int nb = 0;
        ck(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ilut, 32 * warps, smem));
        const int grid = std::max(1, std::min(std::max(nb, 1) * sms, (R + warps - 1) / warps));
        if (e == cudaSuccess) {
            k_ilut<<<grid, 32 * warps, smem, h.st>>>(a);
            ck(cudaGetLastError());
            h.kernel_launches += 1;
        }
        ck(cudaMemcpyAsync(misc.data(), d_misc, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, h.st));
        ck(cudaStreamSynchronize(h.st));
        if (e != cudaSuccess || misc[2] != kErrIlutTable) break;  // only a full table is retried
    }
    std::vector<int32_t> cnt, dpos, oci;
    std::vector<double> ov;
    if (e == cudaSuccess && misc[2] == 0) {
        cnt.resize(R);
        dpos.resize(R);
        oci.resize((size_t)R * W);
        ov.resize((size_t)R * W);
        ck(cudaMemcpyAsync(cnt.data(), d_cnt, (size_t)R * sizeof(int32_t), cudaMemcpyDeviceToHost, h.st));
        ck(cudaMemcpyAsync(dpos.data(), d_dpos, (size_t)R * sizeof(int32_t), cudaMemcpyDeviceToHost, h.st));
        ck(cudaMemcpyAsync(oci.data(), d_oci, (size_t)R * W * sizeof(int32_t), cudaMemcpyDeviceToHost, h.st));
        ck(cudaMemcpyAsync(ov.data(), d_ov, (size_t)R * W * sizeof(double), cudaMemcpyDeviceToHost, h.st));
        ck(cudaStreamSynchronize(h.st));
    }
    release_all();
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ILU_ERR_OOM : ILU_ERR_CUDA;
    const int32_t err = misc[2];
    if (err & kErrIlutZero) return ILU_ERR_ZERO_PIVOT;
    if (err & kErrIlutWait) return ILU_ERR_TIMEOUT;
    if (err & kErrIlutTable) return ILU_ERR_UNSUPPORTED;
    h.npert += misc[1];
    // the factor in Q order, as the host factorisation lays it out
    size_t tot = 0;
    for (int32_t g = 0; g < R; g++) tot += (size_t)cnt[g];
    h.f1_ci.reserve(tot);
    h.f1_host_vals.reserve(tot);
    for (int32_t s = 0; s < p; s++) {
        const int32_t q0 = h.qoff[s];
        const int32_t ns = h.qoff[s + 1] - q0;
        const int32_t m = blk0[s + 1] - blk0[s];
        for (int32_t r = 0; r < ns; r++) {
            const int32_t q = q0 + r;
            if (r < m) {
                const int32_t g = blk0[s] + r;
                for (int32_t t = 0; t < cnt[g]; t++) {
                    if (t == dpos[g]) h.f1_dpos[q] = (int32_t)h.f1_ci.size();
                    h.f1_ci.push_back(oci[(size_t)g * W + t]);
                    h.f1_host_vals.push_back(ov[(size_t)g * W + t]);
                }
            }
            h.f1_rp[q + 1] = (int32_t)h.f1_ci.size();
        }
    }
    return ILU_OK;
}

}  // namespace ilu2l
