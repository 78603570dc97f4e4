// kernels_ilut.cu -- the ILUT(tau, p) numeric factorisation of the local blocks on the GPU.
// The paper factorises with ILUT on the CPU (Sec. 4.2); the dual-threshold rule is the
// standard one, as the host factorisation in setup_host.cpp states it, and this kernel gives
// its result bit for bit.
//
// ILUT's fill is decided row by row, so its rows cannot be level-scheduled in advance. Every
// row of every local block is a work item; items are handed out to persistent warps by an
// atomic counter in a fixed order -- by the fraction of its block a row completes, so that
// every block advances at the same relative pace and the largest block, which sets the
// finishing time, holds proportionally many warps. A row eliminates its pivots k < i in
// ascending order exactly as the sequential definition does; before it reads row k it waits
// for row k's done flag. A row only waits on rows handed out before it, and those are held by
// running warps that only wait on rows before them, so the waits end; they are bounded all
// the same (a wait that runs out sets the error word). A row that fails (full table, zero
// pivot, a wait that ran out, a failed pivot row) still releases its flag, marked failed, so
// no row waits on it for long, and once the error word is set the remaining rows are skipped.
//
// Per row, in one warp:
//   * the working row w is an open-addressing table in shared memory (column -> slot, linear
//     probing), each slot with its value and state, plus a list of the occupied slots so that
//     every scan costs the row's entries, not the table's size;
//   * the row is read one entry a lane; its squares are summed in CSR order through shuffles;
//     t_i = tau * ||a_i||_2;
//   * the smallest pending pivot is a warp minimum (redux); row k's pivot, U count and U part
//     (at a fixed offset of its output) arrive in one round trip; l_ik = w_k / u_kk; |l_ik| <
//     t_i drops it, otherwise each lane merges one entry of row k's U part, w_j -= l_ik * u_kj,
//     product and difference rounded separately (the host code is compiled without
//     contraction), so each w_j sees the same operations in the same order;
//   * the p largest kept L entries and the p largest U entries with |w_j| >= t_i (ties: the
//     smaller column) are those whose rank -- the entries of their part that beat them -- is
//     below p; each pick is written at its rank by column;
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

constexpr uint8_t kFree = 0, kPend = 1, kKeptL = 2, kDropL = 3, kUpper = 4, kPickL = 5, kPickU = 6;
constexpr int32_t kErrIlutWait = 2, kErrIlutTable = 8, kErrIlutZero = 16;
constexpr int32_t kRowDone = 1, kRowFailed = 2;
constexpr uint8_t kPicked = 0x80, kStateMask = 0x7f;
constexpr uint32_t kNoKey = 0x7fffffffu;

// Output of a row id r, W = 2p + 1 slots: its L entries by column in slots [0, nl), its U
// entries by column in slots [p + 1, p + 1 + nu); out_nl[r], out_nu[r] and the pivot
// out_piv[r] beside them. The U part's fixed offset lets a row that eliminates with row r
// load the pivot and the U part in one round trip.
struct IlutArgs {
    const int32_t* rp;     // the local blocks A_s in Q order, block-local column indices; a
    const int32_t* ci;     // row of block s takes its entries with columns below m_s
    const double* v;
    const int32_t* blk;    // per row id: its block s (row ids: block s owns [boff[s], boff[s+1]))
    const int32_t* boff;   // p + 1: first row id of each block; m_s = boff[s+1] - boff[s]
    const int32_t* qoff;   // p + 1: first Q row of each block
    const int32_t* order;  // hand-out order of the row ids
    int32_t nrows;
    int32_t W;             // output slots per row: 2p + 1
    int32_t hmask;         // table slots - 1 (a power of two minus one)
    int32_t warps;         // warps per CTA
    double tau, eps;
    int32_t pkeep;         // p <= 32
    int32_t* out_ci;       // nrows x W
    double* out_v;
    int32_t* out_nl;
    int32_t* out_nu;
    double* out_piv;
    int32_t* done;         // per row: 0, kRowDone or kRowFailed
    uint32_t* queue;       // next hand-out position
    int32_t* npert;        // perturbed pivots
    int32_t* err;          // error word
    uint64_t spin;
};

__device__ __forceinline__ int32_t ld_relaxed(const int32_t* p) {
    int32_t v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ void st_release(int32_t* p, int32_t v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
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

// part of a table entry in the selection: 0 a kept L entry, 1 a U entry other than the pivot,
// -1 neither or below the threshold
__device__ __forceinline__ int sel_part(uint8_t s, int h, int hpiv, double m, double ti) {
    s &= kStateMask;
    if (!(m >= ti)) return -1;
    if (s == kKeptL) return 0;
    if (s == kUpper && h != hpiv) return 1;
    return -1;
}

__global__ void k_ilut(IlutArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t H = (size_t)A.hmask + 1, NW = (size_t)A.warps;
    const int32_t pk = A.pkeep, W = A.W;
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
        const int32_t sb = A.blk[r];
        const int32_t g0 = A.boff[sb];            // the block's first row id
        const int32_t m = A.boff[sb + 1] - g0;    // rows and columns of the factorised block
        const int32_t i = r - g0;                 // local row index
        const int32_t qa = A.rp[A.qoff[sb] + i], qb = A.rp[A.qoff[sb] + i + 1];
        bool bad = false;
        int32_t fail = 0;  // error bits of this row (-1: a pivot row failed, its bits are set)
        int hpiv = -1;     // the pivot's slot, there even when a_ii is not stored
        if (lane == 0) {
            bool fresh;
            hpiv = T.find_or_insert(i, &fresh);
            if (hpiv >= 0) {
                T.val[hpiv] = 0.0;
                T.st[hpiv] = kUpper;
            }
        }
        hpiv = __shfl_sync(kFull, hpiv, 0);
        // the row: one entry a lane; its squares summed in CSR order (every lane the same sum)
        double nrm2 = 0.0, amax = 0.0;
        for (int32_t q0 = qa; q0 < qb; q0 += 32) {
            const int32_t q = q0 + lane;
            int32_t c = -1;
            double a = 0.0;
            if (q < qb) {
                c = A.ci[q];
                a = A.v[q];
            }
            const bool in = (q < qb) && c < m;
            const double sq = __dmul_rn(a, a);
            const int cnt = min(32, qb - q0);
            for (int j = 0; j < cnt; j++) {
                const double sj = __shfl_sync(kFull, sq, j);
                const double aj = __shfl_sync(kFull, fabs(a), j);
                if (__shfl_sync(kFull, (int)in, j)) {
                    nrm2 = __dadd_rn(nrm2, sj);
                    amax = fmax(amax, aj);
                }
            }
            if (in && hpiv >= 0) {
                bool fresh;
                const int h = T.find_or_insert(c, &fresh);
                if (h < 0) {
                    bad = true;
                } else {
                    T.val[h] = a;
                    if (c != i) T.st[h] = (c < i) ? kPend : kUpper;
                }
            }
        }
        const double ti = __dmul_rn(A.tau, __dsqrt_rn(nrm2));
        if (__any_sync(kFull, bad) || hpiv < 0) fail = kErrIlutTable;
        __syncwarp();
        // pivots in ascending order
        while (!fail) {
            const int32_t n = ld_volatile(T.cnt);
            uint32_t kmy = kNoKey;
            int hmy = -1;
            for (int32_t e = lane; e < n; e += 32) {
                const int h = T.list[e];
                if (T.st[h] == kPend && (uint32_t)T.key[h] < kmy) {
                    kmy = (uint32_t)T.key[h];
                    hmy = h;
                }
            }
            const uint32_t kmin = __reduce_min_sync(kFull, kmy);
            if (kmin == kNoKey) break;
            const int owner = __ffs(__ballot_sync(kFull, kmy == kmin)) - 1;
            const int hmin = __shfl_sync(kFull, hmy, owner);
            const int32_t rk = g0 + (int32_t)kmin;  // the pivot's row, handed out before this one
            int32_t d = 0;
            if (lane == 0) {
                d = ld_relaxed(A.done + rk);
                for (uint64_t s = 1; s < A.spin && d == 0; s++) d = ld_relaxed(A.done + rk);
                if (d != 0) fence_acq_rel();  // row k's entries are read after its release
            }
            d = __shfl_sync(kFull, d, 0);
            __syncwarp();
            if (d != kRowDone) {
                fail = (d == 0) ? kErrIlutWait : -1;
                break;
            }
            // row k's pivot, U count and U part, in one round trip
            const double ukk = __ldcg(A.out_piv + rk);
            const int32_t nuk = __ldcg(A.out_nu + rk);
            int32_t j = 0;
            double ukj = 0.0;
            if (lane < pk) {
                j = __ldcg(A.out_ci + (size_t)rk * W + pk + 1 + lane);
                ukj = __ldcg(A.out_v + (size_t)rk * W + pk + 1 + lane);
            }
            const double lik = __ddiv_rn(T.val[hmin], ukk);
            __syncwarp();
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
            if (lane < nuk) {
                bool fresh;
                const int h = T.find_or_insert(j, &fresh);
                if (h < 0) {
                    bad = true;
                } else {
                    const double w0 = fresh ? 0.0 : T.val[h];
                    if (fresh) T.st[h] = (j < i) ? kPend : kUpper;
                    T.val[h] = __dsub_rn(w0, __dmul_rn(lik, ukj));
                }
            }
            __syncwarp();
            if (__any_sync(kFull, bad)) fail = kErrIlutTable;
        }
        __syncwarp();
        const int32_t n = ld_volatile(T.cnt);
        int32_t* oci = A.out_ci + (size_t)r * W;
        double* ov = A.out_v + (size_t)r * W;
        if (!fail) {
            // the p largest of each part by (|w|, then the smaller column): an entry's rank is
            // the number of entries of its part that beat it; ranks below p are picked, marked
            // by the state's high bit (which the ranks of the other entries ignore)
            for (int32_t e = lane; e < n; e += 32) {
                const int h = T.list[e];
                const double mh = fabs(T.val[h]);
                const int part = sel_part(T.st[h], h, hpiv, mh, ti);
                if (part < 0) continue;
                const int32_t ch = T.key[h];
                int32_t rank = 0;
                for (int32_t y = 0; y < n && rank < pk; y++) {
                    const int hy = T.list[y];
                    const double my = fabs(T.val[hy]);
                    if (sel_part(T.st[hy], hy, hpiv, my, ti) == part &&
                        (my > mh || (my == mh && T.key[hy] < ch)))
                        rank++;
                }
                if (rank < pk) T.st[h] |= kPicked;
            }
            __syncwarp();
            int32_t mine[2] = {0, 0};
            for (int32_t e = lane; e < n; e += 32) {
                const int h = T.list[e];
                const uint8_t sh = T.st[h];
                if (!(sh & kPicked)) continue;
                const bool isL = (sh & kStateMask) == kKeptL;
                T.st[h] = isL ? kPickL : kPickU;
                mine[isL ? 0 : 1]++;
            }
            const int32_t nl = (int32_t)__reduce_add_sync(kFull, (uint32_t)mine[0]);
            const int32_t nu = (int32_t)__reduce_add_sync(kFull, (uint32_t)mine[1]);
            __syncwarp();
            // each pick's position: the picks of its part with a smaller column
            for (int32_t e = lane; e < n; e += 32) {
                const int h = T.list[e];
                const uint8_t sh = T.st[h];
                if (sh != kPickL && sh != kPickU) continue;
                const int32_t ch = T.key[h];
                int32_t pos = 0;
                for (int32_t y = 0; y < n; y++) {
                    const int hy = T.list[y];
                    if (T.st[hy] == sh && T.key[hy] < ch) pos++;
                }
                const int32_t at = (sh == kPickL) ? pos : pk + 1 + pos;
                oci[at] = ch;
                ov[at] = T.val[h];
            }
            double uii = T.val[hpiv];
            const double thr = __dmul_rn(A.eps, amax);
            if (A.eps > 0.0 && fabs(uii) < thr) {
                uii = (uii >= 0.0) ? thr : -thr;
                if (lane == 0) atomicAdd(A.npert, 1);
            }
            if (uii == 0.0) {
                fail = kErrIlutZero;
            } else if (lane == 0) {
                A.out_nl[r] = nl;
                A.out_nu[r] = nu;
                A.out_piv[r] = uii;
            }
        }
        // clear the table through its list
        __syncwarp();
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

// The rows' entries packed into the factor's CSR order: row id g of block s is Q row
// qoff[s] + (g - boff[s]); its entries (L part, pivot, U part) start at f1_rp of that row.
// One warp a row.
__global__ void k_ilut_pack(const int32_t* __restrict__ out_ci, const double* __restrict__ out_v,
                            const int32_t* __restrict__ out_nl, const int32_t* __restrict__ out_nu,
                            const double* __restrict__ out_piv, const int32_t* __restrict__ blk,
                            const int32_t* __restrict__ boff, const int32_t* __restrict__ qoff,
                            const int32_t* __restrict__ f1_rp, int32_t nrows, int32_t pk, int32_t* __restrict__ f1_ci,
                            double* __restrict__ f1_v) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t W = 2 * (int64_t)pk + 1;
    for (int64_t g = w0; g < nrows; g += nw) {
        const int32_t sb = blk[g];
        const int32_t i = (int32_t)(g - boff[sb]);
        const int64_t base = f1_rp[qoff[sb] + i];
        const int32_t nl = out_nl[g], nu = out_nu[g];
        for (int32_t t = lane; t < nl + 1 + nu; t += 32) {
            int32_t c;
            double x;
            if (t < nl) {
                c = out_ci[g * W + t];
                x = out_v[g * W + t];
            } else if (t == nl) {
                c = i;
                x = out_piv[g];
            } else {
                c = out_ci[g * W + pk + 1 + (t - nl - 1)];
                x = out_v[g * W + pk + 1 + (t - nl - 1)];
            }
            f1_ci[base + t] = c;
            f1_v[base + t] = x;
        }
    }
}

}  // namespace

// ILUT of the interior blocks B_s (two-level) or of the whole local blocks A_s (block
// Jacobi) -- each block's rows with their local columns below the block's size -- on the
// device. Fills h.f1_rp / f1_ci / f1_dpos as the host factorisation does; the values stay on
// the device in h.d_f1_stage (FP64, in f1 order), which the device setup moves into the value
// array. Leaves d_q_rp and d_q_ci uploaded for the device setup. Returns ILU_ERR_UNSUPPORTED
// when p > 32 or a row touches more columns than the largest table holds (the caller then
// factorises on the host), ILU_ERR_ZERO_PIVOT, ILU_ERR_TIMEOUT, ILU_ERR_OOM or ILU_ERR_CUDA.
// Synchronises h.st.
ilu_status device_ilut(Handle& h) {
    const bool schur = (h.variant != ILU_VARIANT_BJ);
    const int32_t p = h.p, n = h.n, pk = h.o.ilut_p;
    if (pk < 0 || pk > 32) return ILU_ERR_UNSUPPORTED;
    // row ids: block s owns [boff[s], boff[s+1]), its first m_s rows in Q order
    std::vector<int32_t> boff(p + 1, 0);
    int32_t mmax = 0;
    for (int32_t s = 0; s < p; s++) {
        const int32_t m = schur ? h.nint[s] : (h.qoff[s + 1] - h.qoff[s]);
        boff[s + 1] = boff[s] + m;
        mmax = std::max(mmax, m);
    }
    const int32_t R = boff[p];
    h.f1_rp.assign(n + 1, 0);
    h.f1_dpos.assign(n, -1);
    h.f1_ci.clear();
    h.f1_host_vals.clear();
    if (R == 0) return ILU_OK;
    std::vector<int32_t> blk(R), order(R);
    for (int32_t s = 0; s < p; s++)
        for (int32_t g = boff[s]; g < boff[s + 1]; g++) blk[g] = s;
    // hand-out order: by the fraction of its block a row completes, so every block advances at
    // the same relative pace and a large block holds proportionally many warps. Row i of a block
    // of m rows goes to bucket floor(i * mmax / m), strictly increasing in i (m <= mmax); the
    // buckets in order, each by block. A row is thus handed out after the rows before it in
    // its block, which is what the waits need.
    {
        std::vector<int32_t> bstart((size_t)mmax + 1, 0);
        for (int32_t s = 0; s < p; s++) {
            const int32_t m = boff[s + 1] - boff[s];
            for (int32_t i = 0; i < m; i++) bstart[(size_t)((int64_t)i * mmax / m) + 1]++;
        }
        for (int32_t b = 0; b < mmax; b++) bstart[b + 1] += bstart[b];
        for (int32_t s = 0; s < p; s++) {
            const int32_t m = boff[s + 1] - boff[s];
            for (int32_t i = 0; i < m; i++) order[bstart[(size_t)((int64_t)i * mmax / m)]++] = boff[s] + i;
        }
    }
    const int32_t W = 2 * pk + 1;
    int dev = 0, sms = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return ILU_ERR_CUDA;
    auto ck = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    const size_t nnzq = h.q_ci.size();
    if (!h.d_q_rp) {
        h.d_q_rp = h.alloc<int32_t>(h.q_rp.size(), &e);
        if (h.d_q_rp)
            ck(cudaMemcpyAsync(h.d_q_rp, h.q_rp.data(), h.q_rp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h.st));
    }
    if (!h.d_q_ci && e == cudaSuccess) {
        h.d_q_ci = h.alloc<int32_t>(std::max<size_t>(nnzq, 1), &e);
        if (h.d_q_ci && nnzq)
            ck(cudaMemcpyAsync(h.d_q_ci, h.q_ci.data(), nnzq * sizeof(int32_t), cudaMemcpyHostToDevice, h.st));
    }
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ILU_ERR_OOM : ILU_ERR_CUDA;
    double* d_qv = h.alloc<double>(std::max<size_t>(nnzq, 1), &e);
    int32_t* d_blk = h.alloc<int32_t>(R, &e);
    int32_t* d_order = h.alloc<int32_t>(R, &e);
    int32_t* d_boff = h.alloc<int32_t>(p + 1, &e);
    int32_t* d_qoff = h.alloc<int32_t>(p + 1, &e);
    int32_t* d_oci = h.alloc<int32_t>((size_t)R * W, &e);
    double* d_ov = h.alloc<double>((size_t)R * W, &e);
    int32_t* d_nl = h.alloc<int32_t>(R, &e);
    int32_t* d_nu = h.alloc<int32_t>(R, &e);
    double* d_piv = h.alloc<double>(R, &e);
    int32_t* d_done = h.alloc<int32_t>(R, &e);
    int32_t* d_misc = h.alloc<int32_t>(4, &e);  // queue, npert, err
    int32_t* d_f1rp = nullptr;
    int32_t* d_f1ci = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    auto release_all = [&] {
        for (void* q : {(void*)d_qv, (void*)d_blk, (void*)d_order, (void*)d_boff, (void*)d_qoff, (void*)d_oci,
                        (void*)d_ov, (void*)d_nl, (void*)d_nu, (void*)d_piv, (void*)d_done, (void*)d_misc, (void*)d_f1rp,
                        (void*)d_f1ci})
            if (q) h.release(q);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    };
    if (e == cudaSuccess) {
        if (nnzq) ck(cudaMemcpyAsync(d_qv, h.q_v.data(), nnzq * sizeof(double), cudaMemcpyHostToDevice, h.st));
        ck(cudaMemcpyAsync(d_blk, blk.data(), (size_t)R * sizeof(int32_t), cudaMemcpyHostToDevice, h.st));
        ck(cudaMemcpyAsync(d_order, order.data(), (size_t)R * sizeof(int32_t), cudaMemcpyHostToDevice, h.st));
        ck(cudaMemcpyAsync(d_boff, boff.data(), (size_t)(p + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, h.st));
        ck(cudaMemcpyAsync(d_qoff, h.qoff.data(), (size_t)(p + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, h.st));
        ck(cudaEventCreate(&ev0));
        ck(cudaEventCreate(&ev1));
    }
    IlutArgs a{};
    a.rp = h.d_q_rp;
    a.ci = h.d_q_ci;
    a.v = d_qv;
    a.blk = d_blk;
    a.boff = d_boff;
    a.qoff = d_qoff;
    a.order = d_order;
    a.nrows = R;
    a.W = W;
    a.tau = h.o.ilut_tau;
    a.eps = h.o.pivot_eps;
    a.pkeep = pk;
    a.out_ci = d_oci;
    a.out_v = d_ov;
    a.out_nl = d_nl;
    a.out_nu = d_nu;
    a.out_piv = d_piv;
    a.done = d_done;
    a.queue = reinterpret_cast<uint32_t*>(d_misc);
    a.npert = d_misc + 1;
    a.err = d_misc + 2;
    a.spin = h.o.spin_limit ? h.o.spin_limit : (1ull << 22);
    // first a 512-slot table per warp, four warps per CTA; when a row fills it, once more
    // with one warp per CTA and the largest table the shared memory holds
    std::vector<int32_t> misc(4, 0);
    if (e == cudaSuccess) ck(cudaEventRecord(ev0, h.st));
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
    if (e == cudaSuccess) ck(cudaEventRecord(ev1, h.st));
    std::vector<int32_t> nl, nu;
    if (e == cudaSuccess && misc[2] == 0) {
        nl.resize(R);
        nu.resize(R);
        ck(cudaMemcpyAsync(nl.data(), d_nl, (size_t)R * sizeof(int32_t), cudaMemcpyDeviceToHost, h.st));
        ck(cudaMemcpyAsync(nu.data(), d_nu, (size_t)R * sizeof(int32_t), cudaMemcpyDeviceToHost, h.st));
        ck(cudaStreamSynchronize(h.st));
    }
    float kms = 0.0f;
    if (e == cudaSuccess && cudaEventElapsedTime(&kms, ev0, ev1) == cudaSuccess) h.ilut_kernel_ms = kms;
    const int32_t err = misc[2];
    if (e != cudaSuccess || err) {
        release_all();
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ILU_ERR_OOM : ILU_ERR_CUDA;
        if (err & kErrIlutZero) return ILU_ERR_ZERO_PIVOT;
        if (err & kErrIlutWait) return ILU_ERR_TIMEOUT;
        return ILU_ERR_UNSUPPORTED;  // a row wider than the largest table
    }
    h.npert += misc[1];
    // the factor's row pointers and pivot positions in Q order (rows outside the factorised
    // blocks stay empty), then the entries packed on the device
    for (int32_t s = 0; s < p; s++) {
        const int32_t q0 = h.qoff[s], ns = h.qoff[s + 1] - q0, m = boff[s + 1] - boff[s];
        for (int32_t r = 0; r < ns; r++) {
            const int32_t q = q0 + r;
            int32_t c = 0;
            if (r < m) {
                const int32_t g = boff[s] + r;
                c = nl[g] + 1 + nu[g];
                h.f1_dpos[q] = h.f1_rp[q] + nl[g];
            }
            h.f1_rp[q + 1] = h.f1_rp[q] + c;
        }
    }
    const size_t nnz1 = (size_t)h.f1_rp[n];
    d_f1rp = h.alloc<int32_t>((size_t)n + 1, &e);
    d_f1ci = h.alloc<int32_t>(std::max<size_t>(nnz1, 1), &e);
    h.d_f1_stage = h.alloc<double>(std::max<size_t>(nnz1, 1), &e);
    if (e == cudaSuccess) {
        ck(cudaMemcpyAsync(d_f1rp, h.f1_rp.data(), ((size_t)n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, h.st));
        const int grid = std::max(1, std::min(8 * sms, (R + 7) / 8));
        k_ilut_pack<<<grid, 256, 0, h.st>>>(d_oci, d_ov, d_nl, d_nu, d_piv, d_blk, d_boff, d_qoff, d_f1rp, R, pk,
                                            d_f1ci, h.d_f1_stage);
        ck(cudaGetLastError());
        h.kernel_launches += 1;
        h.f1_ci.resize(nnz1);
        if (nnz1) ck(cudaMemcpyAsync(h.f1_ci.data(), d_f1ci, nnz1 * sizeof(int32_t), cudaMemcpyDeviceToHost, h.st));
        ck(cudaStreamSynchronize(h.st));
    }
    release_all();
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ILU_ERR_OOM : ILU_ERR_CUDA;
    return ILU_OK;
}

}  // namespace ilu2l
