// kernels_stream.cu -- the preconditioner apply with TMA-streamed level programs.
//
// The triangular solves are level-scheduled (Sec. 3.1): rows of one level are
// independent, consecutive levels depend on each other, so the apply is bound by the
// latency of one level times the number of levels, not by bytes. Here one CTA serves one
// subdomain:
//   * its level program (stream_layout.h) arrives in fixed-size chunks through a ring of
//     shared-memory stages filled by TMA bulk copies (cp.async.bulk, completion on an
//     mbarrier), issued ahead of use so the global-memory latency overlaps the solve;
//   * a consumer group (one warp, or a few warps on a named barrier) runs the levels on
//     the subdomain's working vector in shared memory; only a warp-level or group
//     barrier separates levels;
//   * the whole CTA performs the coalesced gather of the input and the scatter of the
//     output around the program.
// Every mbarrier wait is bounded: on time-out the kernel sets bit 2 of the device error
// word, stops consuming, waits (bounded) for its own copies in flight, and returns.
//
// Kernels: k_bj_s (block Jacobi), k_fwd_s (f' = L_B^{-1} f, g' = g - W f', c = S~^{-1} g'),
// k_coff (t = C_off v_j, grid-wide), k_inner_a_s (w = v_j + S~^{-1} t, first Gram-Schmidt
// dots), k_bwd_s (y = V t, f'' = f' - Z y, u = U_B^{-1} f'', scatter).
#include <cuda_bf16.h>
#include "devutil.cuh"
#include "handle.h"
#include "inner_lsq.cuh"
#include "stream_layout.h"

namespace ilu2l {

template <class T>
struct StreamDev {
    const uint8_t* blob;
    const int32_t* ch0;
    const int32_t* order;  // p: subdomains by descending estimated cost
    uint32_t chunk;
    int nt;
};

// The subdomain of this CTA in the block-Jacobi, forward and backward kernels: the CTAs take
// the subdomains most expensive first. When there are more subdomains than resident CTAs,
// the block scheduler hands out CTAs in index order as SMs free up, so this is longest-first
// list scheduling of uneven subdomains onto the SMs (the kernels of the inner solve keep one
// CTA per subdomain in index order: its grid barriers need every CTA resident anyway).
template <class T>
__device__ __forceinline__ int sub_of_cta(const StreamDev<T>& S) {
    return S.order ? S.order[blockIdx.x] : (int)blockIdx.x;
}

struct RingCfg {
    int nst;              // stages
    int32_t smem_len;     // working-vector capacity in shared memory (elements)
    uint64_t spin;        // bound of every mbarrier wait
    int32_t* err;         // device error word
};

constexpr int kErrTimeout = 2;
// Bound of the wait for a CTA's own bulk copies before it exits after a time-out: copies
// from valid global memory always complete, this only keeps the wait finite.
constexpr uint64_t kDrainSpin = 1ull << 20;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            saddr(dst)),
        "l"(src), "r"(bytes), "r"(saddr(b))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, uint64_t spin) {
    for (uint64_t i = 0; i < spin; i++)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}

__device__ __forceinline__ void group_sync(int nt) {
    if (nt <= 32)
        __syncwarp();
    else
        asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
}

// Release of a ring stage by one consumer thread (the stage's "empty" barrier counts all
// consumer threads; arrive has release semantics, the producer's wait acquires).
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}

// True in every consumer thread iff v holds in all of them (a group barrier).
__device__ __forceinline__ bool group_all(bool v, int nt) {
    if (nt <= 32) return __all_sync(kFull, v);
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.and.pred po, 1, %2, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(nt)
        : "memory");
    return r != 0;
}

// Shared-memory layout of every stream kernel:
// [mbarriers 128 B: full[nst], empty[nst]][ring nst*chunk][x ...]
struct Smem {
    uint64_t* bars;
    uint8_t* ring;
    uint8_t* xs;
};

__device__ __forceinline__ Smem smem_parts(int nst, uint32_t chunk) {
    extern __shared__ __align__(128) uint8_t sm_raw[];
    Smem s;
    s.bars = reinterpret_cast<uint64_t*>(sm_raw);
    s.ring = sm_raw + 128;
    s.xs = sm_raw + 128 + (size_t)nst * chunk;
    return s;
}

// thread 0: initialise the stage barriers and start the first copies of subdomain s
template <class T>
__device__ __forceinline__ void ring_start(const StreamDev<T>& S, int s, const Smem& sm, int nst) {
    if (threadIdx.x != 0) return;
    for (int i = 0; i < nst; i++) {
        mbar_init(&sm.bars[i], 1);            // full: the copy's bytes arrived
        mbar_init(&sm.bars[nst + i], S.nt);   // empty: every consumer thread is done with it
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const int c0 = S.ch0[s], nch = S.ch0[s + 1] - c0;
    const uint8_t* base = S.blob + (size_t)c0 * S.chunk;
    for (int c = 0; c < nch && c < nst; c++) {
        mbar_expect_tx(&sm.bars[c], S.chunk);
        tma_load_1d(sm.ring + (size_t)c * S.chunk, base + (size_t)c * S.chunk, S.chunk, &sm.bars[c]);
    }
}

__device__ __forceinline__ void mbar_inval(uint64_t* b) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(saddr(b)) : "memory");
}

// Before a further run of the same program in one kernel (all threads call it): when the
// whole program stays in the ring no copy is needed (a second pass finds every stage's
// phase complete); otherwise thread 0 re-initialises the drained barriers and restarts
// the copies. Every copy of the previous run has landed (ring_produce drains them).
template <class T>
__device__ __forceinline__ void ring_rearm(const StreamDev<T>& S, int s, const Smem& sm, int nst) {
    if (S.ch0[s + 1] - S.ch0[s] <= nst) return;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = 0; i < 2 * nst; i++) mbar_inval(&sm.bars[i]);
    ring_start(S, s, sm, nst);
    __syncthreads();
}

// Row record (stream_layout.h), read with 128-bit shared-memory loads. V is the storage
// type of the values: T, or bfloat16 for T = float (values widened on use).
template <class T, int RW, class V = T>
struct __align__(16) RowRec {
    uint32_t head;  // element index of x[row] | n << 24 | skip bit
    T dinv;
    uint32_t col[RW];  // byte offsets (unused entries: the row's own)
    V val[RW];         // (unused entries: zero)
};

template <class T, int RW, class V = T>
union RecU {
    RowRec<T, RW, V> r;
    uint4 v[sizeof(RowRec<T, RW, V>) / 16];
};

template <class T, class V>
__device__ __forceinline__ T widen(V v) {
    return (T)v;
}
template <>
__device__ __forceinline__ float widen<float, __nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

template <class T, int RW, class V>
__device__ __forceinline__ void rec_load(RecU<T, RW, V>& u, const uint8_t* p) {
    constexpr int NV = sizeof(RowRec<T, RW, V>) / 16;
    static_assert(sizeof(RowRec<T, RW, V>) == rec_layout(RW, sizeof(V), sizeof(T)).bytes, "record layout");
    const uint4* s = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int i = 0; i < NV; i++) u.v[i] = s[i];
}

// byte offset of a record's own slot x[row] (the head holds the row's element index)
template <class T>
__device__ __forceinline__ uint32_t row_byte(uint32_t head) {
    return (head & 0xFFFFFFu) * (uint32_t)sizeof(T);
}

template <class T>
__device__ __forceinline__ T ldx(const uint8_t* xb, uint32_t off) {
    return *reinterpret_cast<const T*>(xb + off);
}

// operands of a record: x[col[q]] and x[row]
template <class T, int RW, class V>
__device__ __forceinline__ void rec_operands(const RecU<T, RW, V>& u, const uint8_t* xb, T (&xc)[RW], T& xr) {
#pragma unroll
    for (int q = 0; q < RW; q++) xc[q] = ldx<T>(xb, u.r.col[q]);
    xr = ldx<T>(xb, row_byte<T>(u.r.head));
}

// x[row] = (x[row] - sum_q val[q] x[col[q]]) * dinv, the sum formed pairwise
template <class T, int RW, class V>
__device__ __forceinline__ T rec_value(const RecU<T, RW, V>& u, const T (&xc)[RW], T xr) {
    T p[RW];
#pragma unroll
    for (int q = 0; q < RW; q++) p[q] = widen<T, V>(u.r.val[q]) * xc[q];
#pragma unroll
    for (int w = 1; w < RW; w *= 2)
#pragma unroll
        for (int q = 0; q + w < RW; q += 2 * w) p[q] += p[q + w];
    return (xr - p[0]) * u.r.dinv;
}

// One consumer thread's column of a segment: records p, p + stride, ... (nw of them; the
// first one already in registers).
// Software-pipelined: the record two ahead is loaded, and the operands of the next row
// are loaded before the current row's arithmetic; where the next row reads the slot
// the current row writes, the value is forwarded in registers (the early load predates
// the store). Every address stays inside the chunk and the working vector: past the
// end the pipeline reloads the segment's first record.
template <class T, int RW, class V>
__device__ __forceinline__ void run_segment(const RecU<T, RW, V>& first, const uint8_t* p, uint32_t stride, uint32_t nw,
                                            uint8_t* xb) {
    RecU<T, RW, V> a = first, b;
    T xa[RW], xra;
    rec_operands(a, xb, xa, xra);
    if (nw == 1) {  // a single wave: no pipeline
        if ((a.r.head & kRecSkip) == 0) *reinterpret_cast<T*>(xb + row_byte<T>(a.r.head)) = rec_value(a, xa, xra);
        return;
    }
    rec_load(b, p + (nw > 1 ? stride : 0u));
    for (uint32_t w = 0; w < nw; w++) {
        T xn[RW], xrn;
        rec_operands(b, xb, xn, xrn);
        RecU<T, RW, V> c;
        rec_load(c, p + (w + 2 < nw ? (w + 2) * stride : 0u));
        const uint32_t ha = a.r.head;
        const T v = rec_value(a, xa, xra);
        const bool real = (ha & kRecSkip) == 0;
        const uint32_t fwd = real ? row_byte<T>(ha) : 0xFFFFFFFFu;
        if (real) *reinterpret_cast<T*>(xb + fwd) = v;
#pragma unroll
        for (int q = 0; q < RW; q++) xa[q] = (b.r.col[q] == fwd) ? v : xn[q];
        xra = (row_byte<T>(b.r.head) == fwd) ? v : xrn;
        a = b;
        b = c;
    }
}

// One warp's part of a scan segment (stream_layout.h): lane l runs record l of each of its
// nw waves. A linked record's predecessor is the record one lane below (or, for lane 0,
// the previous wave's last record, already stored): lane l forms x_l = a_l + b_l x_{l-1}
// with a_l from the values final before the wave -- x[row] and its columns, the linked
// one left out -- and b_l = -val[0] / u_ll (column link) or 1 / u_ll (own-slot link), 0
// without a link. Five shuffle rounds compose the maps (Kogge-Stone inclusive scan); a lane
// whose map no longer depends on lower lanes (b = 0) keeps its value, so an unlinked row
// gives exactly the level formula's operations. Loads of the wave precede its stores
// (the shuffles join them), so a row may overwrite a slot an earlier row of the wave read.
// The lanes store in one instruction, so of two rows of a wave writing one slot (a row and
// its successor linked through that slot) only the later stores.
template <class T, int RW, class V>
__device__ __forceinline__ void run_scan_segment(const RecU<T, RW, V>& first, const uint8_t* p, uint32_t stride,
                                                 uint32_t nw, uint8_t* xb) {
    const uint32_t lane = threadIdx.x & 31u;
    RecU<T, RW, V> a = first, b;
    for (uint32_t w = 0; w < nw; w++) {
        rec_load(b, p + (w + 1 < nw ? (w + 1) * stride : 0u));
        T xc[RW], xr;
        rec_operands(a, xb, xc, xr);
        const uint32_t hd = a.r.head;
        const bool lc = lane != 0 && (hd & kRecLinkCol) != 0;
        const bool ls = lane != 0 && (hd & kRecLinkSelf) != 0;
        T pv[RW];
#pragma unroll
        for (int q = 0; q < RW; q++) pv[q] = widen<T, V>(a.r.val[q]) * xc[q];
        if (lc) pv[0] = (T)0;
#pragma unroll
        for (int d = 1; d < RW; d *= 2)
#pragma unroll
            for (int q = 0; q + d < RW; q += 2 * d) pv[q] += pv[q + d];
        const T dinv = a.r.dinv;
        T al = ((ls ? (T)0 : xr) - pv[0]) * dinv;
        T be = lc ? -widen<T, V>(a.r.val[0]) * dinv : (ls ? dinv : (T)0);
#pragma unroll
        for (int d = 1; d < 32; d *= 2) {
            const T au = __shfl_up_sync(kFull, al, d);
            const T bu = __shfl_up_sync(kFull, be, d);
            if (lane >= (uint32_t)d && be != (T)0) {
                al = fma(be, au, al);
                be = be * bu;
            }
        }
        // the lanes of a wave store together: a row whose successor (one lane up) is linked
        // through the same slot leaves the slot to it
        const bool succ_self = __shfl_down_sync(kFull, (hd & kRecLinkSelf) != 0 ? 1 : 0, 1) != 0 && lane < 31;
        if ((hd & kRecSkip) == 0 && !succ_self) *reinterpret_cast<T*>(xb + row_byte<T>(hd)) = al;
        __syncwarp();
        a = b;
    }
}

// A run of levels (segment bit kSegSyncEach): wave w is one level, the group meets at its
// barrier after every wave. Every consumer thread runs the loop (the barrier counts all of
// them), and without a branch: a thread beyond the segment's width works on a stand-in --
// p points at the wave's first record -- and does not store (a divergent branch around
// the row costs more than the row on GB300). A thread loads its operands right after the
// barrier -- the record's column offsets are already in registers -- forms the row, stores
// it, and only then loads the record two levels ahead, so the dependent path of a level
// is operand loads, the product, the store and the barrier.
template <class T, int RW, class V>
__device__ __forceinline__ void run_level_segment(const RecU<T, RW, V>& first, const uint8_t* p, uint32_t stride,
                                                  uint32_t nw, uint8_t* xb, bool mine, int nt) {
    RecU<T, RW, V> a = first, b;
    rec_load(b, p + (nw > 1 ? stride : 0u));
    for (uint32_t w = 0; w < nw; w++) {
        T xc[RW], xr;
        rec_operands(a, xb, xc, xr);
        const T v = rec_value(a, xc, xr);
        if (mine && (a.r.head & kRecSkip) == 0) *reinterpret_cast<T*>(xb + row_byte<T>(a.r.head)) = v;
        a = b;
        rec_load(b, p + (w + 2 < nw ? (w + 2) * stride : 0u));
        group_sync(nt);
    }
}

// The refill side of the ring (one thread outside the consumer group): chunk c >= nst
// goes into stage c % nst once every consumer thread released chunk c - nst. Stops when
// the consumers abort or a wait runs out, then waits (bounded) until every copy it or
// ring_start issued has landed, so none is in flight when the block exits.
template <class T>
__device__ void ring_produce(const StreamDev<T>& S, int s, const Smem& sm, const RingCfg& cfg,
                             volatile int* abort_flag) {
    const int nst = cfg.nst;
    const int c0 = S.ch0[s], nch = S.ch0[s + 1] - c0;
    const uint8_t* base = S.blob + (size_t)c0 * S.chunk;
    int issued = nch < nst ? nch : nst;
    for (int c = nst; c < nch; c++) {
        uint64_t* empty = &sm.bars[nst + c % nst];
        const uint32_t par = (uint32_t)(c / nst - 1) & 1u;
        bool ok = false;
        for (uint64_t i = 0; i < cfg.spin && !ok; i++) {
            ok = mbar_try_wait(empty, par);
            if (!ok && *abort_flag) break;
        }
        if (!ok) {
            if (!*abort_flag) {
                atomicOr(cfg.err, kErrTimeout);
                *abort_flag = 1;
            }
            break;
        }
        mbar_expect_tx(&sm.bars[c % nst], S.chunk);
        tma_load_1d(sm.ring + (size_t)(c % nst) * S.chunk, base + (size_t)c * S.chunk, S.chunk, &sm.bars[c % nst]);
        issued = c + 1;
    }
    for (int d = issued - nst < 0 ? 0 : issued - nst; d < issued; d++)
        mbar_wait(&sm.bars[d % nst], (uint32_t)(d / nst) & 1u, kDrainSpin);
}

// Run the program of subdomain s on x. Threads 0..nt-1 consume; thread nt refills the
// ring. The caller passes whole warps: threads 0..nt+31 (the first barrier below counts
// the consumer warps and the refill warp). Returns false on a time-out (uniform over
// the consumer group; bit 2 of the device error word is set).
template <class T, int RW, class V = T>
__device__ bool ring_run(const StreamDev<T>& S, int s, const Smem& sm, const RingCfg& cfg, T* x) {
    constexpr uint32_t RB = sizeof(RowRec<T, RW, V>);
    __shared__ int abort_flag;
    const int nt = S.nt, tid = threadIdx.x, nst = cfg.nst;
    const int c0 = S.ch0[s], nch = S.ch0[s + 1] - c0;
    uint8_t* xb = reinterpret_cast<uint8_t*>(x);
    if (nch == 0) return true;
    if (tid == 0) abort_flag = 0;
    asm volatile("bar.sync 1, %0;" ::"r"(nt + 32) : "memory");  // consumers + the refill warp
    if (tid >= nt) {
        if (tid == nt) ring_produce(S, s, sm, cfg, &abort_flag);
        return true;
    }
    for (int c = 0; c < nch; c++) {
        const bool got = mbar_wait(&sm.bars[c % nst], (uint32_t)(c / nst) & 1u, cfg.spin);
        if (!group_all(got, nt)) {
            if (tid == 0) {
                atomicOr(cfg.err, kErrTimeout);
                *(volatile int*)&abort_flag = 1;
            }
            return false;
        }
        const uint8_t* cb = sm.ring + (size_t)(c % nst) * S.chunk;
        const uint32_t nseg = *reinterpret_cast<const uint32_t*>(cb);
        const uint2* tab = reinterpret_cast<const uint2*>(cb + kChunkHdr);
        // Lookahead: while segment g runs, the table entry of g + 2 and the first record of
        // g + 1 are in flight, so a level costs its operand loads, arithmetic and barrier.
        // (Every chunk holds at least one segment; reads past the table's end re-read it.)
        // a thread beyond a segment's width addresses its first record instead (loads stay
        // in the chunk and need no branch; such a thread never stores)
        auto mine = [&](uint2 e) { return (uint32_t)tid < ((e.x >> 16) & 0x1FFu); };
        auto first_of = [&](uint2 e) { return cb + (e.x & 0xFFFFu) * 16u + (mine(e) ? (uint32_t)tid * RB : 0u); };
        uint2 e = tab[0];
        uint2 en = tab[nseg > 1 ? 1 : 0];
        RecU<T, RW, V> r;
        rec_load(r, first_of(e));
        for (uint32_t g = 0; g < nseg; g++) {
            const uint2 enn = tab[g + 2 < nseg ? g + 2 : 0];
            RecU<T, RW, V> rn;
            rec_load(rn, first_of(en));
            if (e.y & kSegSyncEach) {
                run_level_segment<T, RW, V>(r, first_of(e), ((e.x >> 16) & 0x1FFu) * RB, e.y & 0xFFFFu, xb, mine(e),
                                            nt);
            } else {
                if (mine(e)) {
                    if (e.y & kSegScan)
                        run_scan_segment<T, RW, V>(r, first_of(e), ((e.x >> 16) & 0x1FFu) * RB, e.y & 0xFFFFu, xb);
                    else
                        run_segment<T, RW, V>(r, first_of(e), ((e.x >> 16) & 0x1FFu) * RB, e.y & 0xFFFFu, xb);
                }
                if (e.y & kSegBarrier) group_sync(nt);
            }
            e = en;
            en = enn;
            r = rn;
        }
        mbar_arrive(&sm.bars[nst + c % nst]);
    }
    return true;
}

// Gather / scatter / copy with several independent loads in flight per thread (the loads
// of a subdomain's vector sit on the critical path before its level program starts).
template <class T>
__device__ __forceinline__ void gather(T* x, const double* __restrict__ r, const int32_t* __restrict__ idx, int n) {
    const int stride = blockDim.x;
    int l = threadIdx.x;
    for (; l + 3 * stride < n; l += 4 * stride) {  // four: the first chunk copies run meanwhile
        int i[4];
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) i[u] = idx[l + u * stride];
#pragma unroll
        for (int u = 0; u < 4; u++) v[u] = r[i[u]];
#pragma unroll
        for (int u = 0; u < 4; u++) x[l + u * stride] = (T)v[u];
    }
    for (; l < n; l += stride) x[l] = (T)r[idx[l]];
}

template <class T>
__device__ __forceinline__ void copy_in(T* x, const T* __restrict__ src, int n) {
    const int stride = blockDim.x;
    int l = threadIdx.x;
    for (; l + 7 * stride < n; l += 8 * stride) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; u++) v[u] = src[l + u * stride];
#pragma unroll
        for (int u = 0; u < 8; u++) x[l + u * stride] = v[u];
    }
    for (; l < n; l += stride) x[l] = src[l];
}

template <class T>
__device__ __forceinline__ void scatter(double* __restrict__ z, const T* x, const int32_t* __restrict__ idx, int n) {
    const int stride = blockDim.x;
    int l = threadIdx.x;
    for (; l + 7 * stride < n; l += 8 * stride) {
        int i[8];
#pragma unroll
        for (int u = 0; u < 8; u++) i[u] = idx[l + u * stride];
#pragma unroll
        for (int u = 0; u < 8; u++) z[i[u]] = (double)x[l + u * stride];
    }
    for (; l < n; l += stride) z[idx[l]] = (double)x[l];
}

// ---------------------------------------------------------------------------------------
// Working vector: in shared memory (XS, every subdomain fits; the pointer comes straight
// from the shared array so the compiler emits shared loads) or a global scratch slice.
template <class T, bool XS>
__device__ __forceinline__ T* xvec(const Smem& sm, T* xg, int q0) {
    if constexpr (XS) {
        extern __shared__ __align__(128) uint8_t sm_raw[];
        return reinterpret_cast<T*>(sm_raw + (sm.xs - sm.ring) + 128);
    } else {
        return xg + q0;
    }
}

template <class T, int RW, bool XS, class V = T>
__global__ void __launch_bounds__(256) k_bj_s(SubDev sd, StreamDev<T> S, RingCfg cfg, const double* __restrict__ r,
                                              double* __restrict__ z, T* xg, const int32_t* done) {
    if (done && *done) return;
    const int s = sub_of_cta(S);
    const int q0 = sd.qoff[s], ns = sd.qoff[s + 1] - q0;
    const Smem sm = smem_parts(cfg.nst, S.chunk);
    ring_start(S, s, sm, cfg.nst);
    T* x = xvec<T, XS>(sm, xg, q0);
    gather(x, r, sd.q_orig + q0, ns);
    __syncthreads();
    if ((int)threadIdx.x < S.nt + 32) ring_run<T, RW, V>(S, s, sm, cfg, x);
    __syncthreads();
    scatter(z, x, sd.q_orig + q0, ns);
}

template <class T, int RW, bool XS, class V = T>
__global__ void __launch_bounds__(256) k_fwd_s(SubDev sd, StreamDev<T> S, RingCfg cfg, InnerDev<T> in,
                                               const double* __restrict__ r, T* __restrict__ fq, T* xg,
                                               const int32_t* done) {
    __shared__ double red[32];
    if (done && *done) return;
    const int s = sub_of_cta(S);
    const int q0 = sd.qoff[s], ns = sd.qoff[s + 1] - q0, ni = sd.nint[s], nf = ns - ni;
    const Smem sm = smem_parts(cfg.nst, S.chunk);
    ring_start(S, s, sm, cfg.nst);
    T* x = xvec<T, XS>(sm, xg, q0);
    gather(x, r, sd.q_orig + q0, ns);
    __syncthreads();
    if ((int)threadIdx.x < S.nt + 32) ring_run<T, RW, V>(S, s, sm, cfg, x);
    __syncthreads();
    for (int l = threadIdx.x; l < ni; l += blockDim.x) fq[q0 + l] = x[l];
    const int g0 = sd.if_ptr[s];
    T acc = (T)0;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        const T c = x[ni + i];
        in.W0[g0 + i] = c;
        acc += c * c;
    }
    acc = block_sum_t<T>(acc, reinterpret_cast<T*>(red));
    if (threadIdx.x == 0) {
        in.part[((size_t)2 * (kMaxInner + 1)) * sd.p + s] = (double)acc;
        if (s == 0) {
            in.ctl->steps = -1;
            in.ctl->zero = 0;
            in.ctl->gbar_count = 0;
            in.ctl->gbar_abort = 0;
        }
    }
}

// t = C_off v_j with v_j = W_in / ||W_in|| (the norm formed from the per-subdomain
// partials in a fixed order); grid-wide, rows of the interface.
template <class T>
__global__ void k_coff(SubDev sd, InnerDev<T> in, int j, T* __restrict__ t, const int32_t* done) {
    if (done && *done) return;
    const InnerCtl* ctl = in.ctl;
    if (*((volatile const int32_t*)&ctl->steps) >= 0 || *((volatile const int32_t*)&ctl->zero)) return;
    const int p = sd.p;
    const double nrm2 = warp_allsum_ldcg(in.part + ((size_t)2 * (kMaxInner + 1)) * p, p);
    if (nrm2 == 0.0) return;
    const T inv = (T)(1.0 / sqrt(nrm2));
    const T* __restrict__ Win = (j & 1) ? in.W1 : in.W0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < sd.n2; i += gridDim.x * blockDim.x) {
        T acc = (T)0;
        for (int q = in.coff_rp[i]; q < in.coff_rp[i + 1]; q++) acc += in.coff_v[q] * Win[in.coff_ci[q]];
        t[i] = acc * inv;
    }
}

template <class T, int RW, bool XS, class V = T>
__global__ void __launch_bounds__(256) k_inner_a_s(SubDev sd, StreamDev<T> S, RingCfg cfg, InnerDev<T> in, int j,
                                                   const T* __restrict__ t, T* xg, const int32_t* done) {
    __shared__ double red[32 * 8];
    if (done && *done) return;
    InnerCtl* ctl = in.ctl;
    if (*((volatile int32_t*)&ctl->steps) >= 0 || *((volatile int32_t*)&ctl->zero)) return;
    const int s = blockIdx.x, p = sd.p, n2 = sd.n2;
    const int q0 = sd.qoff[s], ns = sd.qoff[s + 1] - q0, ni = sd.nint[s], nf = ns - ni;
    const double nrm = sqrt(warp_allsum_ldcg(in.part + ((size_t)2 * (kMaxInner + 1)) * p, p));
    if (j == 0) {
        if (s == 0 && threadIdx.x == 0) ctl->beta = nrm;
        if (nrm == 0.0) {
            if (s == 0 && threadIdx.x == 0) ctl->zero = 1;
            return;
        }
    } else {
        const double beta = ctl->beta;
        if (s == 0 && threadIdx.x == 0) ctl->H[(j - 1) * (kMaxInner + 1) + j] = nrm;
        if (nrm <= 1e-14 * beta) {
            if (s == 0 && threadIdx.x == 0) ctl->steps = j;
            return;
        }
    }
    const Smem sm = smem_parts(cfg.nst, S.chunk);
    ring_start(S, s, sm, cfg.nst);
    const T inv = (T)(1.0 / nrm);
    const T* __restrict__ Win = (j & 1) ? in.W1 : in.W0;
    T* __restrict__ Wout = (j & 1) ? in.W0 : in.W1;
    const int g0 = sd.if_ptr[s];
    T* x = xvec<T, XS>(sm, xg + ni, q0);
    for (int i = threadIdx.x; i < nf; i += blockDim.x) x[i] = t[g0 + i];
    __syncthreads();
    if ((int)threadIdx.x < S.nt + 32) ring_run<T, RW, V>(S, s, sm, cfg, x);
    __syncthreads();
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
            for (int u = 0; u < 8 && i0 + u <= j; u++) in.part[((size_t)(i0 + u)) * p + s] = (double)acc[u];
    }
}

// Grid-wide barrier of the single-launch inner solve (a cooperative launch guarantees
// that every CTA is resident). The arrival counter only grows within a launch (the kernel
// that starts the inner solve clears it): at its b-th barrier (b = 1, 2, ...) thread 0 of
// each CTA adds 1 with release-acquire semantics -- publishing the CTA's partial sums,
// ordered before it by the block barrier -- and waits, with acquire loads, until the
// counter reaches b * nblocks. One atomic and one observed store per barrier; no fences.
// Waits are bounded: a CTA that gives up sets bit 2 of the device error word and the abort
// word, which ends the others' waits too. Returns false (uniform over the CTA) after an
// abort.
__device__ bool grid_sync(InnerCtl* ctl, uint32_t nblocks, uint32_t& epoch, uint64_t spin, int32_t* err) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        epoch++;
        const uint32_t target = epoch * nblocks;
        uint32_t v;
        asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(v) : "l"(&ctl->gbar_count) : "memory");
        int ok = 1;
        if (v + 1 != target) {
            volatile int32_t* abort = &ctl->gbar_abort;
            for (uint64_t i = 0;; i++) {
                asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(&ctl->gbar_count) : "memory");
                if ((int32_t)(v - target) >= 0) break;
                if (*abort || i >= spin) {
                    ok = 0;
                    break;
                }
            }
        }
        if (!ok || *(volatile int32_t*)&ctl->gbar_abort) {
            ok = 0;
            atomicOr(err, kErrTimeout);
            *(volatile int32_t*)&ctl->gbar_abort = 1;
        }
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// terms of the deferred second Gram-Schmidt update w2 = w1 - V h2 that the next step forms
// where it needs an entry (later steps store w2 and pass a third barrier)
constexpr int kLazyMax = 3;

// w - sum_t h[t] V_t, t < nt <= kLazyMax, at entry gi of the interface: the loads issued
// together, then one explicitly rounded fused multiply-add per term, so every CTA that
// evaluates it (the owner of the row and the CTAs that gather it through C_off) obtains the
// same bits
template <class T>
__device__ __forceinline__ T lazy_sub(T w, const T* __restrict__ V, const T* hv, int nt, int n2, int gi) {
    T vv[kLazyMax];
#pragma unroll
    for (int t = 0; t < kLazyMax; t++) vv[t] = t < nt ? __ldcg(V + (size_t)t * n2 + gi) : (T)0;
#pragma unroll
    for (int t = 0; t < kLazyMax; t++)
        if (t < nt) w = fma_rn(-hv[t], vv[t], w);
    return w;
}

// All k steps of the inner GMRES on the preconditioned Schur system (Eq. preSS) in one
// cooperative launch, one CTA per subdomain, W0 = c = S~^{-1} g' and its norm partials
// left by the forward kernel. Step j, with two grid barriers:
//   A: v_j = w2 / ||w2|| of the previous step (or W0 / ||W0||); t = C_off v_j on the CTA's
//      interface rows, the entries of other CTAs formed from what they stored; x = S~_s^{-1}
//      t (the streamed local Schur program); w = v_j + x; partial dots V_i . w (i <= j)
//   B: h1 = sum of the partials (every CTA, fixed order); w1 = w - V h1, stored for the
//      other CTAs; partial dots V_i . w1 and partial ||w1||^2
//   C: h2 likewise; ||w2||^2 = ||w1||^2 - ||h2||^2 (w1 = w2 + V h2 with V h2 orthogonal to
//      w2), the same in every CTA. The next step forms v_{j+1} = (w1 - V h2) / ||w2||
//      wherever it needs an entry, so no barrier closes C. If the subtraction cancels
//      (||w2||^2 <= 1e-2 ||w1||^2, near a breakdown), or from step kLazyMax on, the step
//      falls back to w2 stored explicitly, its norm partials and a third barrier. The last step stores w2 and its
//      norm partials for the least squares of k_bwd_s, which starts after this launch.
// The Hessenberg entries go to ctl (CTA 0). Every CTA forms each norm from the same partials
// in the same order, so the stopping decisions (c = 0, breakdown) are uniform and no CTA
// leaves the barriers early.
template <class T, int RW, bool XS, class V = T>
__global__ void __launch_bounds__(256) k_inner_coop(SubDev sd, StreamDev<T> S, RingCfg cfg, InnerDev<T> in, T* xg,
                                                    const int32_t* done) {
    __shared__ double red[32 * 8];
    __shared__ double hh[kMaxInner + 1];
    __shared__ T hT[kMaxInner + 1];   // the current coefficients in T
    __shared__ T hlz[kMaxInner + 1];  // h2 of the previous step, for w2 = w1 - V h2
    // per-step scalars, formed by thread 0 only (GB300 issues FP64 at 1/64 of its FP32 rate,
    // so a square root or a division in every warp costs thousands of cycles), in the
    // preconditioner type T: the inner GMRES is part of the preconditioner, and with T =
    // float its vectors and partial sums carry FP32 accuracy anyway
    using ST = T;
    __shared__ double nrm_s, beta_s, a_s;
    __shared__ T inv_s;
    __shared__ int stop_s, lazy_s;
    if (done && *done) return;
    InnerCtl* ctl = in.ctl;
    const int s = blockIdx.x, p = sd.p, n2 = sd.n2, tid = threadIdx.x;
    const int q0 = sd.qoff[s], ns = sd.qoff[s + 1] - q0, ni = sd.nint[s], nf = ns - ni;
    const int g0 = sd.if_ptr[s];
    const Smem sm = smem_parts(cfg.nst, S.chunk);
    T* x = xvec<T, XS>(sm, xg + ni, q0);
    double* const nbank = in.part + ((size_t)2 * (kMaxInner + 1)) * p;  // ||w||^2 partials
    double* const nbank2 = nbank + p;                                     // fallback ||w2||^2
    uint32_t gepoch = 0;  // grid barriers passed (thread 0)
    // thread 0: the norm of v_j's numerator is nrm; stopping tests, 1 / nrm
    auto set_norm = [&](int j, ST nrm_t) {
        const double nrm = (double)nrm_t;
        nrm_s = nrm;
        int stop = 0;
        if (j == 0) {
            beta_s = nrm;
            if (s == 0) ctl->beta = nrm;
            if (nrm == 0.0) {
                if (s == 0) ctl->zero = 1;
                stop = 1;
            }
        } else {
            if (s == 0) ctl->H[(j - 1) * (kMaxInner + 1) + j] = nrm;
            if (nrm <= 1e-14 * beta_s) {  // lucky breakdown: the Krylov space is exhausted
                if (s == 0) ctl->steps = j;
                stop = 1;
            }
        }
        stop_s = stop;
        inv_s = stop ? (T)0 : (T)1 / nrm_t;
    };
    if (tid < 32) {
        const double a = warp_allsum_ldcg(nbank, p);
        if (tid == 0) {
            set_norm(0, (ST)sqrt((ST)a));
            lazy_s = 0;
        }
    }
    __syncthreads();
    for (int j = 0; j < in.k; j++) {
        // ---- A
        if (stop_s) break;
        const T inv = inv_s;
        const int nlz = lazy_s ? j : 0;  // terms of the correction w1 - V h2
        const T* __restrict__ Win = (j & 1) ? in.W1 : in.W0;
        T* __restrict__ Wout = (j & 1) ? in.W0 : in.W1;
        // copies start only past the stopping tests: every copy issued is consumed (and
        // drained) by the ring_run below
        if (j == 0)
            ring_start(S, s, sm, cfg.nst);
        else
            ring_rearm(S, s, sm, cfg.nst);
        for (int i = tid; i < nf; i += blockDim.x) {
            const int gi = g0 + i;
            const int qa = in.coff_rp[gi], qb = in.coff_rp[gi + 1];
            T acc = (T)0;
            for (int q0 = qa; q0 < qb; q0 += 4) {  // four gathers in flight, summed in order
                T cv[4], wv[4];
                int c[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const bool ok = q0 + u < qb;
                    c[u] = ok ? in.coff_ci[q0 + u] : 0;
                    cv[u] = ok ? in.coff_v[q0 + u] : (T)0;
                }
                if (nlz) {
                    // the gathers and their correction terms issued together
                    T vv[4][kLazyMax];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const bool ok = q0 + u < qb;
                        wv[u] = ok ? __ldcg(Win + c[u]) : (T)0;
#pragma unroll
                        for (int t = 0; t < kLazyMax; t++)
                            vv[u][t] = (ok && t < nlz) ? __ldcg(in.V + (size_t)t * n2 + c[u]) : (T)0;
                    }
#pragma unroll
                    for (int u = 0; u < 4; u++)
#pragma unroll
                        for (int t = 0; t < kLazyMax; t++)
                            if (t < nlz) wv[u] = fma_rn(-hlz[t], vv[u][t], wv[u]);
                } else {
#pragma unroll
                    for (int u = 0; u < 4; u++) wv[u] = (q0 + u < qb) ? __ldcg(Win + c[u]) : (T)0;
                }
#pragma unroll
                for (int u = 0; u < 4; u++) acc += cv[u] * wv[u];
            }
            x[i] = acc * inv;
        }
        __syncthreads();
        if (tid < S.nt + 32) ring_run<T, RW, V>(S, s, sm, cfg, x);
        __syncthreads();
        T* Vj = in.V + (size_t)j * n2;
        for (int i = tid; i < nf; i += blockDim.x) {
            const int gi = g0 + i;
            T wv = __ldcg(Win + gi);
            if (nlz) wv = lazy_sub<T>(wv, in.V, hlz, nlz, n2, gi);
            const T v = wv * inv;
            Vj[gi] = v;
            x[i] = v + x[i];
        }
        __syncthreads();
        const bool last = j + 1 == in.k;
        for (int bank = 0; bank < 2; bank++) {
            // partial dots V_i . w, i <= j, into bank 0 (A) or 1 (B)
            for (int i0 = 0; i0 <= j; i0 += 8) {
                T acc[8];
#pragma unroll
                for (int u = 0; u < 8; u++) acc[u] = (T)0;
                for (int i = tid; i < nf; i += blockDim.x) {
                    const T w = x[i];
#pragma unroll
                    for (int u = 0; u < 8; u++)
                        if (i0 + u <= j) acc[u] += in.V[(size_t)(i0 + u) * n2 + g0 + i] * w;
                }
                block_sum_nt<T, 8>(acc, reinterpret_cast<T*>(red));
                if (tid == 0)
                    for (int u = 0; u < 8 && i0 + u <= j; u++)
                        in.part[((size_t)(bank * (kMaxInner + 1) + i0 + u)) * p + s] = (double)acc[u];
            }
            if (bank == 1 && !last) {
                // ||w1||^2 beside the second dots
                T n1 = (T)0;
                for (int i = tid; i < nf; i += blockDim.x) n1 += x[i] * x[i];
                n1 = block_sum_t<T>(n1, reinterpret_cast<T*>(red));
                if (tid == 0) nbank[s] = (double)n1;
            }
            if (!grid_sync(ctl, (uint32_t)p, gepoch, cfg.spin, cfg.err)) return;
            // ---- B (bank 0) / C (bank 1): coefficients, Hessenberg column, update
            {
                const int lane = tid & 31, nw = blockDim.x >> 5;
                for (int i = tid >> 5; i <= j; i += nw) {
                    const double h = warp_allsum_ldcg(in.part + ((size_t)(bank * (kMaxInner + 1) + i)) * p, p);
                    if (lane == 0) {
                        hh[i] = h;
                        hT[i] = (T)h;
                    }
                }
                // the last warp sums the ||w1||^2 partials (its coefficients, if any, are done)
                if (bank == 1 && !last && (tid >> 5) == nw - 1) {
                    const double a = warp_allsum_ldcg(nbank, p);
                    if (lane == 0) a_s = a;
                }
            }
            __syncthreads();
            if (s == 0 && tid == 0)
                for (int i = 0; i <= j; i++) {
                    double& H = ctl->H[j * (kMaxInner + 1) + i];
                    H = bank ? H + hh[i] : hh[i];
                }
            if (bank == 0) {
                for (int i = tid; i < nf; i += blockDim.x) {
                    T w = x[i];
                    for (int t = 0; t <= j; t++) w -= hT[t] * in.V[(size_t)t * n2 + g0 + i];
                    x[i] = w;
                    Wout[g0 + i] = w;  // w1, read by the other CTAs in the next step
                }
                __syncthreads();
                continue;
            }
            // C: ||w2||^2 = ||w1||^2 - ||h2||^2, the same in every CTA (thread 0 forms it)
            if (tid == 0) {
                int lz = 0;
                if (!last && j + 1 <= kLazyMax) {
                    const ST a = (ST)a_s;
                    ST hs = (ST)0;
                    for (int i = 0; i <= j; i++) hs += (ST)hh[i] * (ST)hh[i];
                    const ST d = a - hs;
                    if (d > (ST)1e-2 * a) {
                        lz = 1;
                        set_norm(j + 1, (ST)sqrt(d));
                    }
                }
                lazy_s = lz;
            }
            for (int i = tid; i <= j; i += blockDim.x) hlz[i] = hT[i];
            __syncthreads();
            if (!lazy_s) {
                // the last step, or cancellation: w2 explicitly, its norm partials
                T nacc = (T)0;
                for (int i = tid; i < nf; i += blockDim.x) {
                    T w = x[i];
                    for (int t = 0; t <= j; t++) w -= hT[t] * in.V[(size_t)t * n2 + g0 + i];
                    x[i] = w;
                    Wout[g0 + i] = w;
                    nacc += w * w;
                }
                __syncthreads();
                nacc = block_sum_t<T>(nacc, reinterpret_cast<T*>(red));
                if (last) {
                    if (tid == 0) nbank[s] = (double)nacc;  // for the least squares
                } else {
                    if (tid == 0) nbank2[s] = (double)nacc;
                    if (!grid_sync(ctl, (uint32_t)p, gepoch, cfg.spin, cfg.err)) return;
                    if (tid < 32) {
                        const double a = warp_allsum_ldcg(nbank2, p);
                        if (tid == 0) set_norm(j + 1, (ST)sqrt((ST)a));
                    }
                    __syncthreads();
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// Multiplicative two-level variant (Sec. 3.3, Algorithm "Multiplicative RAP-ILU on GPU").
// The coarse operator S v = R A P v is applied unformed: P v by the backward program on a
// zero interior right-hand side (-U_B^{-1} Z v, v), A by the FP64 SpMV, R and S~^{-1} by the
// forward program (L_B, the W rows, L_S, U_S), all from the factorisation defining R, P.

// scatter-add of the local vector into the original ordering
template <class T>
__device__ __forceinline__ void scatter_add(double* __restrict__ z, const T* x, const int32_t* __restrict__ idx,
                                            int n) {
    for (int l = threadIdx.x; l < n; l += blockDim.x) z[idx[l]] += (double)x[l];
}

// step j, first part: v_j = W_in / ||W_in|| (stopping tests as in the additive inner
// solve), P v_j by the backward program, scattered to a full vector in the original order
template <class T, int RW, bool XS, class V = T>
__global__ void __launch_bounds__(256) k_rap_p_s(SubDev sd, StreamDev<T> S, RingCfg cfg, InnerDev<T> in, int j,
                                                 double* __restrict__ pv, T* xg, const int32_t* done) {
    if (done && *done) return;
    InnerCtl* ctl = in.ctl;
    if (*((volatile int32_t*)&ctl->steps) >= 0 || *((volatile int32_t*)&ctl->zero)) return;
    const int s = blockIdx.x, p = sd.p, n2 = sd.n2;
    const int q0 = sd.qoff[s], ns = sd.qoff[s + 1] - q0, ni = sd.nint[s], nf = ns - ni;
    const double nrm = sqrt(warp_allsum_ldcg(in.part + ((size_t)2 * (kMaxInner + 1)) * p, p));
    if (j == 0) {
        if (s == 0 && threadIdx.x == 0) ctl->beta = nrm;
        if (nrm == 0.0) {
            if (s == 0 && threadIdx.x == 0) ctl->zero = 1;
            return;
        }
    } else {
        if (s == 0 && threadIdx.x == 0) ctl->H[(j - 1) * (kMaxInner + 1) + j] = nrm;
        if (nrm <= 1e-14 * ctl->beta) {
            if (s == 0 && threadIdx.x == 0) ctl->steps = j;
            return;
        }
    }
    const Smem sm = smem_parts(cfg.nst, S.chunk);
    ring_start(S, s, sm, cfg.nst);
    T* x = xvec<T, XS>(sm, xg, q0);
    const T inv = (T)(1.0 / nrm);
    const T* __restrict__ Win = (j & 1) ? in.W1 : in.W0;
    const int g0 = sd.if_ptr[s];
    for (int l = threadIdx.x; l < ni; l += blockDim.x) x[l] = (T)0;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        const T v = Win[g0 + i] * inv;
        in.V[(size_t)j * n2 + g0 + i] = v;
        x[ni + i] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x < S.nt + 32) ring_run<T, RW, V>(S, s, sm, cfg, x);
    __syncthreads();
    scatter(pv, x, sd.q_orig + q0, ns);
}

// step j, second part: w = S~^{-1} R (A P v_j) by the forward program on the gathered
// product, stored for the Gram-Schmidt passes, and the first dots V_i . w
template <class T, int RW, bool XS, class V = T>
__global__ void __launch_bounds__(256) k_rap_r_s(SubDev sd, StreamDev<T> S, RingCfg cfg, InnerDev<T> in, int j,
                                                 const double* __restrict__ apv, T* xg, const int32_t* done) {
    __shared__ double red[32 * 8];
    if (done && *done) return;
    const InnerCtl* ctl = in.ctl;
    if (*((volatile const int32_t*)&ctl->steps) >= 0 || *((volatile const int32_t*)&ctl->zero)) return;
    const int s = blockIdx.x, p = sd.p, n2 = sd.n2;
    const int q0 = sd.qoff[s], ns = sd.qoff[s + 1] - q0, ni = sd.nint[s], nf = ns - ni;
    const Smem sm = smem_parts(cfg.nst, S.chunk);
    ring_start(S, s, sm, cfg.nst);
    T* x = xvec<T, XS>(sm, xg, q0);
    gather(x, apv, sd.q_orig + q0, ns);
    __syncthreads();
    if ((int)threadIdx.x < S.nt + 32) ring_run<T, RW, V>(S, s, sm, cfg, x);
    __syncthreads();
    T* __restrict__ Wout = (j & 1) ? in.W0 : in.W1;
    const int g0 = sd.if_ptr[s];
    for (int i = threadIdx.x; i < nf; i += blockDim.x) Wout[g0 + i] = x[ni + i];
    for (int i0 = 0; i0 <= j; i0 += 8) {
        T acc[8];
#pragma unroll
        for (int u = 0; u < 8; u++) acc[u] = (T)0;
        for (int i = threadIdx.x; i < nf; i += blockDim.x) {
            const T w = x[ni + i];
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (i0 + u <= j) acc[u] += in.V[(size_t)(i0 + u) * n2 + g0 + i] * w;
        }
        block_sum_nt<T, 8>(acc, reinterpret_cast<T*>(red));
        if (threadIdx.x == 0)
            for (int u = 0; u < 8 && i0 + u <= j; u++) in.part[((size_t)(i0 + u)) * p + s] = (double)acc[u];
    }
}

// last part: y = V t (least squares of the coarse GMRES), z = x^ + P y
template <class T, int RW, bool XS, class V = T>
__global__ void __launch_bounds__(256) k_rap_fin_s(SubDev sd, StreamDev<T> S, RingCfg cfg, InnerDev<T> in,
                                                   double* __restrict__ z, T* xg, const int32_t* done) {
    __shared__ double tt[kMaxInner];
    if (done && *done) return;
    const int s = blockIdx.x;
    const int q0 = sd.qoff[s], ns = sd.qoff[s + 1] - q0, ni = sd.nint[s], nf = ns - ni;
    const Smem sm = smem_parts(cfg.nst, S.chunk);
    ring_start(S, s, sm, cfg.nst);
    const int steps = inner_lsq<T>(in.ctl, in.part, sd.p, in.k, tt);
    T* x = xvec<T, XS>(sm, xg, q0);
    const int g0 = sd.if_ptr[s];
    for (int l = threadIdx.x; l < ni; l += blockDim.x) x[l] = (T)0;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        T y = (T)0;
        for (int u = 0; u < steps; u++) y += (T)tt[u] * in.V[(size_t)u * sd.n2 + g0 + i];
        x[ni + i] = y;
    }
    __syncthreads();
    if ((int)threadIdx.x < S.nt + 32) ring_run<T, RW, V>(S, s, sm, cfg, x);
    __syncthreads();
    scatter_add(z, x, sd.q_orig + q0, ns);
}

template <class T, int RW, bool XS, class V = T>
__global__ void __launch_bounds__(256) k_bwd_s(SubDev sd, StreamDev<T> S, RingCfg cfg, InnerDev<T> in,
                                               const double* __restrict__ r, const T* __restrict__ fq, int ef,
                                               double* __restrict__ z, T* xg, const int32_t* done) {
    __shared__ double tt[kMaxInner];
    if (done && *done) return;
    const int s = sub_of_cta(S);
    const int q0 = sd.qoff[s], ns = sd.qoff[s + 1] - q0, ni = sd.nint[s], nf = ns - ni;
    const Smem sm = smem_parts(cfg.nst, S.chunk);
    ring_start(S, s, sm, cfg.nst);
    const int steps = (sd.n2 > 0) ? inner_lsq<T>(in.ctl, in.part, sd.p, in.k, tt) : 0;
    T* x = xvec<T, XS>(sm, xg, q0);
    if (ef)
        gather(x, r, sd.q_orig + q0, ni);
    else
        copy_in(x, fq + q0, ni);
    const int g0 = sd.if_ptr[s];
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        T y = (T)0;
        for (int u = 0; u < steps; u++) y += (T)tt[u] * in.V[(size_t)u * sd.n2 + g0 + i];
        x[ni + i] = y;
    }
    __syncthreads();
    if ((int)threadIdx.x < S.nt + 32) ring_run<T, RW, V>(S, s, sm, cfg, x);
    __syncthreads();
    scatter(z, x, sd.q_orig + q0, ns);
}

// standalone start of the inner solve: c = S~^{-1} gp
template <class T, int RW, bool XS, class V = T>
__global__ void __launch_bounds__(256) k_inner_start_s(SubDev sd, StreamDev<T> S, RingCfg cfg, InnerDev<T> in,
                                                       const double* __restrict__ gp, T* xg) {
    __shared__ double red[32];
    const int s = blockIdx.x;
    const int q0 = sd.qoff[s], ns = sd.qoff[s + 1] - q0, ni = sd.nint[s], nf = ns - ni;
    const Smem sm = smem_parts(cfg.nst, S.chunk);
    ring_start(S, s, sm, cfg.nst);
    T* x = xvec<T, XS>(sm, xg + ni, q0);
    const int g0 = sd.if_ptr[s];
    for (int i = threadIdx.x; i < nf; i += blockDim.x) x[i] = (T)gp[g0 + i];
    __syncthreads();
    if ((int)threadIdx.x < S.nt + 32) ring_run<T, RW, V>(S, s, sm, cfg, x);
    __syncthreads();
    T acc = (T)0;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        const T c = x[i];
        in.W0[g0 + i] = c;
        acc += c * c;
    }
    acc = block_sum_t<T>(acc, reinterpret_cast<T*>(red));
    if (threadIdx.x == 0) {
        in.part[((size_t)2 * (kMaxInner + 1)) * sd.p + s] = (double)acc;
        if (s == 0) {
            in.ctl->steps = -1;
            in.ctl->zero = 0;
            in.ctl->gbar_count = 0;
            in.ctl->gbar_abort = 0;
        }
    }
}

// ---------------------------------------------------------------------------------------
// value packing of a stream: blob[voff[e]] = (T) vals[vsrc[e]]; blob[doff[d]] = 1 / vals[dsrc[d]]
// a factor value in the record's storage type (bfloat16: nearest, ties to even, straight
// from the double)
template <class V>
__device__ __forceinline__ V to_store(double v) {
    return (V)v;
}
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(double v) {
    return __double2bfloat16(v);
}

template <class T, class V = T>
__global__ void k_pack_stream(int64_t nv, int64_t nd, const int64_t* __restrict__ voff, const int32_t* __restrict__ vsrc,
                              const int64_t* __restrict__ doff, const int32_t* __restrict__ dsrc,
                              const double* __restrict__ vals, uint8_t* blob) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = tid; e < nv; e += stride) *reinterpret_cast<V*>(blob + voff[e]) = to_store<V>(vals[vsrc[e]]);
    for (int64_t d = tid; d < nd; d += stride) {
        const int32_t src = dsrc[d];
        *reinterpret_cast<T*>(blob + doff[d]) = (src >= 0) ? (T)(1.0 / vals[src]) : (T)1;
    }
}

// ---------------------------------------------------------------------------------------
// launchers

template <class T>
static StreamDev<T> sdev(const Handle& h, int id) {
    StreamDev<T> d;
    d.blob = h.sb[id].blob;
    d.ch0 = h.sb[id].ch0;
    d.order = h.sb[id].order;
    d.chunk = h.sb[id].chunk;
    d.nt = h.sb[id].nt;
    return d;
}

// full[nst] and empty[nst] mbarriers fill the 128-byte barrier block
constexpr int kMaxStages = 8;

static RingCfg rcfg(const Handle& h) {
    RingCfg c;
    c.nst = h.nst < kMaxStages ? h.nst : kMaxStages;
    c.smem_len = h.smem_len_stream;
    c.spin = h.o.spin_limit ? h.o.spin_limit : (1ull << 22);
    c.err = h.d_err;
    return c;
}

// Dynamic shared memory of a stream kernel: barriers, ring and, when every subdomain's
// working vector fits, the vector. Otherwise the vector lives in global memory and the
// shared memory not requested stays L1 cache, which then holds the vector's recent levels.
static size_t stream_smem(const Handle& h, size_t elt) {
    const bool xs = h.max_ns + 1 <= h.smem_len_stream;
    return 128 + (size_t)h.nst * h.chunk + (xs ? (size_t)h.smem_len_stream * elt : 0);
}

// The dynamic shared-memory limit is per kernel and process-wide: it is raised to the
// device maximum once (never to a handle's own size, which would shrink it under
// handles created earlier with larger subdomains).
template <class K>
static cudaError_t raise_smem_limit(K kernel) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

template <class T, int RW, bool XS, class V = T>
static cudaError_t configure_stream_t() {
    cudaError_t e = raise_smem_limit(k_bj_s<T, RW, XS, V>);
    if (e == cudaSuccess) e = raise_smem_limit(k_fwd_s<T, RW, XS, V>);
    if (e == cudaSuccess) e = raise_smem_limit(k_inner_a_s<T, RW, XS, V>);
    if (e == cudaSuccess) e = raise_smem_limit(k_bwd_s<T, RW, XS, V>);
    if (e == cudaSuccess) e = raise_smem_limit(k_inner_start_s<T, RW, XS, V>);
    if (e == cudaSuccess) e = raise_smem_limit(k_inner_coop<T, RW, XS, V>);
    if (e == cudaSuccess) e = raise_smem_limit(k_rap_p_s<T, RW, XS, V>);
    if (e == cudaSuccess) e = raise_smem_limit(k_rap_r_s<T, RW, XS, V>);
    if (e == cudaSuccess) e = raise_smem_limit(k_rap_fin_s<T, RW, XS, V>);
    return e;
}

template <class T>
cudaError_t configure_stream(const Handle& h, size_t bytes) {
    (void)h;
    (void)bytes;
    cudaError_t e = configure_stream_t<T, 4, true>();
    if (e == cudaSuccess) e = configure_stream_t<T, 16, true>();
    if (e == cudaSuccess) e = configure_stream_t<T, 4, false>();
    if (e == cudaSuccess) e = configure_stream_t<T, 16, false>();
    if constexpr (sizeof(T) == 4) {  // bfloat16 value storage
        if (e == cudaSuccess) e = configure_stream_t<T, 4, true, __nv_bfloat16>();
        if (e == cudaSuccess) e = configure_stream_t<T, 16, true, __nv_bfloat16>();
        if (e == cudaSuccess) e = configure_stream_t<T, 4, false, __nv_bfloat16>();
        if (e == cudaSuccess) e = configure_stream_t<T, 16, false, __nv_bfloat16>();
    }
    return e;
}

template <class T>
cudaError_t launch_pack_stream(const StreamHost& sh, const int64_t* voff, const int32_t* vsrc, const int64_t* doff,
                               const int32_t* dsrc, const double* vals, uint8_t* blob, cudaStream_t st) {
    const int64_t nv = (int64_t)sh.voff.size(), nd = (int64_t)sh.doff.size();
    if (nv == 0 && nd == 0) return cudaSuccess;
    if (sizeof(T) == 4 && sh.val_bytes == 2)  // bfloat16 values, float pivot inverses
        k_pack_stream<T, __nv_bfloat16><<<1024, 256, 0, st>>>(nv, nd, voff, vsrc, doff, dsrc, vals, blob);
    else
        k_pack_stream<T><<<1024, 256, 0, st>>>(nv, nd, voff, vsrc, doff, dsrc, vals, blob);
    return cudaGetLastError();
}

#define ILU2L_RW_DISPATCH(h, id, CALL)       \
    if ((h).sb[id].rw == 4) {                \
        constexpr int RW = 4;                \
        CALL;                                \
    } else {                                 \
        constexpr int RW = 16;               \
        CALL;                                \
    }
#define ILU2L_XS_DISPATCH(h, id, CALL)       \
    if ((h).max_ns + 1 <= (h).smem_len_stream) { \
        constexpr bool XS = true;            \
        ILU2L_RW_DISPATCH(h, id, CALL)       \
    } else {                                 \
        constexpr bool XS = false;           \
        ILU2L_RW_DISPATCH(h, id, CALL)       \
    }
// value storage of the records (V): bfloat16 when a float handle stores its factors so
#define ILU2L_V_DISPATCH(h, STMT)                  \
    if constexpr (sizeof(T) == 4) {                \
        if ((h).prec == ILU_PREC_BF16_STORE) {     \
            using V = __nv_bfloat16;               \
            STMT                                   \
        } else {                                   \
            using V = T;                           \
            STMT                                   \
        }                                          \
    } else {                                       \
        using V = T;                               \
        STMT                                       \
    }
#define ILU2L_IDX_DISPATCH(h, id, CALL) ILU2L_V_DISPATCH(h, ILU2L_XS_DISPATCH(h, id, CALL))
#define ILU2L_VRW_DISPATCH(h, id, CALL) ILU2L_V_DISPATCH(h, ILU2L_RW_DISPATCH(h, id, CALL))

template <class T>
cudaError_t launch_bj_s(const Handle& h, const double* r, double* z, const int32_t* done, cudaStream_t st) {
    ILU2L_IDX_DISPATCH(h, PR_BJ, (k_bj_s<T, RW, XS, V><<<h.p, 256, stream_smem(h, sizeof(T)), st>>>(
                              h.sub(), sdev<T>(h, PR_BJ), rcfg(h), r, z, (T*)h.d_xg, done)));
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_fwd_s(const Handle& h, const double* r, const int32_t* done, cudaStream_t st) {
    ILU2L_IDX_DISPATCH(h, PR_FWDS, (k_fwd_s<T, RW, XS, V><<<h.p, 256, stream_smem(h, sizeof(T)), st>>>(
                              h.sub(), sdev<T>(h, PR_FWDS), rcfg(h), h.innerdev<T>(), r, (T*)h.d_fq, (T*)h.d_xg,
                              done)));
    return cudaGetLastError();
}

// Whether the single-launch inner solve fits: every subdomain's CTA resident at once.
template <class T>
cudaError_t inner_coop_fits(const Handle& h, bool* fits) {
    *fits = false;
    int dev = 0, coop = 0, nb = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e != cudaSuccess || !coop) return e;
    ILU2L_IDX_DISPATCH(h, PR_S, (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                     &nb, k_inner_coop<T, RW, XS, V>, 256, stream_smem(h, sizeof(T)))));
    if (e == cudaSuccess) *fits = (int64_t)nb * h.sm_count >= h.p;
    return e;
}

template <class T>
static cudaError_t launch_inner_coop(const Handle& h, const int32_t* done, cudaStream_t st) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)h.p);
    lc.blockDim = dim3(256);
    lc.dynamicSmemBytes = stream_smem(h, sizeof(T));
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    cudaError_t e = cudaSuccess;
    ILU2L_IDX_DISPATCH(h, PR_S, (e = cudaLaunchKernelEx(&lc, k_inner_coop<T, RW, XS, V>, h.sub(), sdev<T>(h, PR_S),
                                                         rcfg(h), h.innerdev<T>(), (T*)h.d_xg, done)));
    return e;
}

template <class T>
cudaError_t launch_inner_s(const Handle& h, const int32_t* done, cudaStream_t st) {
    if (h.n2 == 0) return cudaSuccess;
    if (h.inner_coop) return launch_inner_coop<T>(h, done, st);
    const int gb = std::max(1, std::min(h.sm_count * 4, (h.n2 + 255) / 256));
    for (int j = 0; j < h.inner_k; j++) {
        k_coff<T><<<gb, 256, 0, st>>>(h.sub(), h.innerdev<T>(), j, (T*)h.d_tbuf, done);
        ILU2L_IDX_DISPATCH(h, PR_S, (k_inner_a_s<T, RW, XS, V><<<h.p, 256, stream_smem(h, sizeof(T)), st>>>(
                                  h.sub(), sdev<T>(h, PR_S), rcfg(h), h.innerdev<T>(), j, (const T*)h.d_tbuf,
                                  (T*)h.d_xg, done)));
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_inner_bc<T>(h, j, 0, done, st);
        if (e == cudaSuccess) e = launch_inner_bc<T>(h, j, 1, done, st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_bwd_s(const Handle& h, const double* r, double* z, const int32_t* done, cudaStream_t st) {
    ILU2L_IDX_DISPATCH(h, PR_BWD, (k_bwd_s<T, RW, XS, V><<<h.p, 256, stream_smem(h, sizeof(T)), st>>>(
                              h.sub(), sdev<T>(h, PR_BWD), rcfg(h), h.innerdev<T>(), r, (const T*)h.d_fq,
                              h.form == ILU_FORM_EF ? 1 : 0, z, (T*)h.d_xg, done)));
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_inner_start_s(const Handle& h, const double* gp, cudaStream_t st) {
    ILU2L_IDX_DISPATCH(h, PR_S, (k_inner_start_s<T, RW, XS, V><<<h.p, 256, stream_smem(h, sizeof(T)), st>>>(
                              h.sub(), sdev<T>(h, PR_S), rcfg(h), h.innerdev<T>(), gp, (T*)h.d_xg)));
    return cudaGetLastError();
}

// The inner Schur solve (streamed local Schur programs, working vectors in shared memory)
// on a caller-provided Krylov workspace `in` and product buffer `tbuf`.
template <class T>
cudaError_t launch_inner_io_ws(const Handle& h, const InnerDev<T>& in, T* tbuf, const double* gp, double* y,
                               cudaStream_t st) {
    if (h.n2 == 0) return cudaSuccess;
    constexpr bool XS = true;
    T* xdummy = tbuf;  // unused by the shared-memory kernels
    ILU2L_VRW_DISPATCH(h, PR_S, (k_inner_start_s<T, RW, XS, V><<<h.p, 256, stream_smem(h, sizeof(T)), st>>>(
                                   h.sub(), sdev<T>(h, PR_S), rcfg(h), in, gp, xdummy)));
    cudaError_t e = cudaGetLastError();
    const int gb = std::max(1, std::min(h.sm_count * 4, (h.n2 + 255) / 256));
    for (int j = 0; j < h.inner_k && e == cudaSuccess; j++) {
        k_coff<T><<<gb, 256, 0, st>>>(h.sub(), in, j, tbuf, nullptr);
        ILU2L_VRW_DISPATCH(h, PR_S, (k_inner_a_s<T, RW, XS, V><<<h.p, 256, stream_smem(h, sizeof(T)), st>>>(
                                       h.sub(), sdev<T>(h, PR_S), rcfg(h), in, j, tbuf, xdummy, nullptr)));
        e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_inner_bc_ws<T>(h, in, j, 0, st);
        if (e == cudaSuccess) e = launch_inner_bc_ws<T>(h, in, j, 1, st);
    }
    if (e == cudaSuccess) e = launch_inner_finish_ws<T>(h, in, y, st);
    return e;
}

template <class T>
cudaError_t launch_rap_inner_s(const Handle& h, const int32_t* done, cudaStream_t st) {
    if (h.n2 == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < h.inner_k && e == cudaSuccess; j++) {
        ILU2L_IDX_DISPATCH(h, PR_BWD, (k_rap_p_s<T, RW, XS, V><<<h.p, 256, stream_smem(h, sizeof(T)), st>>>(
                                          h.sub(), sdev<T>(h, PR_BWD), rcfg(h), h.innerdev<T>(), j, h.rap_pv,
                                          (T*)h.d_xg, done)));
        e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_rap_resid(h, nullptr, h.rap_pv, h.rap_apv, done, st);
        if (e == cudaSuccess) {
            ILU2L_IDX_DISPATCH(h, PR_FWDS, (k_rap_r_s<T, RW, XS, V><<<h.p, 256, stream_smem(h, sizeof(T)), st>>>(
                                               h.sub(), sdev<T>(h, PR_FWDS), rcfg(h), h.innerdev<T>(), j,
                                               h.rap_apv, (T*)h.d_xg, done)));
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = launch_inner_bc<T>(h, j, 0, done, st);
        if (e == cudaSuccess) e = launch_inner_bc<T>(h, j, 1, done, st);
    }
    return e;
}

template <class T>
cudaError_t launch_rap_fin_s(const Handle& h, double* z, const int32_t* done, cudaStream_t st) {
    if (h.n2 == 0) return cudaSuccess;
    ILU2L_IDX_DISPATCH(h, PR_BWD, (k_rap_fin_s<T, RW, XS, V><<<h.p, 256, stream_smem(h, sizeof(T)), st>>>(
                                      h.sub(), sdev<T>(h, PR_BWD), rcfg(h), h.innerdev<T>(), z, (T*)h.d_xg,
                                      done)));
    return cudaGetLastError();
}

#define ILU2L_SINST(T)                                                                                      \
    template cudaError_t launch_inner_io_ws<T>(const Handle&, const InnerDev<T>&, T*, const double*,         \
                                               double*, cudaStream_t);                                       \
    template cudaError_t configure_stream<T>(const Handle&, size_t);                                       \
    template cudaError_t launch_pack_stream<T>(const StreamHost&, const int64_t*, const int32_t*,          \
                                               const int64_t*, const int32_t*, const double*, uint8_t*,    \
                                               cudaStream_t);                                              \
    template cudaError_t launch_bj_s<T>(const Handle&, const double*, double*, const int32_t*, cudaStream_t); \
    template cudaError_t launch_fwd_s<T>(const Handle&, const double*, const int32_t*, cudaStream_t);      \
    template cudaError_t launch_inner_s<T>(const Handle&, const int32_t*, cudaStream_t);                   \
    template cudaError_t launch_bwd_s<T>(const Handle&, const double*, double*, const int32_t*,            \
                                         cudaStream_t);                                                    \
    template cudaError_t launch_inner_start_s<T>(const Handle&, const double*, cudaStream_t);             \
    template cudaError_t inner_coop_fits<T>(const Handle&, bool*);                                       \
    template cudaError_t launch_rap_inner_s<T>(const Handle&, const int32_t*, cudaStream_t);             \
    template cudaError_t launch_rap_fin_s<T>(const Handle&, double*, const int32_t*, cudaStream_t);
ILU2L_SINST(float)
ILU2L_SINST(double)

}  // namespace ilu2l
