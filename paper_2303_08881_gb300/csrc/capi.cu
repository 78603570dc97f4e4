// capi.cu -- the C ABI of ilu2l (include/ilu2l.h): handle lifecycle, device uploads, the
// device factorisation, apply dispatch and the FGMRES driver (one CUDA graph per cycle,
// one host read of the device control block per cycle).
#include <algorithm>
#include <vector>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>

#include "handle.h"

namespace ilu2l {

const char* kProfNames[PC_COUNT] = {"apply_fwd",  "apply_inner", "apply_bwd", "apply_bj",
                                    "fg_spmv_dot", "fg_cgs",      "fg_norm",   "fg_next",
                                    "fg_update",  "fg_resid",    "fg_scale0"};

namespace {

#define CK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return map_err(e_); \
    } while (0)

ilu_status map_err(cudaError_t e) {
    if (e == cudaSuccess) return ILU_OK;
    if (e == cudaErrorMemoryAllocation) return ILU_ERR_OOM;
    return ILU_ERR_CUDA;
}

// ---- process-wide resources shared by the handles (guarded: handles live on many threads)
static std::mutex g_res_mutex;

// The default memory pool of a device keeps freed memory for reuse instead of returning it:
// handles come and go without mapping or unmapping device memory.
static cudaError_t pool_keep(int dev) {
    static bool done[64] = {};
    std::lock_guard<std::mutex> lk(g_res_mutex);
    if (dev < 0 || dev >= 64 || done[dev]) return cudaSuccess;
    cudaMemPool_t pool;
    cudaError_t e = cudaDeviceGetDefaultMemPool(&pool, dev);
    uint64_t keep = UINT64_MAX;
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

// Kernel attributes (the dynamic shared-memory limit, raised to the device maximum) are
// set once per device and kernel family.
template <class F>
static cudaError_t once_per_device(int dev, int family, F fn) {
    static bool done[64][8] = {};
    std::lock_guard<std::mutex> lk(g_res_mutex);
    if (dev < 0 || dev >= 64 || family < 0 || family >= 8) return fn();
    if (done[dev][family]) return cudaSuccess;
    cudaError_t e = fn();
    if (e == cudaSuccess) done[dev][family] = true;
    return e;
}

// Pinned host control blocks of the FGMRES driver, recycled (freeing pinned memory would
// synchronise the device).
static std::vector<FgCtl*> g_ctl_free;
static cudaError_t ctl_take(FgCtl** out) {
    {
        std::lock_guard<std::mutex> lk(g_res_mutex);
        if (!g_ctl_free.empty()) {
            *out = g_ctl_free.back();
            g_ctl_free.pop_back();
            return cudaSuccess;
        }
    }
    return cudaMallocHost(out, sizeof(FgCtl));
}
static void ctl_give(FgCtl* c) {
    std::lock_guard<std::mutex> lk(g_res_mutex);
    g_ctl_free.push_back(c);
}

template <class T, class A>
cudaError_t upload(Handle& h, T** dst, const std::vector<T, A>& src) {
    cudaError_t e = cudaSuccess;
    *dst = h.alloc<T>(src.size(), &e);
    if (!*dst) return e;
    if (!src.empty()) e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, h.st);
    return e;
}

template <class T>
ilu_status upload_prog(Handle& h, int id) {
    ProgHost& P = h.prog[id];
    ProgBufs& B = h.pb[id];
    if (P.sub_lvl.size() < (size_t)h.p + 1) P.sub_lvl.resize(h.p + 1, P.sub_lvl.empty() ? 0 : P.sub_lvl.back());
    CK(upload(h, &B.sub_lvl, P.sub_lvl));
    CK(upload(h, &B.lvl_ptr, P.lvl_ptr));
    CK(upload(h, &B.prow, P.prow));
    CK(upload(h, &B.pptr, P.pptr));
    CK(upload(h, &B.pcol, P.pcol));
    CK(upload(h, &B.psrc, P.psrc));
    CK(upload(h, &B.pdsrc, P.pdsrc));
    cudaError_t e = cudaSuccess;
    B.pval = h.alloc<T>(P.pcol.size(), &e);
    if (!B.pval) return map_err(e);
    B.pdinv = h.alloc<T>(P.prow.size(), &e);
    if (!B.pdinv) return map_err(e);
    CK(launch_pack<T>(P, B.psrc, B.pdsrc, h.d_vals, (T*)B.pval, (T*)B.pdinv, h.st));
    return ILU_OK;
}

// Device copy of the streamed program id built on the host (h.sh[id]): the chunks, the
// per-subdomain chunk offsets and launch order, and the values and pivot inverses packed
// into the chunks from the FP64 factors on the device. Replaces (and frees) an earlier copy;
// the host chunks are freed once packed.
template <class T>
ilu_status upload_stream(Handle& h, int id) {
    StreamHost& S = h.sh[id];
    if (S.ch0.empty()) return ILU_OK;
    StreamBufs& B = h.sb[id];
    for (void* q : {(void*)B.blob, (void*)B.ch0, (void*)B.order})
        if (q) h.release(q);
    B = StreamBufs{};
    CK(upload(h, &B.blob, S.blob));
    CK(upload(h, &B.ch0, S.ch0));
    CK(upload(h, &B.order, S.order));
    B.chunk = S.chunk;
    B.nt = S.nt;
    B.rw = S.rw;
    int64_t *dvoff = nullptr, *ddoff = nullptr;
    int32_t *dvsrc = nullptr, *ddsrc = nullptr;
    CK(upload(h, &dvoff, S.voff));
    CK(upload(h, &dvsrc, S.vsrc));
    CK(upload(h, &ddoff, S.doff));
    CK(upload(h, &ddsrc, S.dsrc));
    CK(launch_pack_stream<T>(S, dvoff, dvsrc, ddoff, ddsrc, h.d_vals, B.blob, h.st));
    CK(cudaStreamSynchronize(h.st));
    for (void* q : {(void*)dvoff, (void*)dvsrc, (void*)ddoff, (void*)ddsrc}) h.release(q);
    decltype(S.blob)().swap(S.blob);
    decltype(S.voff)().swap(S.voff);
    decltype(S.doff)().swap(S.doff);
    decltype(S.vsrc)().swap(S.vsrc);
    decltype(S.dsrc)().swap(S.dsrc);
    return ILU_OK;
}

template <class T>
ilu_status device_setup_t(Handle& h) {
    cudaError_t e = cudaSuccess;
    const int n = h.n;
    // shared-memory working vector
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h.device));
    const int64_t cap = std::max<int64_t>(0, (int64_t)optin - 20 * 1024) / (int64_t)sizeof(T);
    h.smem_len = (int32_t)std::min<int64_t>(h.max_ns, cap);
    CK(once_per_device(h.device, sizeof(T) == 4 ? 0 : 1, [&] { return configure_apply<T>((size_t)h.smem_len * sizeof(T)); }));
    if (h.stream_path) {  // the streamed kernels keep the ring in shared memory too
        const int64_t cap_s = ((int64_t)optin - 20 * 1024 - 128 - (int64_t)h.nst * h.chunk) / (int64_t)sizeof(T);
        h.smem_len_stream = (int32_t)std::max<int64_t>(0, std::min<int64_t>((int64_t)h.max_ns + 1, cap_s));
    }
    // a global working vector whenever some kernel family cannot hold every subdomain in
    // shared memory (the generic kernels need max_ns elements, the streamed max_ns + 1)
    const bool need_xg = h.max_ns > h.smem_len || (h.stream_path && h.max_ns + 1 > h.smem_len_stream);
    h.d_xg = h.alloc<T>(need_xg ? (size_t)n : 1, &e);
    if (!h.d_xg) return map_err(e);
    h.d_fq = h.alloc<T>((size_t)std::max(n, 1), &e);
    if (!h.d_fq) return map_err(e);
    // C_off in the PC type
    std::vector<T> cv(h.coff_v.begin(), h.coff_v.end());
    CK(upload(h, &h.d_coff_rp, h.coff_rp));
    CK(upload(h, &h.d_coff_ci, h.coff_ci));
    T* dcv = nullptr;
    CK(upload(h, &dcv, cv));
    h.d_coff_v = dcv;
    // inner GMRES workspace
    h.d_iV = h.alloc<T>((size_t)(h.inner_k + 1) * std::max(h.n2, 1), &e);
    h.d_iW0 = h.alloc<T>((size_t)std::max(h.n2, 1), &e);
    h.d_iW1 = h.alloc<T>((size_t)std::max(h.n2, 1), &e);
    if (!h.d_iV || !h.d_iW0 || !h.d_iW1) return map_err(e);
    if (h.variant == ILU_VARIANT_RAP) {
        h.rap_res = h.alloc<double>((size_t)std::max(n, 1), &e);
        h.rap_pv = h.alloc<double>((size_t)std::max(n, 1), &e);
        h.rap_apv = h.alloc<double>((size_t)std::max(n, 1), &e);
        if (!h.rap_res || !h.rap_pv || !h.rap_apv) return map_err(e);
    }
    cv.clear();
    cv.shrink_to_fit();
    if (h.stream_path) {
        CK(once_per_device(h.device, sizeof(T) == 4 ? 2 : 3, [&] {
            return configure_stream<T>(h, 128 + (size_t)h.nst * h.chunk + (size_t)h.smem_len_stream * sizeof(T));
        }));
        if (h.variant == ILU_VARIANT_SCHUR && h.n2 > 0 && h.o.inner_launch == 0)
            CK(inner_coop_fits<T>(h, &h.inner_coop));
        h.d_tbuf = h.alloc<T>((size_t)std::max(h.n2, 1), &e);
        if (!h.d_tbuf) return map_err(e);
        for (int id = 0; id < PR_COUNT; id++) {
            ilu_status us = upload_stream<T>(h, id);
            if (us != ILU_OK) return us;
        }
    }
    if (h.variant == ILU_VARIANT_BJ) {
        if (h.stream_path) return ILU_OK;
        ilu_status s = upload_prog<T>(h, PR_BJ);
        if (s != ILU_OK) return s;
    } else if (!h.stream_path) {  // the streamed path reads its own chunks only
        for (int id : {PR_FWD, PR_S, PR_BWD}) {
            ilu_status s = upload_prog<T>(h, id);
            if (s != ILU_OK) return s;
        }
    }
    return ILU_OK;
}

ilu_status device_setup(Handle& h) {
    cudaError_t e = cudaSuccess;
    CK(cudaGetDevice(&h.device));
    CK(pool_keep(h.device));
    CK(cudaDeviceGetAttribute(&h.sm_count, cudaDevAttrMultiProcessorCount, h.device));
    const int n = h.n, p = h.p;
    CK(upload(h, &h.d_qoff, h.qoff));
    CK(upload(h, &h.d_nint, h.nint));
    CK(upload(h, &h.d_if_ptr, h.if_ptr));
    CK(upload(h, &h.d_q_orig, h.q_orig));
    if (!h.d_q_rp) CK(upload(h, &h.d_q_rp, h.q_rp));  // the device ILUT may have uploaded both
    if (!h.d_q_ci) CK(upload(h, &h.d_q_ci, h.q_ci));
    CK(upload(h, &h.d_q_dpos, h.q_dpos));
    // value array [F1 | F2 | A_local]
    h.d_vals = h.alloc<double>((size_t)h.nvals, &e);
    if (!h.d_vals) return map_err(e);
    if (!h.q_v.empty())
        CK(cudaMemcpyAsync(h.d_vals + h.a_base, h.q_v.data(), h.q_v.size() * sizeof(double),
                           cudaMemcpyHostToDevice, h.st));
    if (h.d_f1_stage) {  // ILUT values factorised on the device
        if (h.f1.nnz)
            CK(cudaMemcpyAsync(h.d_vals + h.f1.base, h.d_f1_stage, (size_t)h.f1.nnz * sizeof(double),
                               cudaMemcpyDeviceToDevice, h.st));
        h.release(h.d_f1_stage);
        h.d_f1_stage = nullptr;
    } else if (!h.f1_device && !h.f1_host_vals.empty()) {
        CK(cudaMemcpyAsync(h.d_vals + h.f1.base, h.f1_host_vals.data(),
                           h.f1_host_vals.size() * sizeof(double), cudaMemcpyHostToDevice, h.st));
    }
    h.d_err = h.alloc<int32_t>(1, &e);
    h.d_npert = h.alloc<int32_t>(1, &e);
    if (!h.d_err || !h.d_npert) return map_err(e);
    CK(cudaMemsetAsync(h.d_err, 0, sizeof(int32_t), h.st));
    CK(cudaMemsetAsync(h.d_npert, 0, sizeof(int32_t), h.st));
    // numeric factorisation schedule
    CK(upload(h, &h.d_num_sub, h.numprog.sub_lvl));
    CK(upload(h, &h.d_num_lvl, h.numprog.lvl_ptr));
    CK(upload(h, &h.d_num_row, h.numprog.prow));
    if (h.f1_device) CK(launch_ilu_numeric(h, h.d_vals + h.f1.base, h.kB == ILU_FACT_MILU0 ? 1 : 0, h.st));
    if (!h.f2_alias)
        CK(launch_ilu_numeric(h, h.d_vals + h.f2.base,
                              h.kS == ILU_FACT_MILU0 ? 1 : (h.kS == ILU_FACT_PMILU0 ? 2 : 0), h.st));
    int32_t herr = 0, hpert = 0;
    CK(cudaMemcpyAsync(&herr, h.d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, h.st));
    CK(cudaMemcpyAsync(&hpert, h.d_npert, sizeof(int32_t), cudaMemcpyDeviceToHost, h.st));
    CK(cudaStreamSynchronize(h.st));
    if (herr & 1) return ILU_ERR_ZERO_PIVOT;
    h.npert += hpert;
    // inner control + partials
    h.d_ipart = h.alloc<double>((size_t)3 * (kMaxInner + 1) * p, &e);
    h.d_ictl = h.alloc<InnerCtl>(1, &e);
    if (!h.d_ipart || !h.d_ictl) return map_err(e);
    CK(cudaMemsetAsync(h.d_ictl, 0, sizeof(InnerCtl), h.st));
    ilu_status s = (h.prec != ILU_PREC_FP64) ? device_setup_t<float>(h) : device_setup_t<double>(h);
    if (s != ILU_OK) return s;
    CK(cudaStreamSynchronize(h.st));
    (void)n;
    return ILU_OK;
}

ilu_status ensure_fgmres(Handle& h, int m) {
    if (h.fg_m >= m && h.fg.V) {
        h.fg.m = m;
        return ILU_OK;
    }
    cudaError_t e = cudaSuccess;
    const size_t n = (size_t)std::max(h.n, 1);
    h.fg_G = h.sm_count * 4;
    h.fg_threads = 256;
    CK(configure_krylov());
    FgDev f{};
    f.ld = (int64_t)((n + 63) / 64 * 64);
    f.V = h.alloc<double>((size_t)(m + 1) * (size_t)f.ld, &e);
    f.Z = h.alloc<double>((size_t)m * (size_t)f.ld, &e);
    f.w = h.alloc<double>((size_t)f.ld, &e);
    h.fg_b = h.alloc<double>((size_t)f.ld, &e);
    h.fg_x = h.alloc<double>((size_t)f.ld, &e);
    if (!h.fg_b || !h.fg_x) return map_err(e);
    f.H = h.alloc<double>((size_t)(m + 1) * m, &e);
    f.cs = h.alloc<double>((size_t)m + 1, &e);
    f.sn = h.alloc<double>((size_t)m + 1, &e);
    f.g = h.alloc<double>((size_t)m + 1, &e);
    f.h2 = h.alloc<double>((size_t)m + 1, &e);
    f.hnext = h.alloc<double>(2, &e);
    f.y = h.alloc<double>((size_t)m + 1, &e);
    const int ng = (h.fg_G + kRedGroup - 1) / kRedGroup;
    f.gpart = h.alloc<double>((size_t)(m + 2) * ng, &e);
    f.gcount = h.alloc<uint32_t>((size_t)ng, &e);
    if (!f.gpart || !f.gcount) return map_err(e);
    CK(cudaMemsetAsync(f.gcount, 0, sizeof(uint32_t) * ng, h.st));
    f.part = h.alloc<double>((size_t)(m + 2) * h.fg_G, &e);
    f.ctl = h.alloc<FgCtl>(1, &e);
    if (!f.V || !f.Z || !f.w || !f.H || !f.cs || !f.sn || !f.g || !f.h2 || !f.hnext || !f.y || !f.part || !f.ctl)
        return map_err(e);
    f.V32 = nullptr;
    f.w32 = nullptr;
    f.Vlo = nullptr;
    f.wlo = nullptr;
    f.upd32 = h.o.gs_precision >= 2 ? 1 : 0;
    if (h.o.gs_precision > 0) {
        f.V32 = h.alloc<float>((size_t)(m + 1) * (size_t)f.ld, &e);
        f.w32 = h.alloc<float>((size_t)f.ld, &e);
        if (!f.V32 || !f.w32) return map_err(e);
    }
    if (h.o.gs_precision == 3) {
        f.Vlo = h.alloc<float>((size_t)(m + 1) * (size_t)f.ld, &e);
        f.wlo = h.alloc<float>((size_t)f.ld, &e);
        if (!f.Vlo || !f.wlo) return map_err(e);
    }
    CK(cudaMemsetAsync(f.ctl, 0, sizeof(FgCtl), h.st));
    f.m = m;
    f.G = h.fg_G;
    h.fg = f;
    h.fg_m = m;
    if (h.cycle_exec) {
        cudaGraphExecDestroy(h.cycle_exec);
        h.cycle_exec = nullptr;
    }
    if (!h.h_ctl) CK(ctl_take(&h.h_ctl));
    return ILU_OK;
}

// Brackets a group of nkern kernels of one class with CUDA events on the launching
// stream when profiling is on (graphs are off then); always counts the launches.
struct Scope {
    Handle& h;
    int cls, nkern;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    bool capturing;
    static cudaEvent_t take(Handle& h) {
        if (h.ev_used == h.ev_pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            h.ev_pool.push_back(e);
        }
        return h.ev_pool[h.ev_used++];
    }
    Scope(Handle& hh, int c, int nk, cudaStream_t s, bool cap) : h(hh), cls(c), nkern(nk), st(s), capturing(cap) {
        if (!capturing) h.kernel_launches += nk;
        if (h.prof && !capturing) {
            a = take(h);
            b = take(h);
            if (a && b) cudaEventRecord(a, st);
        }
    }
    ~Scope() {
        if (a && b) {
            cudaEventRecord(b, st);
            h.prof_recs.push_back({cls, nkern, a, b});
        }
    }
};

// Two-level multiplicative apply (Algorithm "Multiplicative RAP-ILU on GPU"):
// x^ = smoother(r) into z; res = r - A x^; the forward program on res gives R res and
// c = S~^{-1} R res; k GMRES steps on S~^{-1} R A P v = c, each P v, A (P v), R and S~^{-1},
// then the Gram-Schmidt passes; z = x^ + P v.
template <class T>
cudaError_t apply_rap(Handle& h, const double* r, double* z, const int32_t* done, cudaStream_t st, bool cap) {
    cudaError_t e;
    {
        Scope sc(h, PC_APPLY_FWD, h.n2 > 0 ? 3 : 1, st, cap);
        e = launch_bj_s<T>(h, r, z, done, st);
        if (e == cudaSuccess && h.n2 > 0) e = launch_rap_resid(h, r, z, h.rap_res, done, st);
        if (e == cudaSuccess && h.n2 > 0) e = launch_fwd_s<T>(h, h.rap_res, done, st);
    }
    if (e == cudaSuccess && h.n2 > 0) {
        Scope sc(h, PC_INNER, 5 * h.inner_k, st, cap);
        e = launch_rap_inner_s<T>(h, done, st);
    }
    if (e == cudaSuccess && h.n2 > 0) {
        Scope sc(h, PC_APPLY_BWD, 1, st, cap);
        e = launch_rap_fin_s<T>(h, z, done, st);
    }
    return e;
}

template <class T>
cudaError_t apply_t(Handle& h, const double* r, double* z, const int32_t* done, cudaStream_t st, bool cap) {
    const bool fast = h.stream_path;
    if (h.variant == ILU_VARIANT_RAP) return apply_rap<T>(h, r, z, done, st, cap);
    if (h.variant == ILU_VARIANT_BJ) {
        Scope sc(h, PC_BJ, 1, st, cap);
        return fast ? launch_bj_s<T>(h, r, z, done, st) : launch_bj<T>(h, r, z, done, st);
    }
    cudaError_t e;
    {
        Scope sc(h, PC_APPLY_FWD, 1, st, cap);
        e = fast ? launch_fwd_s<T>(h, r, done, st) : launch_schur_fwd<T>(h, r, done, st);
    }
    if (e == cudaSuccess && h.n2 > 0) {
        Scope sc(h, PC_INNER, fast ? (h.inner_coop ? 1 : 4 * h.inner_k) : 3 * h.inner_k, st, cap);
        e = fast ? launch_inner_s<T>(h, done, st) : launch_inner<T>(h, done, st);
    }
    if (e == cudaSuccess) {
        Scope sc(h, PC_APPLY_BWD, 1, st, cap);
        e = fast ? launch_bwd_s<T>(h, r, z, done, st) : launch_schur_bwd<T>(h, r, z, done, st);
    }
    return e;
}

cudaError_t apply_any(Handle& h, const double* r, double* z, const int32_t* done, cudaStream_t st,
                      bool cap = false) {
    return (h.prec != ILU_PREC_FP64) ? apply_t<float>(h, r, z, done, st, cap)
                                     : apply_t<double>(h, r, z, done, st, cap);
}

// The autotuner (ilu_opts.autotune). For each streamed program in turn, the program is
// rebuilt with consumer groups of 32, 64, 96 and 128 threads; each version is timed as the
// mean of five applies (after one untimed apply) with CUDA events on the handle's stream,
// and the fastest is kept (a candidate replaces the current one only when at least 2 %
// faster). The programs of the handle's variant: block Jacobi; forward, local Schur and
// backward; or, for the multiplicative variant, the smoother, forward and backward.
template <class T>
ilu_status autotune_t(Handle& h) {
    std::vector<int> ids;
    for (int id = 0; id < PR_COUNT; id++)
        if (!h.sh[id].ch0.empty()) ids.push_back(id);
    if (ids.empty()) return ILU_OK;
    cudaError_t e = cudaSuccess;
    double* r = h.alloc<double>((size_t)std::max(h.n, 1), &e);
    double* z = h.alloc<double>((size_t)std::max(h.n, 1), &e);
    if (!r || !z) return map_err(e);
    CK(cudaMemsetAsync(r, 0x3F, (size_t)std::max(h.n, 1) * sizeof(double), h.st));  // 0.49...
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    auto timed = [&](double* ms) -> cudaError_t {
        cudaError_t err = apply_any(h, r, z, nullptr, h.st);
        if (err == cudaSuccess) err = cudaEventRecord(e0, h.st);
        for (int i = 0; i < 5 && err == cudaSuccess; i++) err = apply_any(h, r, z, nullptr, h.st);
        if (err == cudaSuccess) err = cudaEventRecord(e1, h.st);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float f = 0.0f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&f, e0, e1);
        *ms = f / 5.0;
        return err;
    };
    const int vb = (h.prec == ILU_PREC_FP64) ? 8 : 4;
    const int valb = (h.prec == ILU_PREC_BF16_STORE) ? 2 : vb;
    ilu_status st = ILU_OK;
    int32_t chosen[PR_COUNT] = {0, 0, 0, 0, 0};
    auto rebuild = [&](int id, int nt) -> bool {
        StreamHost S;
        S.nt = nt;
        if (!build_stream(h.prog[id], h.p, h.idx_bytes, vb, valb, h.chunk, S, h.o.chain_sched) || S.nt != nt)
            return false;
        h.sh[id] = std::move(S);
        st = upload_stream<T>(h, id);
        return st == ILU_OK;
    };
    for (int id : ids) {
        int best = h.sh[id].nt;
        double best_ms = 0.0;
        if ((e = timed(&best_ms)) != cudaSuccess) break;
        for (int c = 0; c < kTuneCands; c++)
            if (kTuneNt[c] == best) h.tune_ms[id][c] = best_ms;
        int built = best;
        for (int c = 0; c < kTuneCands && st == ILU_OK; c++) {
            if (kTuneNt[c] == built || h.tune_ms[id][c] > 0.0) continue;
            if (!rebuild(id, kTuneNt[c])) continue;
            built = kTuneNt[c];
            double ms = 0.0;
            if ((e = timed(&ms)) != cudaSuccess) break;
            h.tune_ms[id][c] = ms;
            if (ms < 0.98 * best_ms) {
                best_ms = ms;
                best = kTuneNt[c];
            }
        }
        if (e != cudaSuccess || st != ILU_OK) break;
        if (built != best && !rebuild(id, best)) break;
        chosen[id] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h.release(r);
    h.release(z);
    if (e != cudaSuccess) return map_err(e);
    if (st != ILU_OK) return st;
    tune_store(h.tune_key_v, chosen);
    h.tune_state = 1;
    return ILU_OK;
}

#define ILU2L_SCOPED(cls, nk, call)              \
    do {                                        \
        Scope sc_(h, cls, nk, st, cap);          \
        cudaError_t e_ = (call);                 \
        if (e_ != cudaSuccess) return e_;        \
    } while (0)

cudaError_t enqueue_start(Handle& h, const double* b, const double* x, cudaStream_t st, bool cap = false) {
    ILU2L_SCOPED(PC_RESID, 1, launch_fg_resid(h, b, x, 1, st));
    ILU2L_SCOPED(PC_SCALE, 1, launch_fg_scale0(h, st));
    return cudaSuccess;
}

// one FGMRES cycle: m steps (each a no-op once the cycle is done), update, true residual
cudaError_t enqueue_cycle(Handle& h, const double* b, double* x, cudaStream_t st, bool cap) {
    const int32_t* done = &h.fg.ctl->cycle_done;
    for (int j = 0; j < h.fg.m; j++) {
        cudaError_t e = apply_any(h, h.fg.V + (size_t)j * h.fg.ld, h.fg.Z + (size_t)j * h.fg.ld, done, st, cap);
        if (e != cudaSuccess) return e;
        ILU2L_SCOPED(PC_SPMV_DOT, 1, launch_fg_spmv_dot(h, j, st));
        ILU2L_SCOPED(PC_CGS, 1, launch_fg_cgs(h, j, st));
        ILU2L_SCOPED(PC_NORM, 1, launch_fg_norm(h, j, st));
        ILU2L_SCOPED(PC_NEXT, 1, launch_fg_next(h, j, st));
    }
    ILU2L_SCOPED(PC_UPDATE, 1, launch_fg_update(h, x, st));
    ILU2L_SCOPED(PC_RESID, 1, launch_fg_resid(h, b, x, 0, st));
    ILU2L_SCOPED(PC_SCALE, 1, launch_fg_scale0(h, st));
    return cudaSuccess;
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

}  // namespace
}  // namespace ilu2l

using namespace ilu2l;

extern "C" {

void ilu_opts_default(ilu_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->variant = ILU_VARIANT_SCHUR;
    o->factor_B = ILU_FACT_ILU0;
    o->factor_S = ILU_FACT_MILU0;
    o->form = ILU_FORM_AUTO;
    o->ilut_tau = 1e-3;
    o->ilut_p = 10;
    o->inner_iters = 3;
    o->pc_precision = ILU_PREC_FP32;
    o->ordering = ILU_ORDER_NATURAL;
    o->fill_level = 0;
    o->l1_block = 0;
    o->chain_sched = 0;
    o->gs_precision = 3;
    o->autotune = 0;
    o->ilut_setup = 0;
    o->pivot_eps = 1e-8;
    o->stream = nullptr;
    o->spin_limit = 0;
    o->use_graphs = 1;
    o->block_threads = 0;
    o->analysis_only = 0;
    o->kernel_path = 0;
    o->inner_launch = 0;
}

const char* ilu_status_str(ilu_status s) {
    switch (s) {
        case ILU_OK: return "ok";
        case ILU_ERR_ARG: return "invalid argument";
        case ILU_ERR_CSR: return "malformed CSR matrix";
        case ILU_ERR_OOM: return "out of memory";
        case ILU_ERR_ZERO_PIVOT: return "zero pivot";
        case ILU_ERR_NOT_CONVERGED: return "not converged";
        case ILU_ERR_BREAKDOWN: return "Krylov breakdown";
        case ILU_ERR_TIMEOUT: return "device wait timed out";
        case ILU_ERR_CUDA: return "CUDA error";
        case ILU_ERR_TOO_LARGE: return "problem too large";
        case ILU_ERR_UNSUPPORTED: return "unsupported option";
    }
    return "unknown status";
}

ilu_status ilu_free(void* hp) {
    if (!hp) return ILU_OK;
    Handle* h = (Handle*)hp;
    if (!h->o.analysis_only) cudaStreamSynchronize(h->st);
    if (h->cycle_exec) cudaGraphExecDestroy(h->cycle_exec);
    for (void* p : h->allocs) cudaFreeAsync(p, h->st);
    if (h->h_ctl) ctl_give(h->h_ctl);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    delete h;
    return ILU_OK;
}

ilu_status ilu_setup(const ilu_csr* A, const int32_t* part, int32_t p, const ilu_opts* opts, void** hout) {
    if (!hout) return ILU_ERR_ARG;
    *hout = nullptr;
    if (!A || !part || p < 1) return ILU_ERR_ARG;
    const double t0 = now_ms();
    Handle* h = new (std::nothrow) Handle;
    if (!h) return ILU_ERR_OOM;
    if (opts)
        h->o = *opts;
    else
        ilu_opts_default(&h->o);
    const ilu_opts& o = h->o;
    if ((o.variant != ILU_VARIANT_BJ && o.variant != ILU_VARIANT_SCHUR && o.variant != ILU_VARIANT_RAP) ||
        (o.variant == ILU_VARIANT_RAP && o.factor_B == ILU_FACT_ILUT) || o.factor_B < 0 || o.factor_B > 2 ||
        o.factor_S < 0 || o.factor_S > 3 || o.factor_S == ILU_FACT_ILUT ||
        (o.factor_S == ILU_FACT_PMILU0 && o.variant != ILU_VARIANT_SCHUR) || o.factor_B == ILU_FACT_PMILU0 ||
        (o.pc_precision != ILU_PREC_FP64 && o.pc_precision != ILU_PREC_FP32 && o.pc_precision != ILU_PREC_BF16_STORE) ||
        o.inner_iters < 1 || o.inner_iters > kMaxInner || o.form < 0 || o.form > 2 || o.pivot_eps < 0.0 ||
        (o.factor_B == ILU_FACT_ILUT && (o.ilut_p < 0 || o.ilut_tau < 0.0)) ||
        (o.block_threads != 0 && (o.block_threads % 32 != 0 || o.block_threads > 1024)) ||
        o.kernel_path < 0 || o.kernel_path > 1 || o.inner_launch < 0 || o.inner_launch > 1 ||
        (o.ordering != ILU_ORDER_NATURAL && o.ordering != ILU_ORDER_RCM && o.ordering != ILU_ORDER_COLOR) ||
        o.fill_level < 0 ||
        (o.fill_level > 0 && o.factor_B == ILU_FACT_ILUT) || o.l1_block < 0 || o.l1_block > 1 ||
        (o.l1_block && o.variant != ILU_VARIANT_BJ) || o.chain_sched < 0 || o.chain_sched > 2 ||
        o.gs_precision < 0 || o.gs_precision > 3 || o.autotune < 0 || o.autotune > 1 || o.ilut_setup < 0 ||
        o.ilut_setup > 1) {
        delete h;
        return ILU_ERR_ARG;
    }
    if ((o.variant == ILU_VARIANT_RAP && o.kernel_path != 0) ||
        (o.pc_precision == ILU_PREC_BF16_STORE &&
         (o.kernel_path != 0 || o.factor_B == ILU_FACT_ILUT || (o.variant == ILU_VARIANT_SCHUR && o.form == ILU_FORM_EF)))) {
        delete h;
        return ILU_ERR_UNSUPPORTED;
    }
    h->variant = o.variant;
    h->kB = o.factor_B;
    h->kS = o.factor_S;
    h->prec = o.pc_precision;
    h->inner_k = o.inner_iters;
    h->form = (o.variant == ILU_VARIANT_SCHUR && (o.factor_B == ILU_FACT_ILUT || o.form == ILU_FORM_EF))
                  ? ILU_FORM_EF
                  : ILU_FORM_WZ;
    h->st = (cudaStream_t)o.stream;
    h->threads = o.block_threads ? o.block_threads : 256;
    h->stream_path = (o.kernel_path == 0);
    if (!o.analysis_only) {
        int dev = 0, optin = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess && optin > 0)
            h->smem_optin = optin;
    }
    ilu_status s = host_setup(*h, A, part, p);
    if (s == ILU_OK && (h->variant == ILU_VARIANT_RAP || h->prec == ILU_PREC_BF16_STORE) && !h->stream_path)
        s = ILU_ERR_UNSUPPORTED;
    h->host_ms = now_ms() - t0;
    if (s == ILU_OK && o.analysis_only) {
        h->setup_ms = now_ms() - t0;
        *hout = h;
        return ILU_OK;
    }
    if (s == ILU_OK) {
        s = device_setup(*h);
        if (s == ILU_OK) {
            // the original CSR for the FP64 SpMV
            cudaError_t e = cudaSuccess;
            h->d_A_rp = h->alloc<int32_t>((size_t)A->n + 1, &e);
            h->d_A_ci = h->alloc<int32_t>((size_t)A->nnz, &e);
            h->d_A_v = h->alloc<double>((size_t)A->nnz, &e);
            if (!h->d_A_rp || !h->d_A_ci || !h->d_A_v) s = map_err(e);
            if (s == ILU_OK) {
                e = cudaMemcpyAsync(h->d_A_rp, A->rowptr, ((size_t)A->n + 1) * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, h->st);
                if (e == cudaSuccess && A->nnz)
                    e = cudaMemcpyAsync(h->d_A_ci, A->colind, (size_t)A->nnz * sizeof(int32_t),
                                        cudaMemcpyHostToDevice, h->st);
                if (e == cudaSuccess && A->nnz)
                    e = cudaMemcpyAsync(h->d_A_v, A->val, (size_t)A->nnz * sizeof(double), cudaMemcpyHostToDevice,
                                        h->st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
                s = map_err(e);
            }
        }
    }
    if (s == ILU_OK && o.autotune && h->stream_path && !o.block_threads && h->tune_state == 0)
        s = (h->prec != ILU_PREC_FP64) ? autotune_t<float>(*h) : autotune_t<double>(*h);
    if (s != ILU_OK) {
        ilu_free(h);
        return s;
    }
    // host copies of the value arrays are no longer needed
    decltype(h->q_v)().swap(h->q_v);
    std::vector<double>().swap(h->f1_host_vals);
    h->setup_ms = now_ms() - t0;
    h->device_ms = h->setup_ms - h->host_ms;
    *hout = h;
    return ILU_OK;
}

ilu_status ilu_apply(void* hp, const double* r, double* z) {
    if (!hp || !r || !z || r == z) return ILU_ERR_ARG;
    Handle* h = (Handle*)hp;
    if (h->o.analysis_only) return ILU_ERR_ARG;
    return map_err(apply_any(*h, r, z, nullptr, h->st));
}

ilu_status ilu_spmv(void* hp, const double* x, double* y) {
    if (!hp || !x || !y || x == y) return ILU_ERR_ARG;
    Handle* h = (Handle*)hp;
    if (h->o.analysis_only) return ILU_ERR_ARG;
    h->kernel_launches += 1;
    return map_err(launch_spmv(*h, x, y, h->st));
}

ilu_status ilu_inner_solve(void* hp, const double* gp, double* y) {
    if (!hp || !gp || !y || gp == y) return ILU_ERR_ARG;
    Handle* h = (Handle*)hp;
    if (h->o.analysis_only) return ILU_ERR_ARG;
    if (h->variant != ILU_VARIANT_SCHUR) return ILU_ERR_ARG;
    cudaError_t e = (h->prec != ILU_PREC_FP64) ? launch_inner_io<float>(*h, gp, y, h->st)
                                                : launch_inner_io<double>(*h, gp, y, h->st);
    return map_err(e);
}

ilu_status gmres_solve(void* hp, const double* b, double* x, double rtol, int32_t restart, int32_t maxit,
                       ilu_solve_info* info) {
    if (!hp || !b || !x || b == x || restart < 1 || restart > kMaxRestartGS || maxit < 0 || !(rtol >= 0.0))
        return ILU_ERR_ARG;
    Handle* h = (Handle*)hp;
    if (h->o.analysis_only) return ILU_ERR_ARG;
    const double t0 = now_ms();
    ilu_status s = ensure_fgmres(*h, restart);
    if (s != ILU_OK) return s;
    FgCtl init{};
    init.rtol = rtol;
    init.maxit = maxit;
    init.m = restart;
    *h->h_ctl = init;
    CK(cudaMemcpyAsync(h->fg.ctl, h->h_ctl, sizeof(FgCtl), cudaMemcpyHostToDevice, h->st));
    // the cycles run on the handle's own copies of b and x, so the cycle graph captured
    // for this handle stays valid whatever buffers later calls pass
    const double* ub = b;
    double* ux = x;
    b = h->fg_b;
    x = h->fg_x;
    CK(cudaMemcpyAsync(h->fg_b, ub, (size_t)h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(h->fg_x, ux, (size_t)h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    CK(enqueue_start(*h, b, x, h->st));
    const bool graphs = h->o.use_graphs && !h->prof;
    const double tg = now_ms();
    h->graph_ms_last = 0.0;
    if (graphs && (h->cycle_exec == nullptr || h->cycle_b != b || h->cycle_x != x || h->cycle_m != restart)) {
        if (h->cycle_exec) {
            cudaGraphExecDestroy(h->cycle_exec);
            h->cycle_exec = nullptr;
        }
        cudaStream_t cs;
        CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue_cycle(*h, b, x, cs, true);
            e = cudaStreamEndCapture(cs, &g);
            if (e2 != cudaSuccess) e = e2;
        }
        size_t nodes = 0;
        if (e == cudaSuccess) e = cudaGraphGetNodes(g, nullptr, &nodes);
        h->cycle_nodes = (int64_t)nodes;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->cycle_exec, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return map_err(e);
        h->cycle_b = b;
        h->cycle_x = x;
        h->cycle_m = restart;
        h->graph_ms_last = now_ms() - tg;
    }
    int cycles = 0;
    ilu_status result = ILU_OK;
    for (;;) {
        CK(cudaMemcpyAsync(h->h_ctl, h->fg.ctl, sizeof(FgCtl), cudaMemcpyDeviceToHost, h->st));
        CK(cudaMemcpyAsync(&h->h_ctl->err, h->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        const FgCtl& c = *h->h_ctl;
        if (c.err & 2) {
            result = ILU_ERR_TIMEOUT;
            break;
        }
        if (c.converged) {
            if (c.bnorm == 0.0) CK(cudaMemsetAsync(x, 0, (size_t)h->n * sizeof(double), h->st));
            result = ILU_OK;
            break;
        }
        if (c.total >= maxit) {
            result = ILU_ERR_NOT_CONVERGED;
            break;
        }
        if (graphs) {
            CK(cudaGraphLaunch(h->cycle_exec, h->st));
            h->graph_launches++;
            h->kernel_launches += h->cycle_nodes;
        } else {
            CK(enqueue_cycle(*h, b, x, h->st, false));
        }
        cycles++;
    }
    CK(cudaMemcpyAsync(ux, h->fg_x, (size_t)h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->solve_ms_last = now_ms() - t0;
    const FgCtl& c = *h->h_ctl;
    if (info) {
        info->iters = c.total;
        info->restarts = cycles;
        info->rel_res_true = c.bnorm > 0 ? c.res_true / c.bnorm : 0.0;
        info->rel_res_est = c.bnorm > 0 ? c.est / c.bnorm : 0.0;
        info->setup_ms = h->setup_ms;
        info->solve_ms = now_ms() - t0;
        info->status = result;
        info->npert = h->npert;
    }
    return result;
}

ilu_status ilu_get_sizes(void* hp, int64_t* out) {
    if (!hp || !out) return ILU_ERR_ARG;
    Handle* h = (Handle*)hp;
    host_levels(*h);
    out[0] = h->n;
    out[1] = h->p;
    out[2] = h->n1;
    out[3] = h->n2;
    out[4] = h->nnz;
    out[5] = h->nnz_coff;
    out[6] = h->npert;
    out[7] = h->nlev[2];
    out[8] = h->nlev[3];
    out[9] = h->nlev[4];
    out[10] = h->nlev[5];
    out[11] = h->max_ns;
    const int reported[4] = {PR_BJ, PR_FWD, PR_S, PR_BWD};  // out[12..23], as documented
    for (int pr = 0; pr < 4; pr++) {
        const ProgHost& P = h->prog[reported[pr]];
        out[12 + 3 * pr] = (int64_t)P.prow.size();
        out[13 + 3 * pr] = (int64_t)P.pcol.size();
        out[14 + 3 * pr] = P.lvl_ptr.empty() ? 0 : (int64_t)P.lvl_ptr.size() - 1;
    }
    return ILU_OK;
}

ilu_status ilu_get_perm(void* hp, int32_t* perm, int32_t* iperm, int32_t* int_ptr, int32_t* if_ptr,
                        int32_t* iface) {
    if (!hp) return ILU_ERR_ARG;
    Handle* h = (Handle*)hp;
    if (perm) std::memcpy(perm, h->perm.data(), h->perm.size() * sizeof(int32_t));
    if (iperm) std::memcpy(iperm, h->iperm.data(), h->iperm.size() * sizeof(int32_t));
    if (int_ptr) std::memcpy(int_ptr, h->int_ptr.data(), h->int_ptr.size() * sizeof(int32_t));
    if (if_ptr) std::memcpy(if_ptr, h->if_ptr.data(), h->if_ptr.size() * sizeof(int32_t));
    if (iface)
        for (int32_t i = 0; i < h->n; i++) iface[i] = h->iface[i];
    return ILU_OK;
}

ilu_status ilu_get_levels(void* hp, int32_t which, int32_t* lev, int32_t* nlev) {
    if (!hp || !lev || which < 0 || which > 5) return ILU_ERR_ARG;
    Handle* h = (Handle*)hp;
    host_levels(*h);
    std::memcpy(lev, h->lev[which].data(), h->lev[which].size() * sizeof(int32_t));
    if (nlev) *nlev = h->nlev[which];
    return ILU_OK;
}

ilu_status ilu_get_local_factor(void* hp, int32_t s, int32_t fact, double* val) {
    if (!hp || !val) return ILU_ERR_ARG;
    Handle* h = (Handle*)hp;
    if (h->o.analysis_only || s < 0 || s >= h->p || (fact != 1 && fact != 2)) return ILU_ERR_ARG;
    const FPat& F = (fact == 1) ? h->f1 : h->f2;
    const bool pattern_of_A = (fact == 1) ? h->f1_device : true;
    if (!pattern_of_A) return ILU_ERR_ARG;
    const int32_t q0 = h->qoff[s], q1 = h->qoff[s + 1];
    const int64_t b = h->q_rp[q0], e = h->q_rp[q1];
    CK(cudaMemcpy(val, h->d_vals + F.base + b, (size_t)(e - b) * sizeof(double), cudaMemcpyDeviceToHost));
    return ILU_OK;
}

ilu_status ilu_get_local_pattern(void* hp, int32_t s, int32_t* rowptr, int32_t* colind, int32_t* nnz) {
    if (!hp || !nnz) return ILU_ERR_ARG;
    Handle* h = (Handle*)hp;
    if (s < 0 || s >= h->p) return ILU_ERR_ARG;
    const int32_t q0 = h->qoff[s], q1 = h->qoff[s + 1];
    const int32_t b = h->q_rp[q0];
    *nnz = h->q_rp[q1] - b;
    if (rowptr)
        for (int32_t q = q0; q <= q1; q++) rowptr[q - q0] = h->q_rp[q] - b;
    if (colind) std::memcpy(colind, h->q_ci.data() + b, (size_t)*nnz * sizeof(int32_t));
    return ILU_OK;
}

ilu_status ilu_profile(void* hp, int32_t enable) {
    if (!hp) return ILU_ERR_ARG;
    Handle* h = (Handle*)hp;
    if (!h->o.analysis_only) CK(cudaStreamSynchronize(h->st));
    h->prof = enable != 0;
    h->prof_recs.clear();
    h->ev_used = 0;
    for (int i = 0; i < PC_COUNT; i++) {
        h->prof_ms[i] = 0.0;
        h->prof_n[i] = 0;
    }
    return ILU_OK;
}

ilu_status ilu_profile_read(void* hp, const char** names, double* ms, int64_t* launches, int32_t* count) {
    if (!hp || !count) return ILU_ERR_ARG;
    Handle* h = (Handle*)hp;
    if (!h->prof_recs.empty()) {
        CK(cudaEventSynchronize(h->prof_recs.back().b));
        for (const auto& r : h->prof_recs) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, r.a, r.b));
            h->prof_ms[r.cls] += t;
            h->prof_n[r.cls] += r.nkern;
        }
        h->prof_recs.clear();
        h->ev_used = 0;
    }
    const int m = std::min<int>(*count, PC_COUNT);
    for (int i = 0; i < m; i++) {
        if (names) names[i] = kProfNames[i];
        if (ms) ms[i] = h->prof_ms[i];
        if (launches) launches[i] = h->prof_n[i];
    }
    *count = PC_COUNT;
    return ILU_OK;
}

ilu_status ilu_get_stats(void* hp, int64_t* out) {
    if (!hp || !out) return ILU_ERR_ARG;
    Handle* h = (Handle*)hp;
    out[0] = h->kernel_launches;
    out[1] = h->graph_launches;
    out[2] = h->cycle_nodes;
    out[3] = (int64_t)h->fg_G;
    out[4] = 0;
    if (!h->o.analysis_only && h->d_err) {
        int32_t e = 0;
        CK(cudaStreamSynchronize(h->st));
        CK(cudaMemcpy(&e, h->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
        out[4] = e;
    }
    out[5] = h->stream_path ? 1 : 0;
    out[14] = h->inner_coop ? 1 : 0;
    out[15] = (int64_t)h->device_bytes;
    const int ids[4] = {PR_BJ, PR_FWDS, PR_S, PR_BWD};
    for (int i = 0; i < 4; i++) {
        out[6 + 2 * i] = h->sh[ids[i]].ch0.empty() ? 0 : h->sh[ids[i]].rw;
        out[7 + 2 * i] = h->sh[ids[i]].ch0.empty() ? 0 : h->sh[ids[i]].nt;
    }
    return ILU_OK;
}

ilu_status ilu_get_times(void* hp, double* out) {
    if (!hp || !out) return ILU_ERR_ARG;
    const Handle* h = (const Handle*)hp;
    out[0] = h->host_ms;
    out[1] = h->device_ms;
    out[2] = h->solve_ms_last;
    out[3] = h->graph_ms_last;
    out[4] = h->kB == ILU_FACT_ILUT ? h->ilut_ms : 0.0;
    out[5] = (h->kB == ILU_FACT_ILUT && h->ilut_device) ? 1.0 : 0.0;
    out[6] = (h->kB == ILU_FACT_ILUT && h->ilut_device) ? h->ilut_kernel_ms : 0.0;
    return ILU_OK;
}

ilu_status ilu_get_ilut_factor(void* hp, int32_t s, int32_t* rowptr, int32_t* colind, double* val,
                               int32_t* nnz) {
    if (!hp || !nnz) return ILU_ERR_ARG;
    Handle* h = (Handle*)hp;
    if (h->kB != ILU_FACT_ILUT || s < 0 || s >= h->p) return ILU_ERR_ARG;
    const int32_t q0 = h->qoff[s];
    const int32_t m = (h->variant != ILU_VARIANT_BJ) ? h->nint[s] : (h->qoff[s + 1] - q0);
    const int32_t e0 = h->f1_rp[q0], e1 = h->f1_rp[q0 + m];
    *nnz = e1 - e0;
    if (rowptr)
        for (int32_t r = 0; r <= m; r++) rowptr[r] = h->f1_rp[q0 + r] - e0;
    if (colind)
        for (int32_t k = e0; k < e1; k++) colind[k - e0] = h->f1_ci[k];
    if (val && e1 > e0) {
        if (h->o.analysis_only) {
            for (int32_t k = e0; k < e1; k++) val[k - e0] = h->f1_host_vals[k];
        } else {
            cudaError_t e = cudaMemcpyAsync(val, h->d_vals + h->f1.base + e0, (size_t)(e1 - e0) * sizeof(double),
                                            cudaMemcpyDeviceToHost, h->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
            if (e != cudaSuccess) return ILU_ERR_CUDA;
        }
    }
    return ILU_OK;
}

ilu_status ilu_get_tuning(void* hp, int32_t* nt, double* ms, int32_t* state) {
    if (!hp || !nt || !ms || !state) return ILU_ERR_ARG;
    const Handle* h = (const Handle*)hp;
    const int ids[4] = {PR_BJ, PR_FWDS, PR_S, PR_BWD};
    for (int i = 0; i < 4; i++) {
        const StreamHost& S = h->sh[ids[i]];
        nt[i] = S.ch0.empty() ? 0 : S.nt;
        for (int c = 0; c < kTuneCands; c++) ms[4 * i + c] = h->tune_ms[ids[i]][c];
    }
    *state = h->tune_state;
    return ILU_OK;
}

ilu_status ilu_get_krylov(void* hp, int32_t which, int32_t k, double* out) {
    if (!hp || !out || which < 0 || which > 1 || k < 1) return ILU_ERR_ARG;
    Handle* h = (Handle*)hp;
    if (h->o.analysis_only || !h->fg.V || k > (which == 0 ? h->fg_m + 1 : h->fg_m)) return ILU_ERR_ARG;
    if (which == 0 && h->fg.Vlo) {
        // the double-float Gram-Schmidt keeps the basis as two FP32 parts: v = hi + lo (the
        // FP64 array holds their sum, rounded)
        const size_t nk = (size_t)h->n * (size_t)k;
        std::vector<float> hi(nk), lo(nk);
        CK(cudaMemcpy2DAsync(hi.data(), (size_t)h->n * sizeof(float), h->fg.V32, (size_t)h->fg.ld * sizeof(float),
                             (size_t)h->n * sizeof(float), (size_t)k, cudaMemcpyDeviceToHost, h->st));
        CK(cudaMemcpy2DAsync(lo.data(), (size_t)h->n * sizeof(float), h->fg.Vlo, (size_t)h->fg.ld * sizeof(float),
                             (size_t)h->n * sizeof(float), (size_t)k, cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        for (size_t i = 0; i < nk; i++) out[i] = (double)hi[i] + (double)lo[i];
        return ILU_OK;
    }
    const double* src = which == 0 ? h->fg.V : h->fg.Z;
    CK(cudaMemcpy2DAsync(out, (size_t)h->n * sizeof(double), src, (size_t)h->fg.ld * sizeof(double),
                         (size_t)h->n * sizeof(double), (size_t)k, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return ILU_OK;
}

ilu_status ilu_get_stream_stats(void* hp, int32_t program, int64_t* out) {
    if (!hp || !out || program < 0 || program > 3) return ILU_ERR_ARG;
    const Handle* h = (const Handle*)hp;
    const int ids[4] = {PR_BJ, PR_FWDS, PR_S, PR_BWD};
    const StreamHost& S = h->sh[ids[program]];
    for (int i = 0; i < 13; i++) out[i] = 0;
    if (S.ch0.empty()) return ILU_OK;
    out[10] = S.max_scan_waves;
    out[11] = S.max_steps;
    out[12] = S.chain_sections;
    out[8] = (int64_t)h->nst * h->chunk;
    out[9] = (!h->o.analysis_only && h->max_ns + 1 <= h->smem_len_stream) ? 1 : 0;
    out[0] = S.rw;
    out[1] = S.nt;
    out[2] = S.ch0.back();
    out[3] = S.waves;
    out[4] = S.records;
    out[5] = S.skips;
    out[6] = S.max_barriers;
    out[7] = S.max_levels_sub;
    return ILU_OK;
}

ilu_status ilu_get_stream(void* hp, int32_t program, uint8_t* blob, int32_t* ch0, int64_t* meta) {
    if (!hp || !meta || program < 0 || program > 3) return ILU_ERR_ARG;
    const Handle* h = (const Handle*)hp;
    const int ids[4] = {PR_BJ, PR_FWDS, PR_S, PR_BWD};
    const StreamHost& S = h->sh[ids[program]];
    if (S.ch0.empty()) return ILU_ERR_UNSUPPORTED;
    meta[0] = (int64_t)S.blob.size();
    meta[1] = S.chunk;
    meta[2] = S.rw;
    meta[3] = S.val_bytes;
    meta[4] = S.nt;
    meta[5] = S.x_bytes;
    if (blob) memcpy(blob, S.blob.data(), S.blob.size());
    if (ch0) memcpy(ch0, S.ch0.data(), S.ch0.size() * sizeof(int32_t));
    return ILU_OK;
}

}  // extern "C"
