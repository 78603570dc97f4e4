// handle.h -- the ilu2l handle: host-side setup products and device buffers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"

namespace ilu2l {

enum ProgId { PR_BJ = 0, PR_FWD = 1, PR_S = 2, PR_BWD = 3, PR_FWDS = 4, PR_COUNT = 5 };

// A factor's sparsity pattern over all Q rows (rows outside the factor are empty).
// Values live in the handle's value array at [base + k] for pattern entry k.
// A factor pattern in Q order, as a view: rp[n + 1], ci[nnz] (local columns), dpos[n]
// (diagonal entry or -1) point into arrays the handle owns (the local blocks' own q_*
// arrays, or the host ILUT pattern); base = offset of its values in the value array.
struct FPat {
    const int32_t* rp = nullptr;
    const int32_t* ci = nullptr;
    const int32_t* dpos = nullptr;
    int64_t nnz = 0;
    int64_t base = 0;
};

// A level program laid out as TMA chunks (stream_layout.h) for one index width.
struct StreamHost {
    rawvec<uint8_t> blob;        // chunks of every subdomain, kChunk bytes each
    std::vector<int32_t> ch0;    // p+1: subdomain s owns chunks [ch0[s], ch0[s+1])
    rawvec<int64_t> voff, doff;  // byte offsets of value / pivot-inverse slots
    rawvec<int32_t> vsrc, dsrc;  // their sources in the value array
    uint32_t chunk = 8192;
    int idx_bytes = 2, val_bytes = 4, x_bytes = 4;
    int rw = 4;                       // entries per row record (compile-time width on the device)
    uint32_t rec_bytes = 32;
    int nt = 32;                      // threads of the consumer group
    int64_t levels = 0, rows = 0, entries = 0;
    int64_t waves = 0, segments = 0, records = 0, skips = 0;  // totals over the subdomains
    int64_t max_barriers = 0;                   // group barriers of the longest subdomain program
    int64_t max_levels_sub = 0;                 // levels of the deepest subdomain program
    int64_t max_scan_waves = 0;                 // scan waves of the subdomain program with most
    int64_t max_steps = 0;                      // barriers + scan waves, largest over the subdomains
    int64_t chain_sections = 0;                 // subdomains whose chain section runs as chains
    std::vector<int32_t> order;                 // p: subdomains by descending estimated cost (the
                                                // launch order of the apply kernels)
};

struct StreamBufs {
    uint8_t* blob = nullptr;
    int32_t* ch0 = nullptr;
    int32_t* order = nullptr;
    uint32_t chunk = 8192;
    int nt = 32;
    int rw = 4;
};

// The introspection level sets (Handle::lev / nlev), built on the first call.
void host_levels(Handle& h);

// Process-wide record of the consumer-group sizes the autotuner measured, keyed by a
// fingerprint of the problem's structure and options (taken once the programs are built).
uint64_t tune_key(const Handle& h);
bool tune_lookup(uint64_t key, int32_t (&nt)[PR_COUNT]);
void tune_store(uint64_t key, const int32_t (&nt)[PR_COUNT]);
constexpr int kTuneCands = 4;
constexpr int kTuneNt[kTuneCands] = {32, 64, 96, 128};

// Builds the chunked stream of program P; false if a single row does not fit a chunk.
// x_bytes: element size of the working vector (and of dinv); val_bytes: of the values.
// chain_sched: ilu_opts.chain_sched (0 the cheaper of levels and chains, 1 levels, 2 chains).
bool build_stream(const ProgHost& P, int32_t p, int idx_bytes, int x_bytes, int val_bytes, uint32_t chunk,
                  StreamHost& S, int chain_sched);

struct ProgBufs {
    int32_t *sub_lvl = nullptr, *lvl_ptr = nullptr, *prow = nullptr, *pptr = nullptr,
            *pcol = nullptr, *psrc = nullptr, *pdsrc = nullptr;
    void* pval = nullptr;
    void* pdinv = nullptr;
};

struct Handle {
    ilu_opts o{};
    cudaStream_t st = nullptr;
    int device = 0;
    int32_t n = 0, p = 0, n1 = 0, n2 = 0;
    int64_t nnz = 0, nnz_coff = 0;
    int variant = 1, form = 1, prec = 1, kB = 0, kS = 1;
    bool f2_alias = false, f1_device = true;
    bool ilut_device = false;  // the ILUT factor F1 was computed by the device kernel
    double ilut_ms = 0.0;      // wall time of the ILUT factorisation (part of host_ms)
    double ilut_kernel_ms = 0.0;  // of it, the device kernels (CUDA events)
    double* d_f1_stage = nullptr;  // device ILUT values in f1 order until the device setup
    int npert = 0;
    double setup_ms = 0.0;
    double host_ms = 0.0, device_ms = 0.0;        // the two parts of setup_ms
    double solve_ms_last = 0.0, graph_ms_last = 0.0;  // last gmres_solve; its graph build
    double* rap_res = nullptr;                    // multiplicative variant: b - A x^, P v and
    double* rap_pv = nullptr;                     // A P v, full vectors in the original order
    double* rap_apv = nullptr;
    double* fg_b = nullptr;                       // the solve's own copies of b and x: the
    double* fg_x = nullptr;                       // cycle graph is built once per handle
    int threads = 256;       // threads of the per-subdomain kernels
    int32_t smem_len = 0;    // working vector capacity (elements of the PC type)
    int32_t max_ns = 0;
    int sm_count = 152;

    // host products (kept for introspection)
    std::vector<int32_t> part, iface, perm, iperm, int_ptr, if_ptr, qoff, nint, q_orig;
    std::vector<int32_t> q_rp, q_dpos;  // local CSR of every A_s, Q order
    rawvec<int32_t> q_ci;               // (filled by host threads: no zero fill first)
    rawvec<double> q_v;
    std::vector<int32_t> lev[6];
    int32_t nlev[6] = {0, 0, 0, 0, 0, 0};
    FPat f1, f2;           // patterns of the two factorisations (f2 may equal f1)
    FPat apat;             // pattern of the local blocks A_s themselves
    bool lev_ready = false;  // lev / nlev computed (on the first introspection call)
    std::vector<double> f1_host_vals;  // ILUT values (host-computed factor F1)
    std::vector<int32_t> f1_rp, f1_dpos;  // its pattern (f1 views it)
    rawvec<int32_t> f1_ci;
    int64_t a_base = 0;    // region of the original local values in the value array
    int64_t nvals = 0;
    ProgHost prog[PR_COUNT];
    ProgHost numprog;      // L_A levels of every A_s for the numeric factorisation
    std::vector<int32_t> coff_rp, coff_ci;
    std::vector<double> coff_v;

    // device memory
    std::vector<void*> allocs;
    std::vector<size_t> alloc_bytes;  // sizes of allocs, for the device footprint
    size_t device_bytes = 0;
    int32_t *d_qoff = nullptr, *d_nint = nullptr, *d_if_ptr = nullptr, *d_q_orig = nullptr;
    int32_t *d_q_rp = nullptr, *d_q_ci = nullptr, *d_q_dpos = nullptr;
    double* d_vals = nullptr;        // [F1 | F2 | A_local] FP64 values
    int32_t *d_A_rp = nullptr, *d_A_ci = nullptr;
    double* d_A_v = nullptr;         // the original matrix (FP64 SpMV)
    ProgBufs pb[PR_COUNT];
    StreamHost sh[PR_COUNT];          // chunked streams (fast path)
    StreamBufs sb[PR_COUNT];
    bool stream_path = true;          // TMA-streamed level programs (else generic kernels)
    uint64_t tune_key_v = 0;          // structural fingerprint (autotune)
    int tune_state = 0;               // 0 rule, 1 measured, 2 from the process-wide record
    double tune_ms[PR_COUNT][kTuneCands] = {};
    int idx_bytes = 2;                // local index width of the streams
    int nst = 4;                      // ring stages
    uint32_t chunk = 8192;            // bytes per chunk / ring stage
    int smem_optin = 232448;          // the device's shared memory per block (opt-in)
    bool inner_coop = false;          // inner solve as one cooperative launch
    int32_t smem_len_stream = 0;      // working-vector capacity with the ring present
    void* d_tbuf = nullptr;           // C_off product of the inner step (interface numbering)
    int32_t *d_num_sub = nullptr, *d_num_lvl = nullptr, *d_num_row = nullptr;
    int32_t *d_coff_rp = nullptr, *d_coff_ci = nullptr;
    void* d_coff_v = nullptr;        // PC type
    void* d_fq = nullptr;            // f' buffer (Q order, PC type)
    void* d_xg = nullptr;            // global working vectors for oversize subdomains
    void* d_iV = nullptr;            // inner Arnoldi vectors
    void* d_iW0 = nullptr;
    void* d_iW1 = nullptr;
    double* d_ipart = nullptr;
    InnerCtl* d_ictl = nullptr;
    int32_t* d_err = nullptr;        // device error word (bit flags)
    int32_t* d_npert = nullptr;
    double* d_tmp_in = nullptr;      // n2-vector staging for ilu_inner_solve
    int32_t inner_k = 3;

    // FGMRES workspace (grown on demand)
    FgDev fg{};
    int32_t fg_m = 0;
    int fg_G = 0;
    int fg_threads = 256;
    cudaGraphExec_t cycle_exec = nullptr;
    int32_t cycle_m = 0;
    const double* cycle_b = nullptr;
    double* cycle_x = nullptr;
    FgCtl* h_ctl = nullptr;          // pinned host mirror of the control block

    // profiling: one event pair per bracketed launch group, summed at read time
    struct ProfRec {
        int cls;
        int nkern;
        cudaEvent_t a, b;
    };
    bool prof = false;
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    double prof_ms[PC_COUNT] = {};
    int64_t prof_n[PC_COUNT] = {};
    // launch accounting: kernels enqueued directly or as graph nodes
    int64_t kernel_launches = 0;
    int64_t graph_launches = 0;
    int64_t cycle_nodes = 0;

    // Device memory is stream-ordered on the handle's stream (cudaMallocAsync / FreeAsync):
    // freeing never synchronises the device, so handles built, used and freed by several
    // threads at once do not stall each other's work.
    template <class T>
    T* alloc(size_t count, cudaError_t* err) {
        void* p = nullptr;
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMallocAsync(&p, bytes, st);
        if (e != cudaSuccess) {
            *err = e;
            return nullptr;
        }
        allocs.push_back(p);
        alloc_bytes.push_back(bytes);
        device_bytes += bytes;
        return (T*)p;
    }

    void release(void* q) {
        for (size_t i = 0; i < allocs.size(); i++)
            if (allocs[i] == q) {
                cudaFreeAsync(q, st);
                device_bytes -= alloc_bytes[i];
                allocs.erase(allocs.begin() + (long)i);
                alloc_bytes.erase(alloc_bytes.begin() + (long)i);
                return;
            }
    }

    SubDev sub() const {
        SubDev s;
        s.qoff = d_qoff;
        s.nint = d_nint;
        s.if_ptr = d_if_ptr;
        s.q_orig = d_q_orig;
        s.p = p;
        s.n = n;
        s.n1 = n1;
        s.n2 = n2;
        s.smem_len = smem_len;
        return s;
    }

    template <class T>
    ProgDev<T> progdev(int id) const {
        ProgDev<T> d;
        d.sub_lvl = pb[id].sub_lvl;
        d.lvl_ptr = pb[id].lvl_ptr;
        d.prow = pb[id].prow;
        d.pptr = pb[id].pptr;
        d.pcol = pb[id].pcol;
        d.pval = (const T*)pb[id].pval;
        d.pdinv = (const T*)pb[id].pdinv;
        return d;
    }

    template <class T>
    InnerDev<T> innerdev() const {
        InnerDev<T> d;
        d.coff_rp = d_coff_rp;
        d.coff_ci = d_coff_ci;
        d.coff_v = (const T*)d_coff_v;
        d.V = (T*)d_iV;
        d.W0 = (T*)d_iW0;
        d.W1 = (T*)d_iW1;
        d.part = d_ipart;
        d.ctl = d_ictl;
        d.k = inner_k;
        return d;
    }
};

// host setup (setup_host.cpp): validation, classification, permutation, local blocks,
// C_off, factor patterns (ILUT values from device_ilut or on the host), level sets and
// level programs.
ilu_status host_setup(Handle& h, const ilu_csr* A, const int32_t* part, int32_t p);

// ILUT of the local blocks on the device (kernels_ilut.cu), called by host_setup; fills the
// host pattern and values of F1 as the host factorisation does.
ilu_status device_ilut(Handle& h);

}  // namespace ilu2l
