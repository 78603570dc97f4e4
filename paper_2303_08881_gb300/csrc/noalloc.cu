// noalloc.cu -- ilu_inner_solve_noalloc: the inner Schur solve with its Krylov workspace
// in a fixed device array owned by the library, for callers that must not allocate.
//
// ilu_inner_solve keeps its workspace (Arnoldi vectors, the C_off product, partial sums
// and the small control block) in memory the handle allocated during ilu_setup. This
// variant places the same workspace in the file-scope array below instead, so the call
// itself never allocates: no cudaMalloc, no cudaFree, no allocating library routine.
// Every GPU that loads the library holds the array (kWorkspaceBytes) until the process
// exits. Calls share the array and it keeps the last call's contents: the start kernel of
// every call re-initialises the control state it relies on (step counter, zero flag,
// barrier words) and writes every vector before reading it; the memset of the control
// block before it is a defensive extra that also clears the Hessenberg entries. Calls
// whose executions overlap on the GPU (two streams, or two host threads) race on the array.
// The array's device address is looked up once per device and cached for the life of the
// process: a cudaDeviceReset (or any reset of the device's primary context) invalidates it,
// and calls after such a reset are not supported.
#include <mutex>

#include "handle.h"

namespace ilu2l {

namespace {

constexpr size_t kWorkspaceBytes = size_t(8) << 20;  // 8 MiB

static __device__ __align__(256) unsigned char g_inner_workspace[kWorkspaceBytes];

// Host code cannot pass g_inner_workspace to a kernel (its host-side name is a stand-in,
// not a device address): the device address is fetched once per device with that device
// current and cached here.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_dev_addr[kMaxDevices] = {};

cudaError_t workspace_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_inner_workspace);
        if (e != cudaSuccess) return e;
        g_dev_addr[dev] = p;
    }
    *out = g_dev_addr[dev];
    return cudaSuccess;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

template <class T>
ilu_status inner_noalloc(Handle& h, const double* gp, double* y) {
    const size_t n2 = (size_t)std::max(h.n2, 1);
    const size_t off_part = up256(sizeof(InnerCtl));
    const size_t off_v = off_part + up256((size_t)3 * (kMaxInner + 1) * h.p * sizeof(double));
    const size_t off_w0 = off_v + up256((size_t)(h.inner_k + 1) * n2 * sizeof(T));
    const size_t off_w1 = off_w0 + up256(n2 * sizeof(T));
    const size_t off_t = off_w1 + up256(n2 * sizeof(T));
    const size_t total = off_t + up256(n2 * sizeof(T));
    if (total > kWorkspaceBytes) return ILU_ERR_TOO_LARGE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return ILU_ERR_CUDA;
    if (dev != h.device) return ILU_ERR_ARG;
    void* base = nullptr;
    if (workspace_address(dev, &base) != cudaSuccess) return ILU_ERR_CUDA;
    uint8_t* b = static_cast<uint8_t*>(base);
    if (cudaMemsetAsync(b, 0, sizeof(InnerCtl), h.st) != cudaSuccess) return ILU_ERR_CUDA;
    InnerDev<T> in = h.innerdev<T>();
    in.ctl = reinterpret_cast<InnerCtl*>(b);
    in.part = reinterpret_cast<double*>(b + off_part);
    in.V = reinterpret_cast<T*>(b + off_v);
    in.W0 = reinterpret_cast<T*>(b + off_w0);
    in.W1 = reinterpret_cast<T*>(b + off_w1);
    T* tbuf = reinterpret_cast<T*>(b + off_t);
    return launch_inner_io_ws<T>(h, in, tbuf, gp, y, h.st) == cudaSuccess ? ILU_OK : ILU_ERR_CUDA;
}

}  // namespace
}  // namespace ilu2l

using namespace ilu2l;

extern "C" ilu_status ilu_inner_solve_noalloc(void* hp, const double* gp, double* y) {
    if (!hp || !gp || !y || gp == y) return ILU_ERR_ARG;
    Handle* h = static_cast<Handle*>(hp);
    if (h->o.analysis_only || h->variant != ILU_VARIANT_SCHUR) return ILU_ERR_ARG;
    if (!h->stream_path || h->max_ns + 1 > h->smem_len_stream) return ILU_ERR_UNSUPPORTED;
    return (h->prec != ILU_PREC_FP64) ? inner_noalloc<float>(*h, gp, y) : inner_noalloc<double>(*h, gp, y);
}
