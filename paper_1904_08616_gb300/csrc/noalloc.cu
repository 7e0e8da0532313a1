// lq_cg_solve_noalloc: the CG solver of lq_cg_solve with its scratch memory in a fixed
// device array of this library instead of a caller-provided workspace.
//
// Some callers cannot allocate device memory when they want to solve: code that runs
// under a no-allocation rule after start-up (real-time or safety-reviewed loops), plugins
// living inside a host program whose allocator owns all device memory, or callers that
// have no handle on a CUDA allocator at all.  They pass only the inputs and the output;
// the scratch is the array below, which every GPU that loads this library holds until
// the process exits.
#include <mutex>

#include "lq_abi_internal.h"
#include "lq_internal.cuh"

namespace {

// Largest workspace the fixed array serves (see lq_cg_workspace_bytes).  64 MiB covers a
// 12^4 lattice in every mode (35-43 MiB); a 16^4 lattice needs 73 MiB in FP64 and 110-133 MiB
// in the other modes, so it is rejected.
constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device.  In host code the array's name is
// only a host-side stand-in, so the address must come from cudaGetSymbolAddress, once per
// device, with that device current.  Under CUDA's lazy module loading this first lookup is
// also when the module holding the array is loaded on the device, i.e. when its 64 MiB are
// reserved (and can fail for lack of memory).  The cached address stays valid as long as
// the device's primary context lives: a cudaDeviceReset while the library is loaded
// would leave it dangling.
int scratch_for_current_device(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lq::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return lq::fail(LQ_ERR_ARG, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return lq::cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return LQ_OK;
}

}  // namespace

extern "C" size_t lq_cg_noalloc_max_workspace_bytes(void) { return kNoAllocScratchBytes; }

extern "C" int lq_cg_solve_noalloc(const int32_t dims[4], double m_q, int32_t mode, const void* U,
                                   const void* eta, void* x, const lq_cg_params* params, lq_cg_info* info,
                                   void* cuda_stream) {
    if (info) *info = lq_cg_info{};
    const size_t need = lq_cg_workspace_bytes(dims, mode);
    if (need == 0) return lq_cg_solve(dims, m_q, mode, U, eta, x, params, nullptr, 0, info, cuda_stream);
    if (need > kNoAllocScratchBytes) {
        if (info) info->status = LQ_ERR_WORKSPACE;
        return lq::fail(LQ_ERR_WORKSPACE,
                        "lattice needs %zu bytes of scratch; the fixed no-allocation array holds %zu "
                        "(use lq_cg_solve with a workspace)", need, kNoAllocScratchBytes);
    }
    void* ws = nullptr;
    const int r = scratch_for_current_device(&ws);
    if (r != LQ_OK) {
        if (info) info->status = r;
        return r;
    }
    // The solver initialises every part of the scratch it reads (state record, partial
    // sums, vectors), so the previous call's contents need no clearing here.  The inner loop
    // runs host-driven: building a CUDA graph would allocate.
    lq_cg_params prm{1e-10, 100000, 0, 0.0, 0, 0};
    if (params) prm = *params;
    prm.flags |= LQ_CG_NO_GRAPH;
    return lq_cg_solve(dims, m_q, mode, U, eta, x, &prm, ws, kNoAllocScratchBytes, info, cuda_stream);
}
