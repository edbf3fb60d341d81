// Allocation-free form of mlbm_reduce_fields_device.
//
// The two-pass FP64 reduction needs a scratch array of per-block partial
// sums.  Here that scratch is a file-scope device array, so the caller passes
// only its inputs and the 6-double output and nothing is allocated on any call.
// Host code cannot use the array's name as a device address (it is a host-side
// stand-in for the symbol); the device address is looked up with
// cudaGetSymbolAddress, with the device current, the first time a CUDA
// context is seen on that device, and cached for that context.  A context is
// recognised by its process-unique id (cuCtxGetId, reached through the
// runtime's driver entry points, so no driver library is linked), so after
// cudaDeviceReset, or under another context made current by the caller, the
// address is looked up again instead of reusing one from a context that is gone.
#include <cuda.h>

#include <mutex>
#include <string>

#include "kernels.h"
#include "mlbm_internal.h"

namespace {

constexpr int kMaxDevices = 64;

// 6 partial sums per block, at most kReduceMaxBlocks blocks for any n
static __device__ __align__(256) double g_reduce_partials[6 * mlbm::kReduceMaxBlocks];

struct CachedAddress {
    unsigned long long ctx_id = 0;  // 0: nothing cached
    double* ptr = nullptr;
};

std::mutex g_setup_mu;
CachedAddress g_partials[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
bool g_entry_points_tried = false;

// Id of the calling thread's current context (0 if there is none or the
// driver entry points are missing).  Called with g_setup_mu held.
unsigned long long current_ctx_id() {
    if (!g_entry_points_tried) {
        g_entry_points_tried = true;
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa{}, qb{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(a);
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(b);
        }
        (void)cudaGetLastError();
    }
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array in the current device's current
// context (looked up with that device current on the first call in each
// context; a context id of 0, which the driver never hands out, means
// "unknown" and is never cached).
mlbm_status partials_on_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return mlbm::set_error(MLBM_E_CUDA, std::string("reduce_fields_device_noalloc: cudaGetDevice: ") +
                                                cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return mlbm::set_error(MLBM_E_INVALID, "reduce_fields_device_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    CachedAddress& c = g_partials[dev];
    unsigned long long id = current_ctx_id();
    if (id == 0 || id != c.ctx_id || !c.ptr) {
        void* ptr = nullptr;
        // also makes the device's primary context current if none was
        e = cudaGetSymbolAddress(&ptr, g_reduce_partials);
        if (e != cudaSuccess || !ptr)
            return mlbm::set_error(MLBM_E_CUDA, std::string("reduce_fields_device_noalloc: cudaGetSymbolAddress: ") +
                                                    cudaGetErrorString(e));
        c.ptr = static_cast<double*>(ptr);
        c.ctx_id = current_ctx_id();
    }
    *out = c.ptr;
    return MLBM_OK;
}

}  // namespace

extern "C" int64_t mlbm_reduce_noalloc_max_nodes(void) { return (int64_t)INT32_MAX; }

extern "C" mlbm_status mlbm_reduce_fields_device_noalloc(const float* rho, const float* ux, const float* uy,
                                                         const float* area, const uint8_t* mask, int64_t n,
                                                         double* out, void* stream) {
    mlbm::clear_error();
    // the node arrays may be NULL when there are no nodes
    if ((n > 0 && (!rho || !ux || !uy || !area)) || !out)
        return mlbm::set_error(MLBM_E_INVALID, "reduce_fields_device_noalloc: NULL pointer");
    if (n < 0 || n > mlbm_reduce_noalloc_max_nodes())
        return mlbm::set_error(MLBM_E_INVALID, "reduce_fields_device_noalloc: n must be in [0, 2^31 - 1] (got " +
                                                   std::to_string(n) + ")");
    static_assert(sizeof(g_reduce_partials) == 6 * sizeof(double) * mlbm::kReduceMaxBlocks, "scratch size");
    double* partials = nullptr;
    mlbm_status st = partials_on_current_device(&partials);
    if (st != MLBM_OK) return st;
    // every block writes all 6 of its partial sums before the final pass reads
    // them, so nothing in the shared scratch has to start at zero
    cudaError_t e = mlbm::launch_reduce_fields(rho, ux, uy, area, mask, n, partials, out,
                                               static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return mlbm::set_error(MLBM_E_CUDA, std::string("reduce_fields_device_noalloc: launch: ") +
                                                cudaGetErrorString(e));
    return MLBM_OK;
}
