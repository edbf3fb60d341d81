// Allocation-free form of mlbm_reduce_fields_device.
//
// The two-pass FP64 reduction needs a scratch array of per-block partial
// sums.  Here that scratch is a file-scope device array, so the caller passes
// only its inputs and the 6-double output and nothing is allocated on any call.
// Host code cannot use the array's name as a device address (it is a host-side
// stand-in for the symbol); the device address is looked up once per device
// with cudaGetSymbolAddress and cached.
#include <mutex>
#include <string>

#include "kernels.h"
#include "mlbm_internal.h"

namespace {

constexpr int kMaxDevices = 64;

// 6 partial sums per block, at most kReduceMaxBlocks blocks for any n
static __device__ __align__(256) double g_reduce_partials[6 * mlbm::kReduceMaxBlocks];

std::mutex g_setup_mu;
double* g_partials_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up on the
// first call for that device, with that device current).
mlbm_status partials_on_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return mlbm::set_error(MLBM_E_CUDA, std::string("reduce_fields_device_noalloc: cudaGetDevice: ") +
                                                cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return mlbm::set_error(MLBM_E_INVALID, "reduce_fields_device_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_partials_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_reduce_partials);
        if (e != cudaSuccess || !ptr)
            return mlbm::set_error(MLBM_E_CUDA, std::string("reduce_fields_device_noalloc: cudaGetSymbolAddress: ") +
                                                    cudaGetErrorString(e));
        g_partials_ptr[dev] = static_cast<double*>(ptr);
    }
    *out = g_partials_ptr[dev];
    return MLBM_OK;
}

}  // namespace

extern "C" int64_t mlbm_reduce_noalloc_max_nodes(void) { return (int64_t)INT32_MAX; }

extern "C" mlbm_status mlbm_reduce_fields_device_noalloc(const float* rho, const float* ux, const float* uy,
                                                         const float* area, const uint8_t* mask, int64_t n,
                                                         double* out, void* stream) {
    mlbm::clear_error();
    if (!rho || !ux || !uy || !area || !out)
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
