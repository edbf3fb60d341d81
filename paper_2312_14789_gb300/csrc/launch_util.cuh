// Launch helpers shared by the step kernel translation units: the K/4
// dispatch switches, the persistent grid size and the programmatic dependent
// launch.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

namespace mlbm {
namespace {
inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }
}  // namespace

#define MLBM_DISPATCH_KQ(KQ, ...)                        \
    switch (KQ) {                                        \
        case 2: { constexpr int KQC = 2; __VA_ARGS__; } break; \
        case 3: { constexpr int KQC = 3; __VA_ARGS__; } break; \
        case 4: { constexpr int KQC = 4; __VA_ARGS__; } break; \
        case 5: { constexpr int KQC = 5; __VA_ARGS__; } break; \
        case 6: { constexpr int KQC = 6; __VA_ARGS__; } break; \
        case 7: { constexpr int KQC = 7; __VA_ARGS__; } break; \
        case 8: { constexpr int KQC = 8; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;           \
    }

// the tuned variants (4 and up) are instantiated for K = 12, 16, 24, 32 only
#define MLBM_DISPATCH_KQ_MAIN(KQ, ...)                   \
    switch (KQ) {                                        \
        case 3: { constexpr int KQC = 3; __VA_ARGS__; } break; \
        case 4: { constexpr int KQC = 4; __VA_ARGS__; } break; \
        case 6: { constexpr int KQC = 6; __VA_ARGS__; } break; \
        case 8: { constexpr int KQC = 8; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;           \
    }

// RBF-FD stencils per Lagrangian point are up to 64 wide (the union of the
// directions' stencils); the plain RBF-FD kernels are also instantiated for
// K = 48 and 64
#define MLBM_DISPATCH_KQ_RBF(KQ, ...)                    \
    switch (KQ) {                                        \
        case 3: { constexpr int KQC = 3; __VA_ARGS__; } break; \
        case 4: { constexpr int KQC = 4; __VA_ARGS__; } break; \
        case 6: { constexpr int KQC = 6; __VA_ARGS__; } break; \
        case 8: { constexpr int KQC = 8; __VA_ARGS__; } break; \
        case 12: { constexpr int KQC = 12; __VA_ARGS__; } break; \
        case 16: { constexpr int KQC = 16; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;           \
    }

// grid of exactly the resident blocks (occupancy API), at most one per tile
template <class F>
cudaError_t run_persistent(const void* fn, int tile_nodes, int n, cudaStream_t, F launch, size_t smem = 0,
                           int threads = 256) {
    int dev_id = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev_id);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (e != cudaSuccess) return e;
    const int tiles = (n + tile_nodes - 1) / tile_nodes;
    const int grid = std::max(1, std::min(tiles, sms * std::max(per_sm, 1)));
    launch(grid);
    return cudaSuccess;
}

// launch with programmatic stream serialization (the kernel waits for its
// predecessor itself, see pdl_wait)
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace mlbm
