// BGK/TRT step variants 0-3 on least-squares and Lagrange stencils of any K
// (a multiple of 4 up to 32): one or two lanes per node, with and without a
// register cap.
#include "device_common.cuh"
#include "kernels.h"
#include "launch_util.cuh"
#include "step_node.cuh"

namespace mlbm {

// variant v: lanes per node and minimum resident blocks (register cap)
//   0: 1 lane, no cap   1: 2 lanes, no cap   2: 2 lanes, >= 3 blocks of 256
//   3: 2 lanes, >= 4 blocks of 256
cudaError_t launch_bgk_step_generic(const dev::Stencil& S, const float4* f8in, const float* f0in, float4* f8out,
                                    float* f0out, const dev::Collide& C, int variant, cudaStream_t st) {
    if (S.n == 0) return cudaSuccess;
    const int block = 256;
    switch (variant) {
        case 0: MLBM_DISPATCH_KQ(S.Kq, (dev::bgk_step_kernel<KQC, 1, 1><<<blocks_for(S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        case 1: MLBM_DISPATCH_KQ(S.Kq, (dev::bgk_step_kernel<KQC, 2, 1><<<blocks_for(2 * (int64_t)S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        case 2: MLBM_DISPATCH_KQ(S.Kq, (dev::bgk_step_kernel<KQC, 2, 3><<<blocks_for(2 * (int64_t)S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        case 3: MLBM_DISPATCH_KQ(S.Kq, (dev::bgk_step_kernel<KQC, 2, 4><<<blocks_for(2 * (int64_t)S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace mlbm
