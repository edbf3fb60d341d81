// Device side of the run to steady state of a batch: holding the samples
// that have converged (see run_steady in context.cu).
#include <cstdint>

#include "kernels.h"

namespace mlbm {
namespace dev {

// tau = 1: a node of the equilibrium kind copies its stored record (rho - 1,
// u, v, 0) to the output every step; making every node of a sample such a
// node, with its current state as the record, holds the sample's state fixed
__global__ void freeze_tau1(int m, uint8_t* __restrict__ meta, float4* __restrict__ eqv,
                            const float4* __restrict__ state) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    const uint8_t t = meta[p];
    if ((t & 3) != 2) {
        eqv[p] = state[p];
        meta[p] = (uint8_t)((t & ~3u) | 2u);
    }
}

}  // namespace dev

cudaError_t launch_freeze_tau1(int m, uint8_t* meta, float4* eqv, const float4* state, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    dev::freeze_tau1<<<(m + 255) / 256, 256, 0, st>>>(m, meta, eqv, state);
    return cudaGetLastError();
}

}  // namespace mlbm
