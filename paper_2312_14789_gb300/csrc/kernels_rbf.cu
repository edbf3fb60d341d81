// Step kernels on RBF-FD stencils (Sec. 2.2; BGK and tau = 1) and their
// launchers.  The node code is the least-squares one with per-direction
// weight rows (step_node.cuh).
#include "device_common.cuh"
#include "kernels.h"
#include "launch_util.cuh"
#include "step_node.cuh"

namespace mlbm {
namespace dev {

template <int KQ, int MINB, bool SPEC = false>
__global__ void __launch_bounds__(256, MINB) bgk_step_rbf(Stencil S, const float4* __restrict__ f8in,
                                                          const float* __restrict__ f0in, float4* __restrict__ f8out,
                                                          float* __restrict__ f0out, Collide C) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S.n) return;
    bgk_node<KQ, 1, true, true, SPEC>(S, f8in, f0in, f8out, f0out, C, p, 0, 1u << (threadIdx.x & 31u));
}

template <int KQ, int MINB, bool SPEC = false>
__global__ void __launch_bounds__(256, MINB) bgk_step_rbf_persistent(Stencil S, const float4* __restrict__ f8in,
                                                                     const float* __restrict__ f0in,
                                                                     float4* __restrict__ f8out,
                                                                     float* __restrict__ f0out, Collide C, int dist) {
    constexpr int TN = 256;
    const int n_tiles = (S.n + TN - 1) / TN;
    const unsigned lane = threadIdx.x & 31u;
    if (threadIdx.x < 32)
        for (int d = 0; d < dist; ++d) prefetch_tile_rbf<KQ>(S, (blockIdx.x + d * gridDim.x) * TN, TN, lane);
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        if (threadIdx.x < 32) prefetch_tile_rbf<KQ>(S, (tile + dist * gridDim.x) * TN, TN, lane);
        const int p = tile * TN + threadIdx.x;
        if (p < S.n) bgk_node<KQ, 1, true, true, SPEC>(S, f8in, f0in, f8out, f0out, C, p, 0, 1u << lane);
    }
}

template <int KQ, int MINB>
__global__ void __launch_bounds__(256, MINB) tau1_step_rbf(Stencil S, const float4* __restrict__ in,
                                                           float4* __restrict__ out, Collide C) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S.n) return;
    tau1_node<KQ, 1, true>(S, in, out, C, p, 0, 1u << (threadIdx.x & 31u));
}

template <int KQ, int MINB>
__global__ void __launch_bounds__(256, MINB) tau1_step_rbf_persistent(Stencil S, const float4* __restrict__ in,
                                                                      float4* __restrict__ out, Collide C, int dist) {
    constexpr int TN = 256;
    const int n_tiles = (S.n + TN - 1) / TN;
    const unsigned lane = threadIdx.x & 31u;
    if (threadIdx.x < 32)
        for (int d = 0; d < dist; ++d) prefetch_tile_rbf<KQ>(S, (blockIdx.x + d * gridDim.x) * TN, TN, lane);
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        if (threadIdx.x < 32) prefetch_tile_rbf<KQ>(S, (tile + dist * gridDim.x) * TN, TN, lane);
        const int p = tile * TN + threadIdx.x;
        if (p < S.n) tau1_node<KQ, 1, true>(S, in, out, C, p, 0, 1u << lane);
    }
}

}  // namespace dev

// RBF-FD stencils: the per-direction weights of the node's own stencil or of
// the union of its departure points' stencils (up to K = 64)
cudaError_t launch_bgk_step_rbf(const dev::Stencil& S, const float4* f8in, const float* f0in, float4* f8out,
                                float* f0out, const dev::Collide& C, int variant, cudaStream_t st) {
    if (S.n == 0) return cudaSuccess;
    const int block = 256;
    // RBF-FD stencils: variants 10 and 12 map to the persistent kernel
    // (uncapped / 2 blocks per SM), 0 to the plain uncapped kernel, 20
    // and 21 to the plain capped and the persistent uncapped kernel with
    // the early index loads, the rest to the plain kernel capped for 2
    // blocks per SM
    if (variant == 20) {
        MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::bgk_step_rbf<KQC, 2, true><<<blocks_for(S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C)));
    } else if (variant == 21) {
        MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_rbf_persistent<KQC, 1, true>, 256, S.n, st, [&](int g) { dev::bgk_step_rbf_persistent<KQC, 1, true><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); })));
    } else if (variant == 10) {
        MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_rbf_persistent<KQC, 1>, 256, S.n, st, [&](int g) { dev::bgk_step_rbf_persistent<KQC, 1><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); })));
    } else if (variant == 12) {
        MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_rbf_persistent<KQC, 2>, 256, S.n, st, [&](int g) { dev::bgk_step_rbf_persistent<KQC, 2><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); })));
    } else if (variant == 0) {
        MLBM_DISPATCH_KQ_RBF(S.Kq, (dev::bgk_step_rbf<KQC, 1><<<blocks_for(S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C)));
    } else {
        MLBM_DISPATCH_KQ_RBF(S.Kq, (dev::bgk_step_rbf<KQC, 2><<<blocks_for(S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C)));
    }
    return cudaGetLastError();

}

cudaError_t launch_tau1_step_rbf(const dev::Stencil& S, const float4* in, float4* out, const dev::Collide& C,
                                 int variant, cudaStream_t st) {
    if (S.n == 0) return cudaSuccess;
    const int block = 256;
    // RBF-FD stencils: variants map as for the BGK step
    if (variant == 10) {
        MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::tau1_step_rbf_persistent<KQC, 1>, 256, S.n, st, [&](int g) { dev::tau1_step_rbf_persistent<KQC, 1><<<g, block, 0, st>>>(S, in, out, C, 1); })));
    } else if (variant == 12) {
        MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::tau1_step_rbf_persistent<KQC, 2>, 256, S.n, st, [&](int g) { dev::tau1_step_rbf_persistent<KQC, 2><<<g, block, 0, st>>>(S, in, out, C, 1); })));
    } else if (variant == 0) {
        MLBM_DISPATCH_KQ_RBF(S.Kq, (dev::tau1_step_rbf<KQC, 1><<<blocks_for(S.n, block), block, 0, st>>>(S, in, out, C)));
    } else {
        MLBM_DISPATCH_KQ_RBF(S.Kq, (dev::tau1_step_rbf<KQC, 2><<<blocks_for(S.n, block), block, 0, st>>>(S, in, out, C)));
    }
    return cudaGetLastError();

}

}  // namespace mlbm
