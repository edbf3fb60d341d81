// tau = 1 (MLBM1) step kernels on least-squares and Lagrange stencils (the
// node code is in step_node.cuh) and their launcher.
#include "device_common.cuh"
#include "kernels.h"
#include "launch_util.cuh"
#include "step_node.cuh"

namespace mlbm {
namespace dev {

template <int KQ, int LPN, int MINB, bool PDL = false>
__global__ void __launch_bounds__(256, MINB) tau1_step_kernel(Stencil S, const float4* __restrict__ in,
                                                              float4* __restrict__ out, Collide C) {
    if (PDL) {
        if (threadIdx.x < 32) prefetch_tile<KQ>(S, blockIdx.x * (256 / LPN), 256 / LPN, threadIdx.x & 31u);
        pdl_trigger();
        pdl_wait();
    }
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = tid / LPN;
    const int h = tid % LPN;
    if (p >= S.n) return;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned grp = LPN == 1 ? (1u << lane) : (3u << (lane & ~1u));
    tau1_node<KQ, LPN>(S, in, out, C, p, h, grp);
}

template <int KQ, int LPN, int MINB, bool PDL = false>
__global__ void __launch_bounds__(256, MINB) tau1_step_persistent(Stencil S, const float4* __restrict__ in,
                                                                  float4* __restrict__ out, Collide C, int dist) {
    constexpr int TN = 256 / LPN;
    const int n_tiles = (S.n + TN - 1) / TN;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned grp = LPN == 1 ? (1u << lane) : (3u << (lane & ~1u));
    const int h = threadIdx.x % LPN;
    if (threadIdx.x < 32)
        for (int d = 0; d < dist; ++d) prefetch_tile<KQ>(S, (blockIdx.x + d * gridDim.x) * TN, TN, lane);
    if (PDL) {
        pdl_trigger();
        pdl_wait();
    }
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        if (threadIdx.x < 32) prefetch_tile<KQ>(S, (tile + dist * gridDim.x) * TN, TN, lane);
        const int p = tile * TN + threadIdx.x / LPN;
        if (p < S.n) tau1_node<KQ, LPN>(S, in, out, C, p, h, grp);
    }
}

}  // namespace dev

cudaError_t launch_tau1_step(const dev::Stencil& S, const float4* in, float4* out, const dev::Collide& C, int variant,
                             cudaStream_t st) {
    if (S.n == 0) return cudaSuccess;
    const int block = 256;
    if (S.Wr) return launch_tau1_step_rbf(S, in, out, C, variant, st);
    switch (variant) {
        case 0: MLBM_DISPATCH_KQ(S.Kq, (dev::tau1_step_kernel<KQC, 1, 1><<<blocks_for(S.n, block), block, 0, st>>>(S, in, out, C))); break;
        case 1: MLBM_DISPATCH_KQ(S.Kq, (dev::tau1_step_kernel<KQC, 2, 1><<<blocks_for(2 * (int64_t)S.n, block), block, 0, st>>>(S, in, out, C))); break;
        case 2: MLBM_DISPATCH_KQ(S.Kq, (dev::tau1_step_kernel<KQC, 2, 3><<<blocks_for(2 * (int64_t)S.n, block), block, 0, st>>>(S, in, out, C))); break;
        case 3: MLBM_DISPATCH_KQ(S.Kq, (dev::tau1_step_kernel<KQC, 2, 4><<<blocks_for(2 * (int64_t)S.n, block), block, 0, st>>>(S, in, out, C))); break;
        case 8: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::tau1_step_persistent<KQC, 2, 3>, 128, S.n, st, [&](int g) { dev::tau1_step_persistent<KQC, 2, 3><<<g, block, 0, st>>>(S, in, out, C, 1); }))); break;
        case 9: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::tau1_step_persistent<KQC, 2, 3>, 128, S.n, st, [&](int g) { dev::tau1_step_persistent<KQC, 2, 3><<<g, block, 0, st>>>(S, in, out, C, 2); }))); break;
        case 10: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::tau1_step_persistent<KQC, 1, 1>, 256, S.n, st, [&](int g) { dev::tau1_step_persistent<KQC, 1, 1><<<g, block, 0, st>>>(S, in, out, C, 1); }))); break;
        case 11: MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::tau1_step_kernel<KQC, 1, 2><<<blocks_for(S.n, block), block, 0, st>>>(S, in, out, C))); break;
        case 12: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::tau1_step_persistent<KQC, 1, 2>, 256, S.n, st, [&](int g) { dev::tau1_step_persistent<KQC, 1, 2><<<g, block, 0, st>>>(S, in, out, C, 1); }))); break;
        case 13: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::tau1_step_persistent<KQC, 1, 3>, 256, S.n, st, [&](int g) { dev::tau1_step_persistent<KQC, 1, 3><<<g, block, 0, st>>>(S, in, out, C, 1); }))); break;
        case 25: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::tau1_step_persistent<KQC, 1, 2, true>, 256, S.n, st, [&](int g) { (void)launch_pdl(dev::tau1_step_persistent<KQC, 1, 2, true>, g, block, st, S, in, out, C, 1); }))); break;
        case 26: MLBM_DISPATCH_KQ_MAIN(S.Kq, ((void)launch_pdl(dev::tau1_step_kernel<KQC, 1, 2, true>, blocks_for(S.n, block), block, st, S, in, out, C))); break;
        case 14:
        case 15:
        case 16:
        case 17:
        case 18:
        case 19:
        case 20:
        case 21:
        case 22:
        case 23:
        case 24:  // the direction split, the link split, the early index loads, the staging and the other block sizes exist for the BGK state only
            MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::tau1_step_kernel<KQC, 1, 2><<<blocks_for(S.n, block), block, 0, st>>>(S, in, out, C))); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace mlbm
