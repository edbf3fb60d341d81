// BGK/TRT step kernels on least-squares and Lagrange stencils (variants
// 8-13, 20-21, 23-26, K = 12, 16, 24, 32; the node code is in
// step_node.cuh) and their launcher; variants 0-3 (any K) are in
// kernels_bgk_generic.cu, 14-19 and 22 in kernels_bgk_alt.cu.
#include "device_common.cuh"
#include "kernels.h"
#include "launch_util.cuh"
#include "step_node.cuh"

namespace mlbm {

// the BGK step of variant v (the list is in mlbm_set_kernel_variant's notes)
cudaError_t launch_bgk_step(const dev::Stencil& S, const float4* f8in, const float* f0in, float4* f8out,
                            float* f0out, const dev::Collide& C, int variant, cudaStream_t st) {
    if (S.n == 0) return cudaSuccess;
    const int block = 256;
    if (S.Wr) return launch_bgk_step_rbf(S, f8in, f0in, f8out, f0out, C, variant, st);
    switch (variant) {
        case 0: case 1: case 2: case 3:
            return launch_bgk_step_generic(S, f8in, f0in, f8out, f0out, C, variant, st);
        case 8: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_persistent<KQC, 2, 3>, 128, S.n, st, [&](int g) { dev::bgk_step_persistent<KQC, 2, 3><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); }))); break;
        case 9: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_persistent<KQC, 2, 3>, 128, S.n, st, [&](int g) { dev::bgk_step_persistent<KQC, 2, 3><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 2); }))); break;
        case 10: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_persistent<KQC, 1, 1>, 256, S.n, st, [&](int g) { dev::bgk_step_persistent<KQC, 1, 1><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); }))); break;
        case 11: MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::bgk_step_kernel<KQC, 1, 2><<<blocks_for(S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        case 12: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_persistent<KQC, 1, 2>, 256, S.n, st, [&](int g) { dev::bgk_step_persistent<KQC, 1, 2><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); }))); break;
        case 13: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_persistent<KQC, 1, 3>, 256, S.n, st, [&](int g) { dev::bgk_step_persistent<KQC, 1, 3><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); }))); break;
        case 14: case 15: case 16: case 17: case 18: case 19: case 22:
            return launch_bgk_step_alt(S, f8in, f0in, f8out, f0out, C, variant, st);
        case 25: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_persistent<KQC, 1, 2, false, 256, true>, 256, S.n, st, [&](int g) { (void)launch_pdl(dev::bgk_step_persistent<KQC, 1, 2, false, 256, true>, g, block, st, S, f8in, f0in, f8out, f0out, C, 1); }))); break;
        case 26: MLBM_DISPATCH_KQ_MAIN(S.Kq, ((void)launch_pdl(dev::bgk_step_kernel<KQC, 1, 2, false, 256, true>, blocks_for(S.n, block), block, st, S, f8in, f0in, f8out, f0out, C))); break;
        case 23: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_persistent<KQC, 1, 4, false, 128>, 128, S.n, st, [&](int g) { dev::bgk_step_persistent<KQC, 1, 4, false, 128><<<g, 128, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); }, 0, 128))); break;
        case 24: MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::bgk_step_kernel<KQC, 1, 1, false, 512><<<blocks_for(S.n, 512), 512, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        case 20: MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::bgk_step_kernel<KQC, 1, 2, true><<<blocks_for(S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        case 21: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_persistent<KQC, 1, 1, true>, 256, S.n, st, [&](int g) { dev::bgk_step_persistent<KQC, 1, 1, true><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); }))); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace mlbm
