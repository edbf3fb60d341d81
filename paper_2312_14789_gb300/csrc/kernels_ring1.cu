// Persistent step kernels of one lane per node whose stencil rows come from
// a shared-memory ring filled by bulk async copies (variants 27-29), and
// their launcher.
#include "device_common.cuh"
#include "kernels.h"
#include "launch_util.cuh"
#include "step_node.cuh"
#include "ring.cuh"

namespace mlbm {
namespace dev {

// ------------------------------------- one lane per node, bulk-copy ring
// Variants 27-29.  Persistent CTAs of TN consumer threads (one node each) and
// one producer warp that streams the tiles' stencil rows into a STAGES-deep
// shared-memory ring (ring.cuh).  The consumer runs the same node code as the
// plain kernels with its rows read from shared memory, so the loads left on
// its own path are the neighbour gathers; the stencil rows, ~86% of the
// bytes, are in flight ahead of it without holding registers.
template <int KQ, int TN, int STAGES, int MINB>
__global__ void __launch_bounds__(TN + 32, MINB)
    bgk_step_ring1(Stencil S, const float4* __restrict__ f8in, const float* __restrict__ f0in,
                   float4* __restrict__ f8out, float* __restrict__ f0out, Collide C0, int n_tiles,
                   int* __restrict__ err, const Wait W) {
    using L = Tile<KQ, TN, STAGES>;
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::kBar);
    uint64_t* empty = full + STAGES;
    const int warp = threadIdx.x >> 5;
    const unsigned lane = threadIdx.x & 31u;
    init_ring(full, empty, STAGES, TN / 32);
    if (warp == TN / 32) {
        produce<KQ, TN, STAGES>(S, smem, full, empty, n_tiles, err, W);
        return;
    }
    const int t = threadIdx.x;
    int it = 0;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
        const int s = it % STAGES;
        // the warp leaves together if any lane's wait ran out
        if (!__all_sync(0xffffffffu, mbar_wait(&full[s], (it / STAGES) & 1, W.budget_ns))) {
            if (lane == 0) atomicExch(err, 2);
            return;
        }
        const uint8_t* st = smem + s * L::kStage;
        const SmemRows R{reinterpret_cast<const float4*>(st), reinterpret_cast<const int4*>(st + L::kM),
                         st + L::kM + L::kI, t, TN};
        const int p = tile * TN + t;
        if (p < S.n)
            bgk_node<KQ, 1, true, false, false, SmemRows>(S, f8in, f0in, f8out, f0out, C0, p, 0, 1u << lane, &R);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

template <int KQ, int TN, int STAGES, int MINB>
__global__ void __launch_bounds__(TN + 32, MINB)
    tau1_step_ring1(Stencil S, const float4* __restrict__ in, float4* __restrict__ out, Collide C0, int n_tiles,
                    int* __restrict__ err, const Wait W) {
    using L = Tile<KQ, TN, STAGES>;
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::kBar);
    uint64_t* empty = full + STAGES;
    const int warp = threadIdx.x >> 5;
    const unsigned lane = threadIdx.x & 31u;
    init_ring(full, empty, STAGES, TN / 32);
    if (warp == TN / 32) {
        produce<KQ, TN, STAGES>(S, smem, full, empty, n_tiles, err, W);
        return;
    }
    const int t = threadIdx.x;
    int it = 0;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
        const int s = it % STAGES;
        if (!__all_sync(0xffffffffu, mbar_wait(&full[s], (it / STAGES) & 1, W.budget_ns))) {
            if (lane == 0) atomicExch(err, 2);
            return;
        }
        const uint8_t* st = smem + s * L::kStage;
        const SmemRows R{reinterpret_cast<const float4*>(st), reinterpret_cast<const int4*>(st + L::kM),
                         st + L::kM + L::kI, t, TN};
        const int p = tile * TN + t;
        if (p < S.n) tau1_node<KQ, 1, false, SmemRows>(S, in, out, C0, p, 0, 1u << lane, &R);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

}  // namespace dev

namespace {

template <int KQ, int TN, int STAGES, int MINB>
cudaError_t run_ring1(int model, const dev::Stencil& S, const float4* a8, const float* a0, float4* b8, float* b0,
                      const float4* ra, float4* rb, const dev::Collide& C, int* err, const dev::Wait& W,
                      cudaStream_t st) {
    using L = dev::Tile<KQ, TN, STAGES>;
    static_assert(L::kBytes <= 232448, "tile ring exceeds shared memory");
    const void* fn = model == 0 ? (const void*)dev::bgk_step_ring1<KQ, TN, STAGES, MINB>
                                : (const void*)dev::tau1_step_ring1<KQ, TN, STAGES, MINB>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes);
    if (e != cudaSuccess) return e;
    int dev_id = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev_id);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TN + 32, L::kBytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int n_tiles = (S.n + TN - 1) / TN;
    const int grid = std::max(1, std::min(n_tiles, sms * per_sm));
    if (model == 0)
        dev::bgk_step_ring1<KQ, TN, STAGES, MINB><<<grid, TN + 32, L::kBytes, st>>>(S, a8, a0, b8, b0, C, n_tiles, err, W);
    else
        dev::tau1_step_ring1<KQ, TN, STAGES, MINB><<<grid, TN + 32, L::kBytes, st>>>(S, ra, rb, C, n_tiles, err, W);
    return cudaGetLastError();
}

template <int KQ>
cudaError_t run_ring1_variant(int variant, int model, const dev::Stencil& S, const float4* a8, const float* a0,
                              float4* b8, float* b0, const float4* ra, float4* rb, const dev::Collide& C, int* err,
                              const dev::Wait& W, cudaStream_t st) {
    switch (variant) {
        case 27: return run_ring1<KQ, 128, 2, 2>(model, S, a8, a0, b8, b0, ra, rb, C, err, W, st);
        case 28: return run_ring1<KQ, 64, 2, 3>(model, S, a8, a0, b8, b0, ra, rb, C, err, W, st);
        case 29: return run_ring1<KQ, 64, 3, 2>(model, S, a8, a0, b8, b0, ra, rb, C, err, W, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_step_ring1(int variant, int model, const dev::Stencil& S, const float4* f8in, const float* f0in,
                              float4* f8out, float* f0out, const float4* rin, float4* rout, const dev::Collide& C,
                              int* err, const dev::Wait& W, cudaStream_t st) {
    if (S.n == 0) return cudaSuccess;
    switch (S.Kq) {
        case 3: return run_ring1_variant<3>(variant, model, S, f8in, f0in, f8out, f0out, rin, rout, C, err, W, st);
        case 4: return run_ring1_variant<4>(variant, model, S, f8in, f0in, f8out, f0out, rin, rout, C, err, W, st);
        case 6: return run_ring1_variant<6>(variant, model, S, f8in, f0in, f8out, f0out, rin, rout, C, err, W, st);
        case 8: return run_ring1_variant<8>(variant, model, S, f8in, f0in, f8out, f0out, rin, rout, C, err, W, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mlbm
