// Bulk-copy ring shared by the pipelined step kernels (kernels_tma.cu: four
// lanes per node; kernels.cu: one lane per node).  A producer warp streams
// each tile's stencil rows (least-squares matrix, neighbour indices, meta
// bytes: contiguous TN x 16-byte chunks of the interleaved layout) with
// cp.async.bulk into a ring of STAGES shared-memory buffers guarded by
// mbarriers; consumer warps wait for a stage, read it, and release it.
// Every wait is bounded by a time budget (Wait); see kernels_tma.cu.
#pragma once

#include <cstdint>

#include "device_common.cuh"

namespace mlbm {
namespace dev {

__device__ __forceinline__ uint32_t saddr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(b)), "r"(parity)
        : "memory");
    return ok;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// wait for the phase of the given parity to complete; false once budget_ns
// nanoseconds have passed without it
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, unsigned long long budget_ns) {
    if (mbar_try_wait(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(b, parity))
        if (global_ns() - t0 > budget_ns) return false;
    return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     saddr(dst)),
                 "l"(src), "r"(bytes), "r"(saddr(bar))
                 : "memory");
}


template <int KQ, int TN, int STAGES>
struct Tile {
    static constexpr int kM = 6 * KQ * TN * 16;
    static constexpr int kI = KQ * TN * 16;
    static constexpr int kMeta = (TN + 15) / 16 * 16;
    static constexpr int kStage = kM + kI + kMeta;
    static constexpr int kBar = STAGES * kStage;
    static constexpr int kBytes = kBar + 2 * STAGES * 8;
    static constexpr int kConsumers = TN * 4;
    static constexpr int kThreads = kConsumers + 32;
};

// producer warp: fill the ring for this CTA's tiles.  Lane 0 waits for a
// free stage and arms its barrier with the byte count; then the 32 lanes issue
// the tile's 7K/4 + 1 bulk copies in parallel.
template <int KQ, int TN, int STAGES>
__device__ __forceinline__ void produce(const Stencil& S, uint8_t* smem, uint64_t* full, uint64_t* empty,
                                       int n_tiles, int* err, const Wait W) {
    using L = Tile<KQ, TN, STAGES>;
    const unsigned lane = threadIdx.x & 31u;
    constexpr int kCopies = 7 * KQ + 1;
    // test switch: block 0 issues nothing for its first tile (no arrival, no
    // copies), so the consumers' bounded wait for that tile runs out
    const bool withhold = W.withhold && blockIdx.x == 0;
    int it = 0;
    int ok = 1;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
        const int s = it % STAGES;
        const bool skip = withhold && it == 0;
        if (lane == 0) {
            if (it >= STAGES && !mbar_wait(&empty[s], ((it / STAGES) - 1) & 1, W.budget_ns)) {
                atomicExch(err, 1);
                ok = 0;
            } else if (!skip) {
                mbar_expect_tx(&full[s], L::kStage);
            }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        if (skip) continue;
        uint8_t* st = smem + s * L::kStage;
        const size_t base = (size_t)tile * TN;
        for (int c = lane; c < kCopies; c += 32) {
            if (c < 6 * KQ)
                bulk_g2s(st + c * TN * 16, S.M + (size_t)c * S.n_pad + base, TN * 16, &full[s]);
            else if (c < 7 * KQ)
                bulk_g2s(st + L::kM + (c - 6 * KQ) * TN * 16, S.idx + (size_t)(c - 6 * KQ) * S.n_pad + base,
                         TN * 16, &full[s]);
            else
                bulk_g2s(st + L::kM + L::kI, S.meta + base, L::kMeta, &full[s]);
        }
        __syncwarp();
    }
    // drain: do not leave while copies may still be landing in this CTA's
    // shared memory (bounded; the consumers normally have waited already).
    // Every tile of the last STAGES is waited for, even after one wait ran
    // out, so a late copy of one tile does not hide the others.
    if (lane == 0) {
        const int issued = it;
        for (int u = (issued > STAGES ? issued - STAGES : 0); u < issued; ++u) {
            if (withhold && u == 0) continue;  // nothing was issued for it
            if (!mbar_wait(&full[u % STAGES], (u / STAGES) & 1, W.budget_ns)) atomicExch(err, 3);
        }
    }
}

__device__ __forceinline__ void init_ring(uint64_t* full, uint64_t* empty, int stages, int consumer_warps) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], consumer_warps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
}

}  // namespace dev
}  // namespace mlbm
