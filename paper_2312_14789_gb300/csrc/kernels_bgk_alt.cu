// BGK/TRT step kernels of the alternative node layouts: two lanes per node
// split by direction half (variants 14-17), the pass without links followed
// by the link nodes (18-19), and staged neighbourhoods (22); their launcher.
#include "device_common.cuh"
#include "kernels.h"
#include "launch_util.cuh"
#include "step_node.cuh"

namespace mlbm {
namespace dev {

template <int KQ, int MINB, int UQ>
__global__ void __launch_bounds__(256, MINB) bgk_split_kernel(Stencil S, const float4* __restrict__ f8in,
                                                              const float* __restrict__ f0in,
                                                              float4* __restrict__ f8out, float* __restrict__ f0out,
                                                              Collide C) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = tid >> 1;
    if (p >= S.n) return;
    const unsigned lane = threadIdx.x & 31u;
    bgk_node_split<KQ, UQ>(S, f8in, f0in, f8out, f0out, C, p, tid & 1, 3u << (lane & ~1u));
}

// Split form: the persistent pass without the bounce-back code (fewer
// registers, more resident warps), then one thread per node with links
// recomputes that node completely and overwrites its output.
template <int KQ, int MINB>
__global__ void __launch_bounds__(256, MINB) bgk_step_nolink(Stencil S, const float4* __restrict__ f8in,
                                                             const float* __restrict__ f0in,
                                                             float4* __restrict__ f8out, float* __restrict__ f0out,
                                                             Collide C, int dist) {
    constexpr int TN = 256;
    const int n_tiles = (S.n + TN - 1) / TN;
    const unsigned lane = threadIdx.x & 31u;
    if (threadIdx.x < 32)
        for (int d = 0; d < dist; ++d) prefetch_tile<KQ>(S, (blockIdx.x + d * gridDim.x) * TN, TN, lane);
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        if (threadIdx.x < 32) prefetch_tile<KQ>(S, (tile + dist * gridDim.x) * TN, TN, lane);
        const int p = tile * TN + threadIdx.x;
        if (p < S.n) bgk_node<KQ, 1, false>(S, f8in, f0in, f8out, f0out, C, p, 0, 1u << lane);
    }
}

// Second pass of the split form: a group of 16 lanes per node with links.
// Lane r takes the stencil members j = r, r + 16, ...: it gathers a member's
// eight populations once and adds its share both to the departure-point
// values (stored departure basis) and, for interpolated bounce-back, to the
// fit of each reflected population at its link point x + (1 - 2q) s e_k
// (unbasis of the member's matrix column, evaluated at that point), so no
// population is gathered twice.  The group sums its partials with shuffles;
// lane 0 applies the overrides, collides and writes.  A Lagrange-kind node
// with links is recomputed by lane 0 alone.
template <int KQ>
__global__ void __launch_bounds__(128) bgk_link_nodes(Stencil S, const float4* __restrict__ f8in,
                                                      const float* __restrict__ f0in, float4* __restrict__ f8out,
                                                      float* __restrict__ f0out, Collide C0) {
    const int e = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 4);
    if (e >= S.n_link_nodes) return;  // the same for the whole group
    const unsigned lane = threadIdx.x & 31u;
    const int r = (int)(lane & 15u);
    const unsigned gmask = 0xffffu << (lane & 16u);
    const int p = S.link_nodes[e];
    const uint8_t meta = S.meta[p];
    if ((meta & 3) != 0) {
        if (r == 0) bgk_node<KQ, 1, true>(S, f8in, f0in, f8out, f0out, C0, p, 0, 1u << lane);
        return;
    }
    const LinkRec L = S.links[S.link_slot[p]];
    const bool interp = S.bb_mode != 0;
    const float4 oa = __ldg(f8in + 2 * (size_t)p);
    const float4 ob = __ldg(f8in + 2 * (size_t)p + 1);
    const float own[8] = {oa.x, oa.y, oa.z, oa.w, ob.x, ob.y, ob.z, ob.w};
    float acc[8], lk[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = lk[k] = 0.f;
    for (int j = r; j < 4 * KQ; j += 16) {
        const int q = j >> 2, c = j & 3;
        const int id = reinterpret_cast<const int*>(S.idx + (size_t)q * S.n_pad + p)[c];
        float t[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) t[a] = reinterpret_cast<const float*>(S.M + (size_t)(a * KQ + q) * S.n_pad + p)[c];
        const float4 ra = __ldg(f8in + 2 * (size_t)id);
        const float4 rb = __ldg(f8in + 2 * (size_t)id + 1);
        const float d[8] = {ra.x - oa.x, ra.y - oa.y, ra.z - oa.z, ra.w - oa.w,
                            rb.x - ob.x, rb.y - ob.y, rb.z - ob.z, rb.w - ob.w};
        wls_acc_diff(d[0], d[1], d[2], d[3], d[4], d[5], d[6], d[7], t[0], t[1], t[2], t[3], t[4], t[5], acc);
        if (interp) {
            float mm[6];
            unbasis(t, mm);
#pragma unroll
            for (int k = 1; k < 9; ++k) {
                if (!((L.mask >> k) & 1u)) continue;
                float pb[6];
                basis_at(k, L.t[k - 1], pb);
                float w = 0.f;
#pragma unroll
                for (int a = 0; a < 6; ++a) w = fmaf(pb[a], mm[a], w);
                lk[k - 1] = fmaf(w, d[opp_of(k) - 1], lk[k - 1]);
            }
        }
    }
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            acc[k] += __shfl_xor_sync(gmask, acc[k], off, 16);
            lk[k] += __shfl_xor_sync(gmask, lk[k], off, 16);
        }
    }
    if (r != 0) return;
    float g[9];
    g[0] = f0in[p];
#pragma unroll
    for (int k = 1; k < 9; ++k) {
        const int kp = opp_of(k);
        if ((L.mask >> k) & 1u)
            g[k] = interp ? own[kp - 1] + lk[k - 1] : own[kp - 1];
        else
            g[k] = own[k - 1] + acc[k - 1];
    }
    const Collide C = collide_of(S, C0, p);
    collide_part<1>(g, C, 0);
    f8out[2 * (size_t)p] = make_float4(g[1], g[2], g[3], g[4]);
    f8out[2 * (size_t)p + 1] = make_float4(g[5], g[6], g[7], g[8]);
    f0out[p] = g[0];
}

// ---------------------------------------------- staged neighbourhoods (22)
// Persistent blocks walk the node tiles.  A tile's neighbourhood (the sorted
// union of its least-squares nodes' stencil members, listed on the host) is
// copied into shared memory by cp.async, 32 bytes per member, one tile ahead
// of the tile being computed (two buffers); the nodes then gather from shared
// memory through 16-bit local indices, which also halves the index bytes.
// Nodes of other kinds and nodes with bounce-back links take the global path.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int KQ>
__device__ __forceinline__ void prefetch_tile_staged(const Stencil& S, int tile, int n_tiles, unsigned lane) {
    if (tile >= n_tiles) return;
    const int base = tile * kStageTile;
    const int nodes = min(kStageTile, S.n_pad - base);
    for (int c = (int)lane; c < 7 * KQ + 2; c += 32) {
        if (c < 6 * KQ)
            prefetch_l2(S.M + (size_t)c * S.n_pad + base, (uint32_t)nodes * 16u);
        else if (c < 7 * KQ)
            prefetch_l2(S.lidx + (size_t)(c - 6 * KQ) * S.n_pad + base, (uint32_t)nodes * 8u);
        else if (c == 7 * KQ)
            prefetch_l2(S.meta + base, (uint32_t)((nodes + 15) / 16 * 16));
        else {
            // the member list, widened to 16-byte bounds (the list is padded)
            const int a0 = __ldg(S.stage_off + tile) & ~3, a1 = (__ldg(S.stage_off + tile + 1) + 3) & ~3;
            if (a1 > a0) prefetch_l2(S.stage_ids + a0, (uint32_t)(a1 - a0) * 4u);
        }
    }
}

__device__ __forceinline__ void stage_tile(const Stencil& S, const float4* __restrict__ f8in, float4* buf, int tile,
                                           int n_tiles) {
    if (tile < n_tiles) {
        const int a0 = __ldg(S.stage_off + tile), a1 = __ldg(S.stage_off + tile + 1);
        for (int i = a0 + (int)threadIdx.x; i < a1; i += (int)blockDim.x) {
            const int id = __ldg(S.stage_ids + i);
            cp_async16(buf + 2 * (i - a0), f8in + 2 * (size_t)id);
            cp_async16(buf + 2 * (i - a0) + 1, f8in + 2 * (size_t)id + 1);
        }
    }
    cp_async_commit();  // an empty group past the last tile keeps the wait counts uniform
}

template <int KQ>
__device__ __forceinline__ void staged_node(const Stencil& S, const float4* nb, const float4* __restrict__ f8in,
                                            const float* __restrict__ f0in, float4* __restrict__ f8out,
                                            float* __restrict__ f0out, const Collide& C0, int p) {
    const uint8_t meta = S.meta[p];
    if ((meta & 7) != 0) {
        bgk_node<KQ, 1, true>(S, f8in, f0in, f8out, f0out, C0, p, 0, 1u << (threadIdx.x & 31u));
        return;
    }
    const Collide C = collide_of(S, C0, p);
    const float4 oa = __ldg(f8in + 2 * (size_t)p);
    const float4 ob = __ldg(f8in + 2 * (size_t)p + 1);
    ushort4 lv[KQ];
#pragma unroll
    for (int q = 0; q < KQ; ++q) lv[q] = __ldcs(S.lidx + (size_t)q * S.n_pad + p);
    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.f;
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
        float4 m[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) m[a] = ld_stream(S.M + (size_t)(a * KQ + q) * S.n_pad + p);
        const float* mc = reinterpret_cast<const float*>(m);
        const int l[4] = {lv[q].x, lv[q].y, lv[q].z, lv[q].w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float4 ra = nb[2 * l[c]];
            const float4 rb = nb[2 * l[c] + 1];
            wls_acc_diff(ra.x - oa.x, ra.y - oa.y, ra.z - oa.z, ra.w - oa.w, rb.x - ob.x, rb.y - ob.y, rb.z - ob.z,
                         rb.w - ob.w, mc[c], mc[4 + c], mc[8 + c], mc[12 + c], mc[16 + c], mc[20 + c], acc);
        }
    }
    const float own[8] = {oa.x, oa.y, oa.z, oa.w, ob.x, ob.y, ob.z, ob.w};
    float g[9];
    g[0] = f0in[p];
#pragma unroll
    for (int k = 1; k < 9; ++k) g[k] = acc[k - 1] + own[k - 1];
    collide_part<1>(g, C, 0);
    f8out[2 * (size_t)p] = make_float4(g[1], g[2], g[3], g[4]);
    f0out[p] = g[0];
    f8out[2 * (size_t)p + 1] = make_float4(g[5], g[6], g[7], g[8]);
}

template <int KQ>
__global__ void __launch_bounds__(256, 2) bgk_step_staged(Stencil S, const float4* __restrict__ f8in,
                                                          const float* __restrict__ f0in, float4* __restrict__ f8out,
                                                          float* __restrict__ f0out, Collide C) {
    extern __shared__ float4 nbuf[];  // two buffers of 2 * stage_max float4
    const int n_tiles = (S.n + kStageTile - 1) / kStageTile;
    const unsigned lane = threadIdx.x & 31u;
    float4* const buf0 = nbuf;
    float4* const buf1 = nbuf + 2 * (size_t)S.stage_max;
    if (threadIdx.x < 32) prefetch_tile_staged<KQ>(S, blockIdx.x, n_tiles, lane);
    stage_tile(S, f8in, buf0, blockIdx.x, n_tiles);
    int it = 0;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
        if (threadIdx.x < 32) prefetch_tile_staged<KQ>(S, tile + gridDim.x, n_tiles, lane);
        stage_tile(S, f8in, (it & 1) ? buf0 : buf1, tile + gridDim.x, n_tiles);
        cp_async_wait<1>();  // this thread's copies of the current tile have landed
        __syncthreads();     // and every thread's
        const int p = tile * kStageTile + threadIdx.x;
        if (p < S.n) staged_node<KQ>(S, (it & 1) ? buf1 : buf0, f8in, f0in, f8out, f0out, C, p);
        __syncthreads();  // the buffer is free for the tile after next
    }
    cp_async_wait<0>();
}

// RBF-FD stencils: one lane per node, the per-direction weights streamed
// instead of the least-squares matrix; plain grid or persistent blocks that
// prefetch later tiles' weight, index and meta rows into L2.
template <int KQ, int MINB, int UQ>
__global__ void __launch_bounds__(256, MINB) bgk_split_persistent(Stencil S, const float4* __restrict__ f8in,
                                                                  const float* __restrict__ f0in,
                                                                  float4* __restrict__ f8out,
                                                                  float* __restrict__ f0out, Collide C, int dist) {
    constexpr int TN = 128;
    const int n_tiles = (S.n + TN - 1) / TN;
    const unsigned lane = threadIdx.x & 31u;
    if (threadIdx.x < 32)
        for (int d = 0; d < dist; ++d) prefetch_tile<KQ>(S, (blockIdx.x + d * gridDim.x) * TN, TN, lane);
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        if (threadIdx.x < 32) prefetch_tile<KQ>(S, (tile + dist * gridDim.x) * TN, TN, lane);
        const int p = tile * TN + (threadIdx.x >> 1);
        if (p < S.n) bgk_node_split<KQ, UQ>(S, f8in, f0in, f8out, f0out, C, p, threadIdx.x & 1, 3u << (lane & ~1u));
    }
}

// RBF = true (one lane per node): the least-squares-kind nodes take each
// direction's (dr, u, v) increment from their stored RBF-FD weights
}  // namespace dev

// allow the staged kernel the dynamic shared memory of its two buffers
cudaError_t prepare_staged_step(int Kq, int stage_max) {
    const int smem = 4 * stage_max * (int)sizeof(float4);
    MLBM_DISPATCH_KQ_MAIN(Kq, (cudaFuncSetAttribute((const void*)dev::bgk_step_staged<KQC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)));
    return cudaGetLastError();
}

cudaError_t launch_bgk_step_alt(const dev::Stencil& S, const float4* f8in, const float* f0in, float4* f8out,
                                float* f0out, const dev::Collide& C, int variant, cudaStream_t st) {
    if (S.n == 0) return cudaSuccess;
    const int block = 256;
    switch (variant) {
        case 14: MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::bgk_split_kernel<KQC, 3, KQC><<<blocks_for(2 * (int64_t)S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        case 15: MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::bgk_split_kernel<KQC, 4, 1><<<blocks_for(2 * (int64_t)S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        case 16: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_split_persistent<KQC, 4, 1>, 128, S.n, st, [&](int g) { dev::bgk_split_persistent<KQC, 4, 1><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); }))); break;
        case 17: MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::bgk_split_kernel<KQC, 4, 2><<<blocks_for(2 * (int64_t)S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        case 18:
        case 19: {
            // the second pass reads f8in only and writes the link nodes' outputs after the first pass
            if (variant == 18) {
                MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_nolink<KQC, 2>, 256, S.n, st, [&](int g) { dev::bgk_step_nolink<KQC, 2><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); })));
            } else {
                MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_nolink<KQC, 3>, 256, S.n, st, [&](int g) { dev::bgk_step_nolink<KQC, 3><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); })));
            }
            if (S.n_link_nodes > 0) {
                MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::bgk_link_nodes<KQC><<<(S.n_link_nodes + 7) / 8, 128, 0, st>>>(S, f8in, f0in, f8out, f0out, C)));
            }
            break;
        }
        case 22: {
            if (!S.lidx) return cudaErrorInvalidValue;  // no staging structure for this context
            const size_t smem = (size_t)4 * S.stage_max * sizeof(float4);
            MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_staged<KQC>, dev::kStageTile, S.n, st, [&](int g) { dev::bgk_step_staged<KQC><<<g, block, smem, st>>>(S, f8in, f0in, f8out, f0out, C); }, smem)));
            break;
        }
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace mlbm
