// Persistent, bulk-copy-pipelined versions of the fused step kernels.
//
// The per-node stencil data (least-squares matrix M, neighbour indices, meta
// byte) are read exactly once per step and make up ~90% of the bytes, so they
// are streamed through shared memory: one producer warp per CTA issues
// cp.async.bulk copies of whole node tiles (TN nodes: 6K/4 matrix rows, K/4
// index rows and the meta bytes, each a contiguous TN x 16-byte chunk of the
// interleaved layout) into a ring of STAGES buffers guarded by mbarriers;
// TN * 4 consumer threads (four lanes per node, one neighbour group of four
// each) gather the neighbours' populations through L1/L2, combine their
// partial sums with quad shuffles and split the collision.  The grid holds
// as many CTAs as fit on the SMs; each walks the tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...
//
// Every mbarrier wait is bounded by a time budget (nanoseconds of the global
// timer, two seconds unless the context sets another); a wait that runs out
// records an error code in *err and the warp leaves the loop, so a lost copy
// cannot hang the GPU.  The producer then waits (bounded again) for every
// copy it issued that may still be landing before the CTA exits.  The host
// reads *err after the run.  For tests of that path the host can ask one
// launch to withhold the copies of block 0's first tile, so that the
// consumers' wait for it runs out (Wait::withhold).
#include <cstdio>

#include "device_common.cuh"
#include "kernels.h"
#include "ring.cuh"

namespace mlbm {
namespace dev {

// ------------------------------------------------------------------- BGK
template <int KQ, int TN, int STAGES, int MINB>
__global__ void __launch_bounds__(Tile<KQ, TN, STAGES>::kThreads, MINB)
    bgk_step_tma(Stencil S, const float4* __restrict__ f8in, const float* __restrict__ f0in,
                 float4* __restrict__ f8out, float* __restrict__ f0out, Collide C0, int n_tiles, int* __restrict__ err,
                 const Wait W) {
    using L = Tile<KQ, TN, STAGES>;
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::kBar);
    uint64_t* empty = full + STAGES;
    const int warp = threadIdx.x >> 5;
    const unsigned lane = threadIdx.x & 31u;
    init_ring(full, empty, STAGES, L::kConsumers / 32);
    if (warp == L::kConsumers / 32) {
        produce<KQ, TN, STAGES>(S, smem, full, empty, n_tiles, err, W);
        return;
    }
    // lane = h * 8 + node-in-warp: the four lanes of a node are 8 apart, so a
    // quarter warp reads 8 consecutive 16-byte tile entries (no bank conflicts)
    const int t = (threadIdx.x >> 5) * 8 + (int)(lane & 7u);
    const int h = (int)(lane >> 3);
    const unsigned quad = 0x01010101u << (lane & 7u);
    int it = 0;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
        const int s = it % STAGES;
        // the warp leaves together if any lane's wait ran out, so that no
        // shuffle below waits on a lane that has left
        if (!__all_sync(0xffffffffu, mbar_wait(&full[s], (it / STAGES) & 1, W.budget_ns))) {
            if (lane == 0) atomicExch(err, 2);
            return;
        }
        const uint8_t* st = smem + s * L::kStage;
        const float4* sM = reinterpret_cast<const float4*>(st);
        const int4* sI = reinterpret_cast<const int4*>(st + L::kM);
        const int p = tile * TN + t;
        if (p < S.n) {
            const Collide C = collide_of(S, C0, p);
            const uint8_t meta = st[L::kM + L::kI + t];
            const int kind = meta & 3;
            float g[9];
            if (kind == 2) {
                const float4 e = S.eqv[p];
                eq_populations(e.x, e.y, e.z, g);
            } else {
                float acc[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) acc[k] = 0.f;
                const float4 oa = __ldg(f8in + 2 * (size_t)p);
                const float4 ob = __ldg(f8in + 2 * (size_t)p + 1);
                const float r = (kind == 1) ? __ldg(S.lag_r + p) : 0.f;
                const float cx = (kind == 1) ? (float)ex_of(meta >> 4) : 0.f;
                const float cy = (kind == 1) ? (float)ey_of(meta >> 4) : 0.f;
                if (kind == 0) {
#pragma unroll
                    for (int i = 0; i < (KQ + 3) / 4; ++i) {
                        const int q = 4 * i + h;
                        if (q < KQ) {
                            const int4 id = sI[q * TN + t];
                            float4 m[6];
#pragma unroll
                            for (int a = 0; a < 6; ++a) m[a] = sM[(a * KQ + q) * TN + t];
                            wls_acc(f8in, id.x, m[0].x, m[1].x, m[2].x, m[3].x, m[4].x, m[5].x, oa, ob, acc);
                            wls_acc(f8in, id.y, m[0].y, m[1].y, m[2].y, m[3].y, m[4].y, m[5].y, oa, ob, acc);
                            wls_acc(f8in, id.z, m[0].z, m[1].z, m[2].z, m[3].z, m[4].z, m[5].z, oa, ob, acc);
                            wls_acc(f8in, id.w, m[0].w, m[1].w, m[2].w, m[3].w, m[4].w, m[5].w, oa, ob, acc);
                        }
                    }
                } else {
                    const int4 i0 = sI[t], i1 = sI[TN + t], i2 = sI[2 * TN + t];
                    const int ids[9] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w, i2.x};
                    float xp[3], x0[3], xm[3], yp[3], y0[3], ym[3];
                    lag3(-r - cx, xp[0], xp[1], xp[2]);
                    lag3(-cx, x0[0], x0[1], x0[2]);
                    lag3(r - cx, xm[0], xm[1], xm[2]);
                    lag3(-r - cy, yp[0], yp[1], yp[2]);
                    lag3(-cy, y0[0], y0[1], y0[2]);
                    lag3(r - cy, ym[0], ym[1], ym[2]);
#pragma unroll
                    for (int bp = 0; bp < 9; ++bp) {
                        if ((bp & 3) != h) continue;
                        const int b = bp / 3, a = bp % 3;
                        const int j = ids[bp];
                        const float4 ra = __ldg(f8in + 2 * (size_t)j);
                        const float4 rb = __ldg(f8in + 2 * (size_t)j + 1);
                        acc[0] = fmaf(xp[a] * y0[b], ra.x - oa.x, acc[0]);
                        acc[1] = fmaf(x0[a] * yp[b], ra.y - oa.y, acc[1]);
                        acc[2] = fmaf(xm[a] * y0[b], ra.z - oa.z, acc[2]);
                        acc[3] = fmaf(x0[a] * ym[b], ra.w - oa.w, acc[3]);
                        acc[4] = fmaf(xp[a] * yp[b], rb.x - ob.x, acc[4]);
                        acc[5] = fmaf(xm[a] * yp[b], rb.y - ob.y, acc[5]);
                        acc[6] = fmaf(xm[a] * ym[b], rb.z - ob.z, acc[6]);
                        acc[7] = fmaf(xp[a] * ym[b], rb.w - ob.w, acc[7]);
                    }
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    acc[k] += __shfl_xor_sync(quad, acc[k], 8);
                    acc[k] += __shfl_xor_sync(quad, acc[k], 16);
                }
                const float own[8] = {oa.x, oa.y, oa.z, oa.w, ob.x, ob.y, ob.z, ob.w};
#pragma unroll
                for (int k = 0; k < 8; ++k) acc[k] += own[k];
                if (meta & 4) {
                    const LinkRec Lk = S.links[S.link_slot[p]];
                    for (int k = 1; k < 9; ++k) {
                        if (!((Lk.mask >> k) & 1u)) continue;
                        const int kp = opp_of(k);
                        float v;
                        if (S.bb_mode == 0) {
                            v = pop(f8in, p, kp);
                        } else if (kind == 0) {
                            float pb[6];
                            basis_at(k, Lk.t[k - 1], pb);
                            v = wls_general<KQ>(S, f8in, p, kp, pb);
                        } else {
                            int ids[9];
                            lag_block(S, p, ids);
                            float lx[3], ly[3];
                            lag3(Lk.t[k - 1] * r * ex_of(k) - cx, lx[0], lx[1], lx[2]);
                            lag3(Lk.t[k - 1] * r * ey_of(k) - cy, ly[0], ly[1], ly[2]);
                            const float o = pop(f8in, p, kp);
                            float sacc = 0.f;
                            for (int b = 0; b < 3; ++b)
                                for (int a = 0; a < 3; ++a)
                                    sacc = fmaf(lx[a] * ly[b], pop(f8in, ids[b * 3 + a], kp) - o, sacc);
                            v = o + sacc;
                        }
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk)
                            if (kk == k - 1) acc[kk] = v;
                    }
                }
                g[0] = f0in[p];
#pragma unroll
                for (int k = 1; k < 9; ++k) g[k] = acc[k - 1];
                collide_pairs(g, C, 1u << h, h == 0);
            }
            // lane h owns pair h: (1,3) (2,4) (5,7) (6,8); lanes 0 and 2 write
            float x = (h == 1) ? g[2] : g[6];
            float y = (h == 1) ? g[4] : g[8];
            x = __shfl_down_sync(quad, x, 8);
            y = __shfl_down_sync(quad, y, 8);
            if (kind == 2) {  // every lane holds all populations
                x = (h == 0) ? g[2] : g[6];
                y = (h == 0) ? g[4] : g[8];
            }
            if (h == 0) {
                f8out[2 * (size_t)p] = make_float4(g[1], x, g[3], y);
                f0out[p] = g[0];
            } else if (h == 2) {
                f8out[2 * (size_t)p + 1] = make_float4(g[5], x, g[7], y);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// --------------------------------------------------------------- tau = 1
template <int KQ, int TN, int STAGES, int MINB>
__global__ void __launch_bounds__(Tile<KQ, TN, STAGES>::kThreads, MINB)
    tau1_step_tma(Stencil S, const float4* __restrict__ in, float4* __restrict__ out, Collide C0, int n_tiles,
                  int* __restrict__ err, const Wait W) {
    using L = Tile<KQ, TN, STAGES>;
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::kBar);
    uint64_t* empty = full + STAGES;
    const int warp = threadIdx.x >> 5;
    const unsigned lane = threadIdx.x & 31u;
    init_ring(full, empty, STAGES, L::kConsumers / 32);
    if (warp == L::kConsumers / 32) {
        produce<KQ, TN, STAGES>(S, smem, full, empty, n_tiles, err, W);
        return;
    }
    // lane = h * 8 + node-in-warp: the four lanes of a node are 8 apart, so a
    // quarter warp reads 8 consecutive 16-byte tile entries (no bank conflicts)
    const int t = (threadIdx.x >> 5) * 8 + (int)(lane & 7u);
    const int h = (int)(lane >> 3);
    const unsigned quad = 0x01010101u << (lane & 7u);
    int it = 0;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
        const int s = it % STAGES;
        // the warp leaves together if any lane's wait ran out, so that no
        // shuffle below waits on a lane that has left
        if (!__all_sync(0xffffffffu, mbar_wait(&full[s], (it / STAGES) & 1, W.budget_ns))) {
            if (lane == 0) atomicExch(err, 2);
            return;
        }
        const uint8_t* st = smem + s * L::kStage;
        const float4* sM = reinterpret_cast<const float4*>(st);
        const int4* sI = reinterpret_cast<const int4*>(st + L::kM);
        const int p = tile * TN + t;
        if (p < S.n) {
            const Collide C = collide_of(S, C0, p);
            const uint8_t meta = st[L::kM + L::kI + t];
            const int kind = meta & 3;
            if (kind == 2) {
                if (h == 0) out[p] = S.eqv[p];
            } else {
                const float4 me = __ldg(in + p);
                float c[3][6];
                float4 v9[9];
                float r = 0.f, cx = 0.f, cy = 0.f;
                if (kind == 0) {
#pragma unroll
                    for (int f = 0; f < 3; ++f)
#pragma unroll
                        for (int a = 0; a < 6; ++a) c[f][a] = 0.f;
#pragma unroll
                    for (int i = 0; i < (KQ + 3) / 4; ++i) {
                        const int q = 4 * i + h;
                        if (q < KQ) {
                            const int4 id = sI[q * TN + t];
                            float4 m[6];
#pragma unroll
                            for (int a = 0; a < 6; ++a) m[a] = sM[(a * KQ + q) * TN + t];
                            const int ids[4] = {id.x, id.y, id.z, id.w};
#pragma unroll
                            for (int cc = 0; cc < 4; ++cc) {
                                const float4 rv = __ldg(in + ids[cc]);
                                const float vx = rv.x - me.x, vy = rv.y - me.y, vz = rv.z - me.z;
                                const float* mc = reinterpret_cast<const float*>(m);
#pragma unroll
                                for (int a = 0; a < 6; ++a) {
                                    const float ma = mc[4 * a + cc];
                                    c[0][a] = fmaf(ma, vx, c[0][a]);
                                    c[1][a] = fmaf(ma, vy, c[1][a]);
                                    c[2][a] = fmaf(ma, vz, c[2][a]);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int f = 0; f < 3; ++f)
#pragma unroll
                        for (int a = 0; a < 6; ++a) {
                            c[f][a] += __shfl_xor_sync(quad, c[f][a], 8);
                            c[f][a] += __shfl_xor_sync(quad, c[f][a], 16);
                        }
#pragma unroll
                    for (int f = 0; f < 3; ++f) {
                        float tc[6];
#pragma unroll
                        for (int a = 0; a < 6; ++a) tc[a] = c[f][a];
                        unbasis(tc, c[f]);
                    }
                } else {
                    const int4 i0 = sI[t], i1 = sI[TN + t], i2 = sI[2 * TN + t];
                    const int ids[9] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w, i2.x};
#pragma unroll
                    for (int b = 0; b < 9; ++b) v9[b] = __ldg(in + ids[b]);
                    r = __ldg(S.lag_r + p);
                    cx = (float)ex_of(meta >> 4);
                    cy = (float)ey_of(meta >> 4);
                }
                LinkRec Lk;
                Lk.mask = 0;
                if (meta & 4) Lk = S.links[S.link_slot[p]];
                const float rhox = 1.0f + me.x;
                float dm = 0.f, mx = 0.f, my = 0.f;
                if (h == 0)
                    dm = w_of(0) * rhox * (-1.5f * (me.y * me.y + me.z * me.z)) +
                         0.5f * src(0, rhox, me.y, me.z, C.ax, C.ay);
#pragma unroll
                for (int k = 1; k < 9; ++k) {
                    if (((k - 1) >> 1) != h) continue;
                    const bool is_link = (Lk.mask >> k) & 1u;
                    const int sk = is_link ? opp_of(k) : k;
                    float d[3] = {0.f, 0.f, 0.f};
                    if (!(is_link && S.bb_mode == 0)) {
                        const float tt = is_link ? Lk.t[k - 1] : -1.0f;
                        if (kind == 0) {
                            float pb[6];
                            basis_at(k, tt, pb);
#pragma unroll
                            for (int f = 0; f < 3; ++f) {
                                float v = 0.f;
#pragma unroll
                                for (int a = 0; a < 6; ++a) v = fmaf(pb[a], c[f][a], v);
                                d[f] = v;
                            }
                        } else {
                            float lx[3], ly[3];
                            lag3(tt * r * ex_of(k) - cx, lx[0], lx[1], lx[2]);
                            lag3(tt * r * ey_of(k) - cy, ly[0], ly[1], ly[2]);
#pragma unroll
                            for (int b = 0; b < 3; ++b)
#pragma unroll
                                for (int a = 0; a < 3; ++a) {
                                    const float w = lx[a] * ly[b];
                                    const float4 v = v9[b * 3 + a];
                                    d[0] = fmaf(w, v.x - me.x, d[0]);
                                    d[1] = fmaf(w, v.y - me.y, d[1]);
                                    d[2] = fmaf(w, v.z - me.z, d[2]);
                                }
                        }
                    }
                    tau1_accumulate(k, sk, is_link, d[0], d[1], d[2], rhox, me.y, me.z, C, dm, mx, my);
                }
                dm += __shfl_xor_sync(quad, dm, 8);
                mx += __shfl_xor_sync(quad, mx, 8);
                my += __shfl_xor_sync(quad, my, 8);
                dm += __shfl_xor_sync(quad, dm, 16);
                mx += __shfl_xor_sync(quad, mx, 16);
                my += __shfl_xor_sync(quad, my, 16);
                if (h == 0) {
                    const float rho = rhox + dm;
                    const float inv = 1.0f / rho;
                    const float nux = me.y + (mx + 0.5f * rho * C.ax - dm * me.y) * inv;
                    const float nuy = me.z + (my + 0.5f * rho * C.ay - dm * me.z) * inv;
                    out[p] = make_float4(me.x + dm, nux, nuy, 0.f);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

}  // namespace dev

// ------------------------------------------------------------- launchers
namespace {

template <int KQ, int TN, int STAGES, int MINB>
cudaError_t run_tma(int model, const dev::Stencil& S, const float4* a8, const float* a0, float4* b8, float* b0,
                    const float4* ra, float4* rb, const dev::Collide& C, int* err, const dev::Wait& W,
                    cudaStream_t st) {
    using L = dev::Tile<KQ, TN, STAGES>;
    static_assert(L::kBytes <= 232448, "tile ring exceeds shared memory");
    const void* fn = model == 0 ? (const void*)dev::bgk_step_tma<KQ, TN, STAGES, MINB>
                                : (const void*)dev::tau1_step_tma<KQ, TN, STAGES, MINB>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes);
    if (e != cudaSuccess) return e;
    int dev_id = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev_id);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, L::kThreads, L::kBytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int n_tiles = (S.n + TN - 1) / TN;
    const int grid = std::max(1, std::min(n_tiles, sms * per_sm));
    if (model == 0)
        dev::bgk_step_tma<KQ, TN, STAGES, MINB><<<grid, L::kThreads, L::kBytes, st>>>(S, a8, a0, b8, b0, C, n_tiles, err, W);
    else
        dev::tau1_step_tma<KQ, TN, STAGES, MINB><<<grid, L::kThreads, L::kBytes, st>>>(S, ra, rb, C, n_tiles, err, W);
    return cudaGetLastError();
}

template <int KQ>
cudaError_t run_tma_variant(int variant, int model, const dev::Stencil& S, const float4* a8, const float* a0,
                            float4* b8, float* b0, const float4* ra, float4* rb, const dev::Collide& C, int* err,
                            const dev::Wait& W, cudaStream_t st) {
    // stage count from the shared-memory budget
    constexpr int kStage128 = dev::Tile<KQ, 128, 1>::kStage;
    constexpr int kStage64 = dev::Tile<KQ, 64, 1>::kStage;
    constexpr int S128 = std::min(3, 232000 / kStage128);
    constexpr int S64 = std::min(3, 232000 / kStage64);
    switch (variant) {
        case 4: return run_tma<KQ, 128, S128, 1>(model, S, a8, a0, b8, b0, ra, rb, C, err, W, st);
        case 5: return run_tma<KQ, 128, 2, 2>(model, S, a8, a0, b8, b0, ra, rb, C, err, W, st);
        case 6: return run_tma<KQ, 64, S64, 2>(model, S, a8, a0, b8, b0, ra, rb, C, err, W, st);
        case 7: return run_tma<KQ, 64, 2, 3>(model, S, a8, a0, b8, b0, ra, rb, C, err, W, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool tma_supported(int Kq) { return Kq == 3 || Kq == 4 || Kq == 6 || Kq == 8; }

cudaError_t launch_step_tma(int variant, int model, const dev::Stencil& S, const float4* f8in, const float* f0in,
                            float4* f8out, float* f0out, const float4* rin, float4* rout, const dev::Collide& C,
                            int* err, const dev::Wait& W, cudaStream_t st) {
    if (S.n == 0) return cudaSuccess;
    switch (S.Kq) {
        case 3: return run_tma_variant<3>(variant, model, S, f8in, f0in, f8out, f0out, rin, rout, C, err, W, st);
        case 4: return run_tma_variant<4>(variant, model, S, f8in, f0in, f8out, f0out, rin, rout, C, err, W, st);
        case 6: return run_tma_variant<6>(variant, model, S, f8in, f0in, f8out, f0out, rin, rout, C, err, W, st);
        case 8: return run_tma_variant<8>(variant, model, S, f8in, f0in, f8out, f0out, rin, rout, C, err, W, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mlbm
