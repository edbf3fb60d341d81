// Fused MLBM step kernels (one thread per node) and the state I/O kernels.
//
// BGK/TRT step (Sec. 2.2 streaming, Eq. (3)-(9) collision), per node x:
//   gather the post-collision populations of the K stencil nodes, evaluate the
//   fit at the departure points x - s e_k (Eq. (12)) for k = 1..8, apply the
//   bounce-back links (Sec. 3.1 simple, Eq. (22) interpolated), take f_0 from
//   the node itself, form rho and u (+ g/2), collide (TRT; BGK when
//   tau- = tau+) with the second-order body-force source, write the other
//   buffer.  One pass, no intermediate array.
// tau = 1 step (MLBM1, Eq. (14)-(15)): the same gather on (rho, u, v), fitted
// quadratic coefficients of the three fields, equilibria (+ half the source)
// at the departure points summed into the new moments.
//
// All population values are stored minus their weight omega_k (and rho as
// rho - 1) so that FP32 keeps the small deviations that carry the flow.
// Interpolation is centred on the node's own value, f(x_d) = f(x) +
// sum_j w_j (f_j - f(x)), which equals sum_j w_j f_j because the weights sum
// to one; with FP32 weights the sum is one only to ~1e-7, and the centred form
// keeps that error off the mean value (it would otherwise act as a steady
// mass/momentum source that the slow viscous modes amplify).
#include <cstdio>

#include "device_common.cuh"
#include "kernels.h"

namespace mlbm {
namespace dev {

// ------------------------------------------------------------ BGK / TRT
// LPN lanes (1 or 2) cooperate on one node: lane h takes the neighbour groups
// q = h, h + LPN, ... and the partial sums are combined with a pair shuffle.
// LINKS = false leaves out the bounce-back overrides (the split variants
// recompute the nodes with links in a second pass); RBF = true interpolates
// the least-squares-kind nodes with their stored RBF-FD weights.  SPEC = true
// loads the first three index rows and the rest population before the node
// kind is known (they are read by every stencil kind), so they are in flight
// together with the meta byte
template <int KQ, int LPN, bool LINKS = true, bool RBF = false, bool SPEC = false>
__device__ __forceinline__ void bgk_node(const Stencil& S, const float4* __restrict__ f8in,
                                         const float* __restrict__ f0in, float4* __restrict__ f8out,
                                         float* __restrict__ f0out, const Collide& C0, int p, int h, unsigned grp) {
    const Collide C = collide_of(S, C0, p);
    const uint8_t meta = S.meta[p];
    const int kind = meta & 3;
    int4 idv[(KQ + LPN - 1) / LPN];
    float f0own = 0.f;
    if (SPEC) {
#pragma unroll
        for (int i = 0; i < (KQ + LPN - 1) / LPN; ++i) {
            const int q = i * LPN + h;
            if (q < KQ && q < 3) idv[i] = ld_stream(S.idx + (size_t)q * S.n_pad + p);
        }
        f0own = f0in[p];
    }
    float g[9];
    if (kind == 2) {
        const float4 e = S.eqv[p];
        eq_populations(e.x, e.y, e.z, g);
    } else {
        float acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = 0.f;
        const float r = (kind == 1) ? __ldg(S.lag_r + p) : 0.f;
        const float cx = (kind == 1) ? (float)ex_of(meta >> 4) : 0.f;
        const float cy = (kind == 1) ? (float)ey_of(meta >> 4) : 0.f;
        const float4 oa = __ldg(f8in + 2 * (size_t)p);
        const float4 ob = __ldg(f8in + 2 * (size_t)p + 1);
        if (kind == 0 && RBF) {
            // f_k(x) = own_k + sum_j w_kj (f_k(j) - own_k), weights per direction
#pragma unroll
            for (int i = 0; i < (KQ + LPN - 1) / LPN; ++i) {
                const int q = i * LPN + h;
                if (q < KQ && (!SPEC || q >= 3)) idv[i] = ld_stream(S.idx + (size_t)q * S.n_pad + p);
            }
#pragma unroll
            for (int i = 0; i < (KQ + LPN - 1) / LPN; ++i) {
                const int q = i * LPN + h;
                if (q < KQ) {
                    const int4 id = idv[i];
                    float wt[8][4];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const float4 w4 = ld_stream(S.Wr + (size_t)(k * KQ + q) * S.n_pad + p);
                        wt[k][0] = w4.x; wt[k][1] = w4.y; wt[k][2] = w4.z; wt[k][3] = w4.w;
                    }
                    const int ids[4] = {id.x, id.y, id.z, id.w};
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float4 ra = __ldg(f8in + 2 * (size_t)ids[c]);
                        const float4 rb = __ldg(f8in + 2 * (size_t)ids[c] + 1);
                        acc[0] = fmaf(wt[0][c], ra.x - oa.x, acc[0]);
                        acc[1] = fmaf(wt[1][c], ra.y - oa.y, acc[1]);
                        acc[2] = fmaf(wt[2][c], ra.z - oa.z, acc[2]);
                        acc[3] = fmaf(wt[3][c], ra.w - oa.w, acc[3]);
                        acc[4] = fmaf(wt[4][c], rb.x - ob.x, acc[4]);
                        acc[5] = fmaf(wt[5][c], rb.y - ob.y, acc[5]);
                        acc[6] = fmaf(wt[6][c], rb.z - ob.z, acc[6]);
                        acc[7] = fmaf(wt[7][c], rb.w - ob.w, acc[7]);
                    }
                }
            }
        } else if (kind == 0) {
            // all index rows first, so the gathers of later stencil quads need
            // not wait for their index load behind the matrix rows
#pragma unroll
            for (int i = 0; i < (KQ + LPN - 1) / LPN; ++i) {
                const int q = i * LPN + h;
                if (q < KQ && (!SPEC || q >= 3)) idv[i] = ld_stream(S.idx + (size_t)q * S.n_pad + p);
            }
#pragma unroll
            for (int i = 0; i < (KQ + LPN - 1) / LPN; ++i) {
                const int q = i * LPN + h;
                if (q < KQ) {
                    const int4 id = idv[i];
                    float4 m[6];
#pragma unroll
                    for (int a = 0; a < 6; ++a) m[a] = ld_stream(S.M + (size_t)(a * KQ + q) * S.n_pad + p);
                    wls_acc(f8in, id.x, m[0].x, m[1].x, m[2].x, m[3].x, m[4].x, m[5].x, oa, ob, acc);
                    wls_acc(f8in, id.y, m[0].y, m[1].y, m[2].y, m[3].y, m[4].y, m[5].y, oa, ob, acc);
                    wls_acc(f8in, id.z, m[0].z, m[1].z, m[2].z, m[3].z, m[4].z, m[5].z, oa, ob, acc);
                    wls_acc(f8in, id.w, m[0].w, m[1].w, m[2].w, m[3].w, m[4].w, m[5].w, oa, ob, acc);
                }
            }
        } else {
            int ids[9];
            lag_block(S, p, ids);
            // basis values for e_x, e_y in {+1, 0, -1}: t = -r e - c
            float xp[3], x0[3], xm[3], yp[3], y0[3], ym[3];
            lag3(-r - cx, xp[0], xp[1], xp[2]);
            lag3(-cx, x0[0], x0[1], x0[2]);
            lag3(r - cx, xm[0], xm[1], xm[2]);
            lag3(-r - cy, yp[0], yp[1], yp[2]);
            lag3(-cy, y0[0], y0[1], y0[2]);
            lag3(r - cy, ym[0], ym[1], ym[2]);
#pragma unroll
            for (int bp = 0; bp < 9; ++bp) {
                if (LPN == 2 && (bp & 1) != h) continue;
                const int b = bp / 3, a = bp % 3;
                const int j = ids[bp];
                const float4 ra = __ldg(f8in + 2 * (size_t)j);
                const float4 rb = __ldg(f8in + 2 * (size_t)j + 1);
                const float4 fa = make_float4(ra.x - oa.x, ra.y - oa.y, ra.z - oa.z, ra.w - oa.w);
                const float4 fb = make_float4(rb.x - ob.x, rb.y - ob.y, rb.z - ob.z, rb.w - ob.w);
                acc[0] = fmaf(xp[a] * y0[b], fa.x, acc[0]);
                acc[1] = fmaf(x0[a] * yp[b], fa.y, acc[1]);
                acc[2] = fmaf(xm[a] * y0[b], fa.z, acc[2]);
                acc[3] = fmaf(x0[a] * ym[b], fa.w, acc[3]);
                acc[4] = fmaf(xp[a] * yp[b], fb.x, acc[4]);
                acc[5] = fmaf(xm[a] * yp[b], fb.y, acc[5]);
                acc[6] = fmaf(xm[a] * ym[b], fb.z, acc[6]);
                acc[7] = fmaf(xp[a] * ym[b], fb.w, acc[7]);
            }
        }
        if (LPN == 2) {
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] += __shfl_xor_sync(grp, acc[k], 1);
        }
        float own[8] = {oa.x, oa.y, oa.z, oa.w, ob.x, ob.y, ob.z, ob.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += own[k];
        if (LINKS && (meta & 4)) {
            // bounce-back links (rare): every lane of the node computes them
            const LinkRec L = S.links[S.link_slot[p]];
#pragma unroll
            for (int k = 1; k < 9; ++k) {
                if (!((L.mask >> k) & 1u)) continue;
                const int kp = opp_of(k);
                if (S.bb_mode == 0) {
                    acc[k - 1] = own[kp - 1];
                } else if (kind == 0 && RBF) {
                    acc[k - 1] = rbf_general<KQ>(S, f8in, p, k - 1, kp);
                } else if (kind == 0) {
                    float pb[6];
                    basis_at(k, L.t[k - 1], pb);
                    acc[k - 1] = wls_general<KQ>(S, f8in, p, kp, pb);
                } else {
                    int ids[9];
                    lag_block(S, p, ids);
                    const float tt = L.t[k - 1];
                    float lx[3], ly[3];
                    lag3(tt * r * ex_of(k) - cx, lx[0], lx[1], lx[2]);
                    lag3(tt * r * ey_of(k) - cy, ly[0], ly[1], ly[2]);
                    const float o = own[kp - 1];
                    float v = 0.f;
                    for (int b = 0; b < 3; ++b)
                        for (int a = 0; a < 3; ++a) v = fmaf(lx[a] * ly[b], pop(f8in, ids[b * 3 + a], kp) - o, v);
                    acc[k - 1] = o + v;
                }
            }
        }
        g[0] = SPEC ? f0own : f0in[p];
#pragma unroll
        for (int k = 1; k < 9; ++k) g[k] = acc[k - 1];
        collide_part<LPN>(g, C, h);
    }
    if (LPN == 1 || h == 0) {
        f8out[2 * (size_t)p] = make_float4(g[1], g[2], g[3], g[4]);
        f0out[p] = g[0];
    }
    if (LPN == 1 || h == 1) f8out[2 * (size_t)p + 1] = make_float4(g[5], g[6], g[7], g[8]);
}

// Two lanes per node split by direction half: lane h gathers only the
// 16-byte half record f_{4h+1..4h+4} of each stencil node (one load per
// neighbour) and needs only four of the six matrix rows; every direction's
// opposite lies in the same half, so bounce-back stays in the lane.  The
// halves are exchanged with four shuffles before the pair-split collision
// (pairs (1,3), (2,4) on lane 0, (5,7), (6,8) on lane 1).
template <int KQ, int UQ>
__device__ __forceinline__ void bgk_node_split(const Stencil& S, const float4* __restrict__ f8in,
                                               const float* __restrict__ f0in, float4* __restrict__ f8out,
                                               float* __restrict__ f0out, const Collide& C0, int p, int h,
                                               unsigned grp) {
    const Collide C = collide_of(S, C0, p);
    const uint8_t meta = S.meta[p];
    const int kind = meta & 3;
    float g[9];
    if (kind == 2) {
        const float4 e = S.eqv[p];
        eq_populations(e.x, e.y, e.z, g);
    } else {
        const float4 own = __ldg(f8in + 2 * (size_t)p + h);
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const float r = (kind == 1) ? __ldg(S.lag_r + p) : 0.f;
        const float cx = (kind == 1) ? (float)ex_of(meta >> 4) : 0.f;
        const float cy = (kind == 1) ? (float)ey_of(meta >> 4) : 0.f;
        if (kind == 0) {
            const int ra = h ? 2 : 0, rb = h ? 3 : 1;
            // UQ neighbour groups in flight at a time (register budget)
#pragma unroll UQ
            for (int q = 0; q < KQ; ++q) {
                const int4 id = ld_stream(S.idx + (size_t)q * S.n_pad + p);
                const float4 mA = ld_stream(S.M + (size_t)(ra * KQ + q) * S.n_pad + p);
                const float4 mB = ld_stream(S.M + (size_t)(rb * KQ + q) * S.n_pad + p);
                const float4 m1 = ld_stream(S.M + (size_t)(4 * KQ + q) * S.n_pad + p);
                const float4 m2 = ld_stream(S.M + (size_t)(5 * KQ + q) * S.n_pad + p);
                const int ids[4] = {id.x, id.y, id.z, id.w};
                const float A4[4] = {mA.x, mA.y, mA.z, mA.w}, B4[4] = {mB.x, mB.y, mB.z, mB.w};
                const float P4[4] = {m1.x, m1.y, m1.z, m1.w}, Q4[4] = {m2.x, m2.y, m2.z, m2.w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float4 v = __ldg(f8in + 2 * (size_t)ids[c] + h);
                    const float a0 = v.x - own.x, a1 = v.y - own.y, a2 = v.z - own.z, a3 = v.w - own.w;
                    // h = 0: A = U, B = V, X = m1, Y = m2 ; h = 1: A = W, B = W', X = m1 + m2, Y = m1 - m2
                    const float X = h ? P4[c] + Q4[c] : P4[c];
                    const float Y = h ? P4[c] - Q4[c] : Q4[c];
                    // h = 0: k = 1 (A - X), 2 (B - Y), 3 (A + X), 4 (B + Y)
                    // h = 1: k = 5 (A - X), 6 (B + Y), 7 (A + X), 8 (B - Y)
                    const float sy = h ? 1.f : -1.f;
                    acc[0] = fmaf(-X, a0, fmaf(A4[c], a0, acc[0]));
                    acc[1] = fmaf(sy * Y, a1, fmaf(B4[c], a1, acc[1]));
                    acc[2] = fmaf(X, a2, fmaf(A4[c], a2, acc[2]));
                    acc[3] = fmaf(-sy * Y, a3, fmaf(B4[c], a3, acc[3]));
                }
            }
        } else {
            int ids[9];
            lag_block(S, p, ids);
            float xp[3], x0[3], xm[3], yp[3], y0[3], ym[3];
            lag3(-r - cx, xp[0], xp[1], xp[2]);
            lag3(-cx, x0[0], x0[1], x0[2]);
            lag3(r - cx, xm[0], xm[1], xm[2]);
            lag3(-r - cy, yp[0], yp[1], yp[2]);
            lag3(-cy, y0[0], y0[1], y0[2]);
            lag3(r - cy, ym[0], ym[1], ym[2]);
#pragma unroll
            for (int bp = 0; bp < 9; ++bp) {
                const int b = bp / 3, a = bp % 3;
                const float4 v = __ldg(f8in + 2 * (size_t)ids[bp] + h);
                // weights of this half's four directions
                const float w0 = h ? xp[a] * yp[b] : xp[a] * y0[b];
                const float w1 = h ? xm[a] * yp[b] : x0[a] * yp[b];
                const float w2 = h ? xm[a] * ym[b] : xm[a] * y0[b];
                const float w3 = h ? xp[a] * ym[b] : x0[a] * ym[b];
                acc[0] = fmaf(w0, v.x - own.x, acc[0]);
                acc[1] = fmaf(w1, v.y - own.y, acc[1]);
                acc[2] = fmaf(w2, v.z - own.z, acc[2]);
                acc[3] = fmaf(w3, v.w - own.w, acc[3]);
            }
        }
        acc[0] += own.x;
        acc[1] += own.y;
        acc[2] += own.z;
        acc[3] += own.w;
        if (meta & 4) {
            const LinkRec L = S.links[S.link_slot[p]];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 4 * h + i + 1;
                if (!((L.mask >> k) & 1u)) continue;
                const int kp = opp_of(k);
                float v;
                if (S.bb_mode == 0) {
                    v = pop(f8in, p, kp);
                } else if (kind == 0) {
                    float pb[6];
                    basis_at(k, L.t[k - 1], pb);
                    v = wls_general<KQ>(S, f8in, p, kp, pb);
                } else {
                    int ids[9];
                    lag_block(S, p, ids);
                    const float tt = L.t[k - 1];
                    float lx[3], ly[3];
                    lag3(tt * r * ex_of(k) - cx, lx[0], lx[1], lx[2]);
                    lag3(tt * r * ey_of(k) - cy, ly[0], ly[1], ly[2]);
                    const float o = pop(f8in, p, kp);
                    float sacc = 0.f;
                    for (int b = 0; b < 3; ++b)
                        for (int a = 0; a < 3; ++a) sacc = fmaf(lx[a] * ly[b], pop(f8in, ids[b * 3 + a], kp) - o, sacc);
                    v = o + sacc;
                }
                acc[i] = v;
            }
        }
        float oth[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) oth[i] = __shfl_xor_sync(grp, acc[i], 1);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            g[1 + i] = h ? oth[i] : acc[i];
            g[5 + i] = h ? acc[i] : oth[i];
        }
        g[0] = f0in[p];
        collide_pairs(g, C, h == 0 ? 0x3u : 0xCu, h == 0);
    }
    if (h == 0) {
        f8out[2 * (size_t)p] = make_float4(g[1], g[2], g[3], g[4]);
        f0out[p] = g[0];
    } else {
        f8out[2 * (size_t)p + 1] = make_float4(g[5], g[6], g[7], g[8]);
    }
}

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

// Bulk prefetch of a node tile's stencil rows (matrix, indices, meta) into L2,
// issued by the lanes of one warp; no registers or shared memory are used.
__device__ __forceinline__ void prefetch_l2(const void* ptr, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(ptr), "r"(bytes) : "memory");
}

template <int KQ>
__device__ __forceinline__ void prefetch_tile(const Stencil& S, int base, int tn, unsigned lane) {
    if (base >= S.n) return;
    const int nodes = min(tn, S.n_pad - base);
    for (int c = (int)lane; c < 7 * KQ + 1; c += 32) {
        if (c < 6 * KQ)
            prefetch_l2(S.M + (size_t)c * S.n_pad + base, (uint32_t)nodes * 16u);
        else if (c < 7 * KQ)
            prefetch_l2(S.idx + (size_t)(c - 6 * KQ) * S.n_pad + base, (uint32_t)nodes * 16u);
        else
            prefetch_l2(S.meta + base, (uint32_t)((nodes + 15) / 16 * 16));
    }
}

// Programmatic dependent launch (variants 25, 26): a step grid lets the next
// step's grid be scheduled on the SM slots it frees (launch_dependents), and
// the next grid issues only reads of the fixed stencil rows (L2 prefetch)
// before it waits for the previous grid to complete and its writes to be
// visible (wait); populations are read and written only after the wait.
// Without a programmatic predecessor the wait returns at once.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <int KQ, int LPN, int MINB, bool SPEC = false, int BS = 256, bool PDL = false>
__global__ void __launch_bounds__(BS, MINB) bgk_step_kernel(Stencil S, const float4* __restrict__ f8in,
                                                             const float* __restrict__ f0in,
                                                             float4* __restrict__ f8out, float* __restrict__ f0out,
                                                             Collide C) {
    if (PDL) {
        if (threadIdx.x < 32) prefetch_tile<KQ>(S, blockIdx.x * (BS / LPN), BS / LPN, threadIdx.x & 31u);
        pdl_trigger();
        pdl_wait();
    }
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = tid / LPN;
    const int h = tid % LPN;
    if (p >= S.n) return;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned grp = LPN == 1 ? (1u << lane) : (3u << (lane & ~1u));
    bgk_node<KQ, LPN, true, false, SPEC>(S, f8in, f0in, f8out, f0out, C, p, h, grp);
}

// Persistent form: gridDim.x resident blocks walk the node tiles; before a
// tile, warp 0 prefetches the stencil rows of the tile `dist` rounds ahead
// into L2, so the streamed loads of later tiles hit L2 instead of waiting on
// HBM while this tile gathers and collides.
template <int KQ, int LPN, int MINB, bool SPEC = false, int BS = 256, bool PDL = false>
__global__ void __launch_bounds__(BS, MINB) bgk_step_persistent(Stencil S, const float4* __restrict__ f8in,
                                                                const float* __restrict__ f0in,
                                                                float4* __restrict__ f8out,
                                                                float* __restrict__ f0out, Collide C, int dist) {
    constexpr int TN = BS / LPN;
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
        if (p < S.n) bgk_node<KQ, LPN, true, false, SPEC>(S, f8in, f0in, f8out, f0out, C, p, h, grp);
    }
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
template <int KQ>
__device__ __forceinline__ void prefetch_tile_rbf(const Stencil& S, int base, int tn, unsigned lane) {
    if (base >= S.n) return;
    const int nodes = min(tn, S.n_pad - base);
    for (int c = (int)lane; c < 9 * KQ + 1; c += 32) {
        if (c < 8 * KQ)
            prefetch_l2(S.Wr + (size_t)c * S.n_pad + base, (uint32_t)nodes * 16u);
        else if (c < 9 * KQ)
            prefetch_l2(S.idx + (size_t)(c - 8 * KQ) * S.n_pad + base, (uint32_t)nodes * 16u);
        else
            prefetch_l2(S.meta + base, (uint32_t)((nodes + 15) / 16 * 16));
    }
}

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

// --------------------------------------------------------- tau = 1 (MLBM1)
// (dr, u, v) at a departure point from the fitted quadratic coefficients
__device__ __forceinline__ void eval_coeffs(const float (*c)[6], const float* pb, float* out) {
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        float v = 0.f;
#pragma unroll
        for (int a = 0; a < 6; ++a) v = fmaf(pb[a], c[f][a], v);
        out[f] = v;
    }
}

// LPN lanes per node: neighbour groups split as in the BGK kernel, the 18
// fitted coefficients combined by a pair shuffle, the 8 directions split
// (lane 0: k = 0..4, lane 1: k = 5..8) and the moment sums combined again.
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
template <int KQ, int LPN, bool RBF = false>
__device__ __forceinline__ void tau1_node(const Stencil& S, const float4* __restrict__ in, float4* __restrict__ out,
                                          const Collide& C0, int p, int h, unsigned grp) {
    const Collide C = collide_of(S, C0, p);
    const uint8_t meta = S.meta[p];
    const int kind = meta & 3;
    if (kind == 2) {
        if (h == 0) out[p] = S.eqv[p];
        return;
    }
    const float4 me = __ldg(in + p);
    float c[3][6];
    float4 v9[9];
    float dd[RBF ? 8 : 1][3];  // RBF-FD increments per direction
    float r = 0.f, cx = 0.f, cy = 0.f;
    if (kind == 0 && RBF) {
#pragma unroll
        for (int k = 0; k < (RBF ? 8 : 1); ++k) dd[k][0] = dd[k][1] = dd[k][2] = 0.f;
        int4 idv[KQ];
#pragma unroll
        for (int q = 0; q < KQ; ++q) idv[q] = ld_stream(S.idx + (size_t)q * S.n_pad + p);
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            const int4 id = idv[q];
            float wt[8][4];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float4 w4 = ld_stream(S.Wr + (size_t)(k * KQ + q) * S.n_pad + p);
                wt[k][0] = w4.x; wt[k][1] = w4.y; wt[k][2] = w4.z; wt[k][3] = w4.w;
            }
            const int ids[4] = {id.x, id.y, id.z, id.w};
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const float4 rv = __ldg(in + ids[cc]);
                const float vx = rv.x - me.x, vy = rv.y - me.y, vz = rv.z - me.z;
#pragma unroll
                for (int k = 0; k < (RBF ? 8 : 1); ++k) {
                    dd[k][0] = fmaf(wt[k][cc], vx, dd[k][0]);
                    dd[k][1] = fmaf(wt[k][cc], vy, dd[k][1]);
                    dd[k][2] = fmaf(wt[k][cc], vz, dd[k][2]);
                }
            }
        }
    } else if (kind == 0) {
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int a = 0; a < 6; ++a) c[f][a] = 0.f;
        int4 idv[(KQ + LPN - 1) / LPN];
#pragma unroll
        for (int i = 0; i < (KQ + LPN - 1) / LPN; ++i) {
            const int q = i * LPN + h;
            if (q < KQ) idv[i] = ld_stream(S.idx + (size_t)q * S.n_pad + p);
        }
#pragma unroll
        for (int i = 0; i < (KQ + LPN - 1) / LPN; ++i) {
            const int q = i * LPN + h;
            if (q < KQ) {
                const int4 id = idv[i];
                float4 m[6];
#pragma unroll
                for (int a = 0; a < 6; ++a) m[a] = ld_stream(S.M + (size_t)(a * KQ + q) * S.n_pad + p);
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
        if (LPN == 2) {
#pragma unroll
            for (int f = 0; f < 3; ++f)
#pragma unroll
                for (int a = 0; a < 6; ++a) c[f][a] += __shfl_xor_sync(grp, c[f][a], 1);
        }
        // coefficients of the stored basis -> monomial basis
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            float tc[6];
#pragma unroll
            for (int a = 0; a < 6; ++a) tc[a] = c[f][a];
            unbasis(tc, c[f]);
        }
    } else {
        int ids[9];
        lag_block(S, p, ids);
#pragma unroll
        for (int b = 0; b < 9; ++b) v9[b] = __ldg(in + ids[b]);
        r = __ldg(S.lag_r + p);
        cx = (float)ex_of(meta >> 4);
        cy = (float)ey_of(meta >> 4);
    }
    LinkRec L;
    L.mask = 0;
    if (meta & 4) L = S.links[S.link_slot[p]];
    const float rhox = 1.0f + me.x;
    float dm = 0.f, mx = 0.f, my = 0.f;
    if (LPN == 1 || h == 0)
        dm = w_of(0) * rhox * (-1.5f * (me.y * me.y + me.z * me.z)) + 0.5f * src(0, rhox, me.y, me.z, C.ax, C.ay);
#pragma unroll
    for (int k = 1; k < 9; ++k) {
        if (LPN == 2 && ((k - 1) >> 2) != h) continue;
        const bool is_link = (L.mask >> k) & 1u;
        const int sk = is_link ? opp_of(k) : k;
        float d[3] = {0.f, 0.f, 0.f};  // increments over the node's own (dr, u, v)
        if (!(is_link && S.bb_mode == 0)) {
            const float tt = is_link ? L.t[k - 1] : -1.0f;
            if (kind == 0 && RBF) {
                // the stored row is at the departure point, or at the reflected
                // point of an interpolated bounce-back link
                d[0] = dd[RBF ? k - 1 : 0][0];
                d[1] = dd[RBF ? k - 1 : 0][1];
                d[2] = dd[RBF ? k - 1 : 0][2];
            } else if (kind == 0) {
                float pb[6];
                basis_at(k, tt, pb);
                eval_coeffs(c, pb, d);
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
    if (LPN == 2) {
        dm += __shfl_xor_sync(grp, dm, 1);
        mx += __shfl_xor_sync(grp, mx, 1);
        my += __shfl_xor_sync(grp, my, 1);
    }
    if (LPN == 1 || h == 0) {
        const float rho = rhox + dm;
        const float inv = 1.0f / rho;
        const float nux = me.y + (mx + 0.5f * rho * C.ax - dm * me.y) * inv;
        const float nuy = me.z + (my + 0.5f * rho * C.ay - dm * me.z) * inv;
        out[p] = make_float4(me.x + dm, nux, nuy, 0.f);
    }
}

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

// ------------------------------------------------------------- state I/O
__global__ void set_bgk_from_f64(int n, const int* __restrict__ perm, const double* __restrict__ f,
                                 float4* __restrict__ f8, float* __restrict__ f0) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double* fi = f + 9 * (size_t)perm[p];
    float g[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double w = k == 0 ? 4.0 / 9.0 : (k <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        g[k] = (float)(fi[k] - w);
    }
    f8[2 * (size_t)p] = make_float4(g[1], g[2], g[3], g[4]);
    f8[2 * (size_t)p + 1] = make_float4(g[5], g[6], g[7], g[8]);
    f0[p] = g[0];
}

__global__ void get_bgk_to_f64(int n, const int* __restrict__ perm, const float4* __restrict__ f8,
                               const float* __restrict__ f0, double* __restrict__ f) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double* fi = f + 9 * (size_t)perm[p];
    const float4 a = f8[2 * (size_t)p], b = f8[2 * (size_t)p + 1];
    const float g[9] = {f0[p], a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double w = k == 0 ? 4.0 / 9.0 : (k <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        fi[k] = (double)g[k] + w;
    }
}

// state at t = 0 from (rho, u): BGK populations at equilibrium, computed in FP64
__global__ void set_bgk_equilibrium(int n, const int* __restrict__ perm, const double* __restrict__ ru,
                                    float4* __restrict__ f8, float* __restrict__ f0) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double* v = ru + 3 * (size_t)perm[p];
    const double rho = v[0], ux = v[1], uy = v[2];
    const double usq = ux * ux + uy * uy;
    float g[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double w = k == 0 ? 4.0 / 9.0 : (k <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        const double eu = ex_of(k) * ux + ey_of(k) * uy;
        g[k] = (float)(w * ((rho - 1.0) + rho * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq)));
    }
    f8[2 * (size_t)p] = make_float4(g[1], g[2], g[3], g[4]);
    f8[2 * (size_t)p + 1] = make_float4(g[5], g[6], g[7], g[8]);
    f0[p] = g[0];
}

__global__ void set_tau1_from_f64(int n, const int* __restrict__ perm, const double* __restrict__ ru,
                                  float4* __restrict__ s) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double* v = ru + 3 * (size_t)perm[p];
    s[p] = make_float4((float)(v[0] - 1.0), (float)v[1], (float)v[2], 0.f);
}

__global__ void get_tau1_to_f64(int n, const int* __restrict__ perm, const float4* __restrict__ s,
                                double* __restrict__ ru) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double* v = ru + 3 * (size_t)perm[p];
    const float4 a = s[p];
    v[0] = (double)a.x + 1.0;
    v[1] = a.y;
    v[2] = a.z;
}

// rho, u of the state into FP32 sorted-order arrays (and optionally FP64
// caller-order rho_u[n][3]).  BGK: rho = sum f, rho u = sum f e - rho a / 2.
__global__ void macroscopics_bgk(int n, const int* __restrict__ perm, const float4* __restrict__ f8,
                                 const float* __restrict__ f0, float ax0, float ay0,
                                 const uint16_t* __restrict__ node_sample, const Collide* __restrict__ coll,
                                 float* __restrict__ rho_o, float* __restrict__ ux_o, float* __restrict__ uy_o,
                                 double* __restrict__ ru) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float ax = node_sample ? coll[node_sample[p]].ax : ax0;
    const float ay = node_sample ? coll[node_sample[p]].ay : ay0;
    const float4 a = f8[2 * (size_t)p], b = f8[2 * (size_t)p + 1];
    const float g0 = f0[p];
    const float dr = g0 + (a.x + a.y + a.z + a.w) + (b.x + b.y + b.z + b.w);
    const float jx = (a.x - a.z) + (b.x - b.y) + (b.w - b.z);
    const float jy = (a.y - a.w) + (b.x + b.y) - (b.z + b.w);
    const float rho = 1.0f + dr;
    const float ux = jx / rho - 0.5f * ax, uy = jy / rho - 0.5f * ay;
    rho_o[p] = rho;
    ux_o[p] = ux;
    uy_o[p] = uy;
    if (ru) {
        double* v = ru + 3 * (size_t)perm[p];
        v[0] = 1.0 + (double)dr;
        v[1] = ux;
        v[2] = uy;
    }
}

__global__ void macroscopics_tau1(int n, const int* __restrict__ perm, const float4* __restrict__ s,
                                  float* __restrict__ rho_o, float* __restrict__ ux_o, float* __restrict__ uy_o,
                                  double* __restrict__ ru) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float4 a = s[p];
    rho_o[p] = 1.0f + a.x;
    ux_o[p] = a.y;
    uy_o[p] = a.z;
    if (ru) {
        double* v = ru + 3 * (size_t)perm[p];
        v[0] = 1.0 + (double)a.x;
        v[1] = a.y;
        v[2] = a.z;
    }
}

// --------------------------------------------------------- wall force
// Momentum handed to the solids in the next streaming step: sum over links of
// 2 (f_k(t+1, x) - omega_k) e_{k'} area_x / s^2 (relative to the rest state,
// whose uniform pressure exerts no net force on a closed body), per-block
// FP64 partials added in a fixed order.
template <int KQ>
__global__ void __launch_bounds__(128) force_kernel(Stencil S, int model, int n_link_nodes,
                                                    const int* __restrict__ link_nodes,
                                                    const float* __restrict__ area_over_s2,
                                                    const float4* __restrict__ st8, const float4* __restrict__ ruv,
                                                    Collide C, double* __restrict__ partial) {
    double fx = 0.0, fy = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_link_nodes; e += gridDim.x * blockDim.x) {
        const int p = link_nodes[e];
        const Collide Cn = collide_of(S, C, p);
        const uint8_t meta = S.meta[p];
        const int kind = meta & 3;
        const LinkRec L = S.links[S.link_slot[p]];
        const float r = (kind == 1) ? S.lag_r[p] : 0.f;
        const float cx = (kind == 1) ? (float)ex_of(meta >> 4) : 0.f;
        const float cy = (kind == 1) ? (float)ey_of(meta >> 4) : 0.f;
        const double a = area_over_s2[p];
        for (int k = 1; k < 9; ++k) {
            if (!((L.mask >> k) & 1u)) continue;
            const int kp = opp_of(k);
            float val;
            if (model == 0) {
                if (S.bb_mode == 0) {
                    val = pop(st8, p, kp);
                } else if (kind == 0 && S.Wr) {
                    val = rbf_general<KQ>(S, st8, p, k - 1, kp);
                } else if (kind == 0) {
                    float pb[6];
                    basis_at(k, L.t[k - 1], pb);
                    val = wls_general<KQ>(S, st8, p, kp, pb);
                } else {
                    int ids[9];
                    lag_block(S, p, ids);
                    float lx[3], ly[3];
                    lag3(L.t[k - 1] * r * ex_of(k) - cx, lx[0], lx[1], lx[2]);
                    lag3(L.t[k - 1] * r * ey_of(k) - cy, ly[0], ly[1], ly[2]);
                    val = 0.f;
                    for (int b = 0; b < 3; ++b)
                        for (int aa = 0; aa < 3; ++aa) val = fmaf(lx[aa] * ly[b], pop(st8, ids[b * 3 + aa], kp), val);
                }
            } else {
                float d[3];
                if (S.bb_mode == 0) {
                    const float4 me = ruv[p];
                    d[0] = me.x; d[1] = me.y; d[2] = me.z;
                } else if (kind == 0 && S.Wr) {
                    d[0] = d[1] = d[2] = 0.f;
                    for (int q = 0; q < KQ; ++q) {
                        const int4 id = S.idx[(size_t)q * S.n_pad + p];
                        const float4 wq = S.Wr[(size_t)((k - 1) * KQ + q) * S.n_pad + p];
                        const int ids[4] = {id.x, id.y, id.z, id.w};
                        const float ws[4] = {wq.x, wq.y, wq.z, wq.w};
                        for (int cq = 0; cq < 4; ++cq) {
                            const float4 v = ruv[ids[cq]];
                            d[0] = fmaf(ws[cq], v.x, d[0]);
                            d[1] = fmaf(ws[cq], v.y, d[1]);
                            d[2] = fmaf(ws[cq], v.z, d[2]);
                        }
                    }
                } else if (kind == 0) {
                    float pb[6];
                    basis_at(k, L.t[k - 1], pb);
                    d[0] = d[1] = d[2] = 0.f;
                    for (int q = 0; q < KQ; ++q) {
                        const int4 id = S.idx[(size_t)q * S.n_pad + p];
                        const int ids[4] = {id.x, id.y, id.z, id.w};
                        for (int c = 0; c < 4; ++c) {
                            float tcol[6], mm[6];
                            for (int aa = 0; aa < 6; ++aa) {
                                const float4 m = S.M[(size_t)(aa * KQ + q) * S.n_pad + p];
                                tcol[aa] = c == 0 ? m.x : (c == 1 ? m.y : (c == 2 ? m.z : m.w));
                            }
                            unbasis(tcol, mm);
                            float w = 0.f;
                            for (int aa = 0; aa < 6; ++aa) w = fmaf(pb[aa], mm[aa], w);
                            const float4 v = ruv[ids[c]];
                            d[0] = fmaf(w, v.x, d[0]);
                            d[1] = fmaf(w, v.y, d[1]);
                            d[2] = fmaf(w, v.z, d[2]);
                        }
                    }
                } else {
                    int ids[9];
                    lag_block(S, p, ids);
                    float lx[3], ly[3];
                    lag3(L.t[k - 1] * r * ex_of(k) - cx, lx[0], lx[1], lx[2]);
                    lag3(L.t[k - 1] * r * ey_of(k) - cy, ly[0], ly[1], ly[2]);
                    d[0] = d[1] = d[2] = 0.f;
                    for (int b = 0; b < 3; ++b)
                        for (int aa = 0; aa < 3; ++aa) {
                            const float w = lx[aa] * ly[b];
                            const float4 v = ruv[ids[b * 3 + aa]];
                            d[0] = fmaf(w, v.x, d[0]);
                            d[1] = fmaf(w, v.y, d[1]);
                            d[2] = fmaf(w, v.z, d[2]);
                        }
                }
                const float rd = 1.0f + d[0];
                val = geq(kp, d[0], rd, d[1], d[2]) + 0.5f * src(kp, rd, d[1], d[2], Cn.ax, Cn.ay);
            }
            fx += 2.0 * (double)val * ex_of(kp) * a;
            fy += 2.0 * (double)val * ey_of(kp) * a;
        }
    }
    // fixed-order block reduction
    __shared__ double sx[128], sy[128];
    sx[threadIdx.x] = fx;
    sy[threadIdx.x] = fy;
    __syncthreads();
    for (int h = 64; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sx[threadIdx.x] += sx[threadIdx.x + h];
            sy[threadIdx.x] += sy[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = sx[0];
        partial[2 * blockIdx.x + 1] = sy[0];
    }
}

__global__ void sum_pairs(int nb, const double* __restrict__ partial, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0, b = 0;
        for (int i = 0; i < nb; ++i) { a += partial[2 * i]; b += partial[2 * i + 1]; }
        out[0] = a;
        out[1] = b;
    }
}

// ------------------------------------------------------------ reductions
// Six area-weighted FP64 sums: A, rho A, ux A, uy A, |u| A, |u|^2 A.
constexpr int kRedThreads = 256;

__global__ void __launch_bounds__(kRedThreads) reduce_fields_partial(int64_t n, const float* __restrict__ rho,
                                                                      const float* __restrict__ ux,
                                                                      const float* __restrict__ uy,
                                                                      const float* __restrict__ area,
                                                                      const uint8_t* __restrict__ mask,
                                                                      double* __restrict__ partial) {
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (mask && !mask[i]) continue;
        const double a = area[i], u = ux[i], v = uy[i];
        const double m2 = u * u + v * v;
        s[0] += a;
        s[1] += (double)rho[i] * a;
        s[2] += u * a;
        s[3] += v * a;
        s[4] += sqrt(m2) * a;
        s[5] += m2 * a;
    }
    __shared__ double sh[6][kRedThreads];
#pragma unroll
    for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int h = kRedThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
#pragma unroll
            for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 6) partial[6 * (size_t)blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kRedThreads) reduce_fields_final(int nb, const double* __restrict__ partial,
                                                                    double* __restrict__ out) {
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < 6; ++q) s[q] += partial[6 * (size_t)b + q];
    __shared__ double sh[6][kRedThreads];
#pragma unroll
    for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int h = kRedThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
#pragma unroll
            for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 6) out[threadIdx.x] = sh[threadIdx.x][0];
}

// over masked nodes: sum |u - u_prev|^2, sum |u|^2, and the number of nodes
// whose density is not positive or whose fields are not finite; then copy u
// into u_prev
__global__ void __launch_bounds__(kRedThreads) change_partial(int64_t n, const float* __restrict__ rho,
                                                               const float* __restrict__ ux,
                                                               const float* __restrict__ uy,
                                                               float* __restrict__ px, float* __restrict__ py,
                                                               const uint8_t* __restrict__ mask,
                                                               double* __restrict__ partial) {
    double d = 0, m = 0, bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float u = ux[i], v = uy[i];
        if (!mask || mask[i]) {
            const float r = rho[i];
            if (!(r > 0.f) || !isfinite(r) || !isfinite(u) || !isfinite(v)) bad += 1.0;
            const double du = (double)u - px[i], dv = (double)v - py[i];
            d += du * du + dv * dv;
            m += (double)u * u + (double)v * v;
        }
        px[i] = u;
        py[i] = v;
    }
    __shared__ double sd[kRedThreads], sm[kRedThreads], sb[kRedThreads];
    sd[threadIdx.x] = d;
    sm[threadIdx.x] = m;
    sb[threadIdx.x] = bad;
    __syncthreads();
    for (int h = kRedThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sd[threadIdx.x] += sd[threadIdx.x + h];
            sm[threadIdx.x] += sm[threadIdx.x + h];
            sb[threadIdx.x] += sb[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[3 * (size_t)blockIdx.x] = sd[0];
        partial[3 * (size_t)blockIdx.x + 1] = sm[0];
        partial[3 * (size_t)blockIdx.x + 2] = sb[0];
    }
}

__global__ void sum_triples(int nb, const double* __restrict__ partial, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        for (int i = 0; i < nb; ++i) {
            a += partial[3 * i];
            b += partial[3 * i + 1];
            c += partial[3 * i + 2];
        }
        out[0] = a;
        out[1] = b;
        out[2] = c;
    }
}

}  // namespace dev

// ------------------------------------------------------------ launchers
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

// allow the staged kernel the dynamic shared memory of its two buffers
cudaError_t prepare_staged_step(int Kq, int stage_max) {
    const int smem = 4 * stage_max * (int)sizeof(float4);
    MLBM_DISPATCH_KQ_MAIN(Kq, (cudaFuncSetAttribute((const void*)dev::bgk_step_staged<KQC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)));
    return cudaGetLastError();
}

// variant v: lanes per node and minimum resident blocks (register cap)
//   0: 1 lane, no cap   1: 2 lanes, no cap   2: 2 lanes, >= 3 blocks of 256
//   3: 2 lanes, >= 4 blocks of 256
cudaError_t launch_bgk_step(const dev::Stencil& S, const float4* f8in, const float* f0in, float4* f8out,
                            float* f0out, const dev::Collide& C, int variant, cudaStream_t st) {
    if (S.n == 0) return cudaSuccess;
    const int block = 256;
    if (S.Wr) {
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
            MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::bgk_step_rbf<KQC, 1><<<blocks_for(S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C)));
        } else {
            MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::bgk_step_rbf<KQC, 2><<<blocks_for(S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C)));
        }
        return cudaGetLastError();
    }
    switch (variant) {
        case 0: MLBM_DISPATCH_KQ(S.Kq, (dev::bgk_step_kernel<KQC, 1, 1><<<blocks_for(S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        case 1: MLBM_DISPATCH_KQ(S.Kq, (dev::bgk_step_kernel<KQC, 2, 1><<<blocks_for(2 * (int64_t)S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        case 2: MLBM_DISPATCH_KQ(S.Kq, (dev::bgk_step_kernel<KQC, 2, 3><<<blocks_for(2 * (int64_t)S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        case 3: MLBM_DISPATCH_KQ(S.Kq, (dev::bgk_step_kernel<KQC, 2, 4><<<blocks_for(2 * (int64_t)S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        case 8: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_persistent<KQC, 2, 3>, 128, S.n, st, [&](int g) { dev::bgk_step_persistent<KQC, 2, 3><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); }))); break;
        case 9: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_persistent<KQC, 2, 3>, 128, S.n, st, [&](int g) { dev::bgk_step_persistent<KQC, 2, 3><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 2); }))); break;
        case 10: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_persistent<KQC, 1, 1>, 256, S.n, st, [&](int g) { dev::bgk_step_persistent<KQC, 1, 1><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); }))); break;
        case 11: MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::bgk_step_kernel<KQC, 1, 2><<<blocks_for(S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        case 12: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_persistent<KQC, 1, 2>, 256, S.n, st, [&](int g) { dev::bgk_step_persistent<KQC, 1, 2><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); }))); break;
        case 13: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_persistent<KQC, 1, 3>, 256, S.n, st, [&](int g) { dev::bgk_step_persistent<KQC, 1, 3><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); }))); break;
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
        case 25: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_persistent<KQC, 1, 2, false, 256, true>, 256, S.n, st, [&](int g) { (void)launch_pdl(dev::bgk_step_persistent<KQC, 1, 2, false, 256, true>, g, block, st, S, f8in, f0in, f8out, f0out, C, 1); }))); break;
        case 26: MLBM_DISPATCH_KQ_MAIN(S.Kq, ((void)launch_pdl(dev::bgk_step_kernel<KQC, 1, 2, false, 256, true>, blocks_for(S.n, block), block, st, S, f8in, f0in, f8out, f0out, C))); break;
        case 23: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_persistent<KQC, 1, 4, false, 128>, 128, S.n, st, [&](int g) { dev::bgk_step_persistent<KQC, 1, 4, false, 128><<<g, 128, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); }, 0, 128))); break;
        case 24: MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::bgk_step_kernel<KQC, 1, 1, false, 512><<<blocks_for(S.n, 512), 512, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        case 22: {
            if (!S.lidx) return cudaErrorInvalidValue;  // no staging structure for this context
            const size_t smem = (size_t)4 * S.stage_max * sizeof(float4);
            MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_staged<KQC>, dev::kStageTile, S.n, st, [&](int g) { dev::bgk_step_staged<KQC><<<g, block, smem, st>>>(S, f8in, f0in, f8out, f0out, C); }, smem)));
            break;
        }
        case 20: MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::bgk_step_kernel<KQC, 1, 2, true><<<blocks_for(S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C))); break;
        case 21: MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::bgk_step_persistent<KQC, 1, 1, true>, 256, S.n, st, [&](int g) { dev::bgk_step_persistent<KQC, 1, 1, true><<<g, block, 0, st>>>(S, f8in, f0in, f8out, f0out, C, 1); }))); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_tau1_step(const dev::Stencil& S, const float4* in, float4* out, const dev::Collide& C, int variant,
                             cudaStream_t st) {
    if (S.n == 0) return cudaSuccess;
    const int block = 256;
    if (S.Wr) {
        // RBF-FD stencils: variants map as for the BGK step
        if (variant == 10) {
            MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::tau1_step_rbf_persistent<KQC, 1>, 256, S.n, st, [&](int g) { dev::tau1_step_rbf_persistent<KQC, 1><<<g, block, 0, st>>>(S, in, out, C, 1); })));
        } else if (variant == 12) {
            MLBM_DISPATCH_KQ_MAIN(S.Kq, (run_persistent((const void*)dev::tau1_step_rbf_persistent<KQC, 2>, 256, S.n, st, [&](int g) { dev::tau1_step_rbf_persistent<KQC, 2><<<g, block, 0, st>>>(S, in, out, C, 1); })));
        } else if (variant == 0) {
            MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::tau1_step_rbf<KQC, 1><<<blocks_for(S.n, block), block, 0, st>>>(S, in, out, C)));
        } else {
            MLBM_DISPATCH_KQ_MAIN(S.Kq, (dev::tau1_step_rbf<KQC, 2><<<blocks_for(S.n, block), block, 0, st>>>(S, in, out, C)));
        }
        return cudaGetLastError();
    }
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

cudaError_t launch_set_bgk(int n, const int* perm, const double* f, float4* f8, float* f0, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    dev::set_bgk_from_f64<<<blocks_for(n, 256), 256, 0, st>>>(n, perm, f, f8, f0);
    return cudaGetLastError();
}
cudaError_t launch_get_bgk(int n, const int* perm, const float4* f8, const float* f0, double* f, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    dev::get_bgk_to_f64<<<blocks_for(n, 256), 256, 0, st>>>(n, perm, f8, f0, f);
    return cudaGetLastError();
}
cudaError_t launch_set_bgk_equilibrium(int n, const int* perm, const double* ru, float4* f8, float* f0,
                                       cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    dev::set_bgk_equilibrium<<<blocks_for(n, 256), 256, 0, st>>>(n, perm, ru, f8, f0);
    return cudaGetLastError();
}
cudaError_t launch_set_tau1(int n, const int* perm, const double* ru, float4* s, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    dev::set_tau1_from_f64<<<blocks_for(n, 256), 256, 0, st>>>(n, perm, ru, s);
    return cudaGetLastError();
}
cudaError_t launch_get_tau1(int n, const int* perm, const float4* s, double* ru, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    dev::get_tau1_to_f64<<<blocks_for(n, 256), 256, 0, st>>>(n, perm, s, ru);
    return cudaGetLastError();
}
cudaError_t launch_macroscopics(int model, int n, const int* perm, const float4* f8, const float* f0,
                                const float4* ruv, float ax, float ay, const uint16_t* node_sample,
                                const dev::Collide* coll, float* rho, float* ux, float* uy, double* ru,
                                cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (model == 0)
        dev::macroscopics_bgk<<<blocks_for(n, 256), 256, 0, st>>>(n, perm, f8, f0, ax, ay, node_sample, coll, rho, ux,
                                                                   uy, ru);
    else
        dev::macroscopics_tau1<<<blocks_for(n, 256), 256, 0, st>>>(n, perm, ruv, rho, ux, uy, ru);
    return cudaGetLastError();
}

int force_blocks(int n_link_nodes) { return std::max(1, std::min(256, blocks_for(n_link_nodes, 128))); }

cudaError_t launch_force(const dev::Stencil& S, int model, int n_link_nodes, const int* link_nodes,
                         const float* area_over_s2, const float4* f8, const float4* ruv, const dev::Collide& C,
                         double* partial, double* out, cudaStream_t st) {
    const int nb = force_blocks(n_link_nodes);
    MLBM_DISPATCH_KQ(S.Kq, (dev::force_kernel<KQC><<<nb, 128, 0, st>>>(S, model, n_link_nodes, link_nodes, area_over_s2, f8, ruv, C, partial)));
    dev::sum_pairs<<<1, 32, 0, st>>>(nb, partial, out);
    return cudaGetLastError();
}

int reduce_blocks(int64_t n) {
    const int64_t b = (n + 4 * dev::kRedThreads - 1) / (4 * dev::kRedThreads);
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, kReduceMaxBlocks));
}

cudaError_t launch_reduce_fields(const float* rho, const float* ux, const float* uy, const float* area,
                                 const uint8_t* mask, int64_t n, double* partial, double* out, cudaStream_t st) {
    const int nb = reduce_blocks(n);
    dev::reduce_fields_partial<<<nb, dev::kRedThreads, 0, st>>>(n, rho, ux, uy, area, mask, partial);
    dev::reduce_fields_final<<<1, dev::kRedThreads, 0, st>>>(nb, partial, out);
    return cudaGetLastError();
}

cudaError_t launch_change(const float* rho, const float* ux, const float* uy, float* px, float* py,
                          const uint8_t* mask, int64_t n, double* partial, double* out, cudaStream_t st) {
    const int nb = reduce_blocks(n);
    dev::change_partial<<<nb, dev::kRedThreads, 0, st>>>(n, rho, ux, uy, px, py, mask, partial);
    dev::sum_triples<<<1, 32, 0, st>>>(nb, partial, out);
    return cudaGetLastError();
}

}  // namespace mlbm
