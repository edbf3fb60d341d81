// Per-node device code of the fused step kernels, shared by the translation
// units that instantiate them (kernels_bgk.cu, kernels_tau1.cu,
// kernels_rbf.cu, kernels_ring1.cu).
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
#pragma once

#include <cstdint>

#include "device_common.cuh"

namespace mlbm {
namespace dev {

// ------------------------------------------------------- stencil row sources
// Where a node's streamed stencil rows (meta byte, neighbour index groups,
// matrix rows) come from: global memory (streaming loads, each row read once
// per step), or a tile that a producer warp has already copied into shared
// memory (the one-lane-per-node bulk-copy ring, variants 27-29).
struct GlobalRows {
    const int4* idx;
    const float4* M;
    const uint8_t* mt;
    int n_pad, p;
    __device__ __forceinline__ GlobalRows(const Stencil& S, int p_)
        : idx(S.idx), M(S.M), mt(S.meta), n_pad(S.n_pad), p(p_) {}
    __device__ __forceinline__ uint8_t meta() const { return mt[p]; }
    __device__ __forceinline__ int4 idx_row(int q) const { return ld_stream(idx + (size_t)q * n_pad + p); }
    __device__ __forceinline__ float4 m_row(int r) const { return ld_stream(M + (size_t)r * n_pad + p); }
    __device__ __forceinline__ void lag(int* ids) const {
        const int4 i0 = __ldg(idx + p), i1 = __ldg(idx + (size_t)n_pad + p), i2 = __ldg(idx + 2 * (size_t)n_pad + p);
        ids[0] = i0.x; ids[1] = i0.y; ids[2] = i0.z; ids[3] = i0.w;
        ids[4] = i1.x; ids[5] = i1.y; ids[6] = i1.z; ids[7] = i1.w;
        ids[8] = i2.x;
    }
};

struct SmemRows {
    const float4* sM;     // [6 K/4][TN]
    const int4* sI;       // [K/4][TN]
    const uint8_t* sMeta; // [TN]
    int t, tn;
    __device__ __forceinline__ uint8_t meta() const { return sMeta[t]; }
    __device__ __forceinline__ int4 idx_row(int q) const { return sI[q * tn + t]; }
    __device__ __forceinline__ float4 m_row(int r) const { return sM[r * tn + t]; }
    __device__ __forceinline__ void lag(int* ids) const {
        const int4 i0 = sI[t], i1 = sI[tn + t], i2 = sI[2 * tn + t];
        ids[0] = i0.x; ids[1] = i0.y; ids[2] = i0.z; ids[3] = i0.w;
        ids[4] = i1.x; ids[5] = i1.y; ids[6] = i1.z; ids[7] = i1.w;
        ids[8] = i2.x;
    }
};

__device__ __forceinline__ GlobalRows rows_of(const Stencil& S, int p, const GlobalRows*) { return GlobalRows(S, p); }
__device__ __forceinline__ SmemRows rows_of(const Stencil&, int, const SmemRows* r) { return *r; }

// ------------------------------------------------------------ BGK / TRT
// LPN lanes (1 or 2) cooperate on one node: lane h takes the neighbour groups
// q = h, h + LPN, ... and the partial sums are combined with a pair shuffle.
// LINKS = false leaves out the bounce-back overrides (the split variants
// recompute the nodes with links in a second pass); RBF = true interpolates
// the least-squares-kind nodes with their stored RBF-FD weights.  SPEC = true
// loads the first three index rows and the rest population before the node
// kind is known (they are read by every stencil kind), so they are in flight
// together with the meta byte
template <int KQ, int LPN, bool LINKS = true, bool RBF = false, bool SPEC = false, class Rows = GlobalRows>
__device__ __forceinline__ void bgk_node(const Stencil& S, const float4* __restrict__ f8in,
                                         const float* __restrict__ f0in, float4* __restrict__ f8out,
                                         float* __restrict__ f0out, const Collide& C0, int p, int h, unsigned grp,
                                         const Rows* rows = nullptr) {
    const Rows R = rows_of(S, p, rows);
    const Collide C = collide_of(S, C0, p);
    const uint8_t meta = R.meta();
    const int kind = meta & 3;
    int4 idv[(KQ + LPN - 1) / LPN];
    float f0own = 0.f;
    if (SPEC) {
#pragma unroll
        for (int i = 0; i < (KQ + LPN - 1) / LPN; ++i) {
            const int q = i * LPN + h;
            if (q < KQ && q < 3) idv[i] = R.idx_row(q);
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
                if (q < KQ && (!SPEC || q >= 3)) idv[i] = R.idx_row(q);
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
                if (q < KQ && (!SPEC || q >= 3)) idv[i] = R.idx_row(q);
            }
#pragma unroll
            for (int i = 0; i < (KQ + LPN - 1) / LPN; ++i) {
                const int q = i * LPN + h;
                if (q < KQ) {
                    const int4 id = idv[i];
                    float4 m[6];
#pragma unroll
                    for (int a = 0; a < 6; ++a) m[a] = R.m_row(a * KQ + q);
                    wls_acc(f8in, id.x, m[0].x, m[1].x, m[2].x, m[3].x, m[4].x, m[5].x, oa, ob, acc);
                    wls_acc(f8in, id.y, m[0].y, m[1].y, m[2].y, m[3].y, m[4].y, m[5].y, oa, ob, acc);
                    wls_acc(f8in, id.z, m[0].z, m[1].z, m[2].z, m[3].z, m[4].z, m[5].z, oa, ob, acc);
                    wls_acc(f8in, id.w, m[0].w, m[1].w, m[2].w, m[3].w, m[4].w, m[5].w, oa, ob, acc);
                }
            }
        } else {
            int ids[9];
            R.lag(ids);
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
template <int KQ, int LPN, bool RBF = false, class Rows = GlobalRows>
__device__ __forceinline__ void tau1_node(const Stencil& S, const float4* __restrict__ in, float4* __restrict__ out,
                                          const Collide& C0, int p, int h, unsigned grp, const Rows* rows = nullptr) {
    const Rows R = rows_of(S, p, rows);
    const Collide C = collide_of(S, C0, p);
    const uint8_t meta = R.meta();
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
        for (int q = 0; q < KQ; ++q) idv[q] = R.idx_row(q);
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
            if (q < KQ) idv[i] = R.idx_row(q);
        }
#pragma unroll
        for (int i = 0; i < (KQ + LPN - 1) / LPN; ++i) {
            const int q = i * LPN + h;
            if (q < KQ) {
                const int4 id = idv[i];
                float4 m[6];
#pragma unroll
                for (int a = 0; a < 6; ++a) m[a] = R.m_row(a * KQ + q);
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
        R.lag(ids);
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

// ---- BGK step grids (instantiated in kernels_bgk.cu and kernels_bgk_generic.cu)
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

}  // namespace dev
}  // namespace mlbm
