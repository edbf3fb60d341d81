// Device-side layout and helpers shared by the step, force and I/O kernels.
//
// Node data live in Hilbert order ("positions" p = 0..n-1), padded to n_pad
// (a multiple of 128) so every row of the interleaved arrays starts on a
// 512-byte boundary:
//   idx  int4   [K/4][n_pad]     neighbour positions, 4 per int4 (Lagrange
//                                nodes: slots 0..8 hold the 3x3 block, row b
//                                outer, column a inner)
//   M    float4 [6*(K/4)][n_pad] least-squares matrix in units of s: row a,
//                                neighbour group g at (a*K/4 + g)*n_pad + p
//   meta uint8  [n_pad]          bits 0-1 kind (0 WLS, 1 Lagrange, 2 equilibrium),
//                                bit 2 has bounce-back links, bits 4-7 block centre
//   lag_r float [n_pad]          s / h of the Lagrange block
//   link_slot int [n_pad], links LinkRec[]  bounce-back links of a node
//   eqv  float4 [n_pad]          (rho_b - 1, ux_b, uy_b, 0) of equilibrium nodes
// State (two buffers each):
//   BGK:  f8 float4[n_pad][2] = f_k - omega_k for k = 1..8, f0 float[n_pad]
//   TAU1: ruv float4[n_pad]   = (rho - 1, ux, uy, 0)
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mlbm {
namespace dev {

struct LinkRec {
    uint32_t mask;  // bit k: direction k is a link
    float t[8];     // departure factor 1 - 2q of direction k at t[k-1]
};

struct Collide {
    float omega_p, omega_m;  // 1/tau+, 1/tau-
    float src_p, src_m;      // 1 - 1/(2 tau+), 1 - 1/(2 tau-)
    float ax, ay;            // body acceleration
};

struct Stencil {
    int n, n_pad, K, Kq;
    int bb_mode;
    const int4* idx;
    const float4* M;
    const uint8_t* meta;
    const float* lag_r;
    const int* link_slot;
    const LinkRec* links;
    const float4* eqv;
    // batches of independent samples: sample of each node and the collision
    // parameters of each sample (both null for a single sample)
    const uint16_t* node_sample;
    const Collide* coll;
    // positions of the nodes with bounce-back links (for the split variants)
    const int* link_nodes;
    int n_link_nodes;
    // RBF-FD stencils: per-direction weights [8 K/4][n_pad] float4 (row
    // r = direction k - 1), null for the least-squares fit
    const float4* Wr;
    // neighbourhood staging (step variant 22, least-squares BGK): for each
    // tile of kStageTile consecutive nodes the sorted union of the stencil
    // members of its least-squares nodes without links (stage_ids, from
    // stage_off[tile] to stage_off[tile + 1]), at most stage_max per tile,
    // and each member's position in its tile's list as a 16-bit local index
    // [K/4][n_pad] ushort4 (slot order as idx); all null when not built
    const ushort4* lidx;
    const int* stage_off;
    const int* stage_ids;
    int stage_max;
};

// bounded waits of the bulk-copy ring kernels: time budget of one wait, and a
// test switch that makes block 0 withhold its first tile's copies
struct Wait {
    unsigned long long budget_ns;
    int withhold;
};

constexpr int kStageTile = 256;   // nodes per staged tile (one block)
constexpr int kStageMax = 1536;   // largest neighbourhood that is staged (48 KiB per buffer)

// collision parameters of node p
__device__ __forceinline__ Collide collide_of(const Stencil& S, const Collide& C0, int p) {
    return S.node_sample ? S.coll[S.node_sample[p]] : C0;
}

__device__ __forceinline__ int ex_of(int k) { return (k == 1 || k == 5 || k == 8) ? 1 : ((k == 3 || k == 6 || k == 7) ? -1 : 0); }
__device__ __forceinline__ int ey_of(int k) { return (k == 2 || k == 5 || k == 6) ? 1 : ((k == 4 || k == 7 || k == 8) ? -1 : 0); }
__device__ __forceinline__ int opp_of(int k) { return k == 0 ? 0 : ((k - 1 + 2) & 3) + 1 + (k >= 5 ? 4 : 0); }
__device__ __forceinline__ float w_of(int k) { return k == 0 ? (4.0f / 9.0f) : (k <= 4 ? (1.0f / 9.0f) : (1.0f / 36.0f)); }

// Streaming loads for data read once per step (matrix, indices): keep them
// out of L1 and mark them first for eviction in L2.
__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcs(p); }
__device__ __forceinline__ int4 ld_stream(const int4* p) { return __ldcs(p); }

// 1D quadratic Lagrange basis on {-1, 0, 1} at t
__device__ __forceinline__ void lag3(float t, float& l0, float& l1, float& l2) {
    l0 = 0.5f * t * (t - 1.0f);
    l1 = (1.0f - t) * (1.0f + t);
    l2 = 0.5f * t * (t + 1.0f);
}

// value of the quadratic basis at the departure point (in units of s) of
// direction k scaled by tt: offset tt * e_k (tt = -1 for plain streaming)
__device__ __forceinline__ void basis_at(int k, float tt, float* pb) {
    const float ux = tt * ex_of(k), uy = tt * ey_of(k);
    pb[0] = 1.0f; pb[1] = ux; pb[2] = uy; pb[3] = ux * ux; pb[4] = ux * uy; pb[5] = uy * uy;
}

// ---------------------------------------------------------------- helpers
// shifted equilibrium g_k = f_k^eq - omega_k of (rho = 1 + dr, u)
__device__ __forceinline__ float geq(int k, float dr, float rho, float ux, float uy) {
    const float eu = ex_of(k) * ux + ey_of(k) * uy;
    const float usq = ux * ux + uy * uy;
    return w_of(k) * (dr + rho * (3.0f * eu + 4.5f * eu * eu - 1.5f * usq));
}

// second-order body-force source S_k (Guo form), F = rho a
__device__ __forceinline__ float src(int k, float rho, float ux, float uy, float ax, float ay) {
    const float ex = ex_of(k), ey = ey_of(k);
    const float eu = ex * ux + ey * uy, ea = ex * ax + ey * ay;
    return w_of(k) * rho * (3.0f * ea - 3.0f * (ux * ax + uy * ay) + 9.0f * eu * ea);
}

__device__ __forceinline__ void eq_populations(float dr, float ux, float uy, float* g) {
    const float rho = 1.0f + dr;
#pragma unroll
    for (int k = 0; k < 9; ++k) g[k] = geq(k, dr, rho, ux, uy);
}

// single population k (1..8) of the BGK state at position j
__device__ __forceinline__ float pop(const float4* f8, int j, int k) {
    return __ldg(reinterpret_cast<const float*>(f8) + 8 * (size_t)j + (k - 1));
}

// The device keeps each node's 6 x K least-squares matrix (units of s) in
// the basis the D2Q9 departure points need: with m_0..m_5 the rows of M for
// p = [1, x, y, x^2, x y, y^2], the stored rows are
//   U = m0 + m3, V = m0 + m5, W = m0 + m3 + m4 + m5, W' = m0 + m3 - m4 + m5, m1, m2,
// so the weight of direction k at offset -e_k is one add or subtract:
//   w1 = U - m1, w3 = U + m1, w2 = V - m2, w4 = V + m2,
//   w5 = W - (m1 + m2), w7 = W + (m1 + m2), w6 = W' + (m1 - m2), w8 = W' - (m1 - m2).
// unbasis() recovers m0..m5 for departure points elsewhere (bounce-back).
__device__ __forceinline__ void unbasis(const float* t, float* m) {
    const float s = 0.5f * (t[2] + t[3]);
    m[0] = (t[0] + t[1]) - s;
    m[1] = t[4];
    m[2] = t[5];
    m[3] = t[0] - m[0];
    m[4] = 0.5f * (t[2] - t[3]);
    m[5] = t[1] - m[0];
}

// Accumulate one stencil node's contribution (centred on the node's own
// populations oa, ob) for the 8 moving directions; U..m2 is the node's
// column of the stored matrix.
__device__ __forceinline__ void wls_acc_diff(float a1, float a2, float a3, float a4, float a5, float a6, float a7,
                                             float a8, float U, float V, float W, float Wp, float m1, float m2,
                                             float* acc) {
    const float G = m1 + m2, Hh = m1 - m2;
    acc[0] = fmaf(-m1, a1, fmaf(U, a1, acc[0]));
    acc[1] = fmaf(-m2, a2, fmaf(V, a2, acc[1]));
    acc[2] = fmaf(m1, a3, fmaf(U, a3, acc[2]));
    acc[3] = fmaf(m2, a4, fmaf(V, a4, acc[3]));
    acc[4] = fmaf(-G, a5, fmaf(W, a5, acc[4]));
    acc[5] = fmaf(Hh, a6, fmaf(Wp, a6, acc[5]));
    acc[6] = fmaf(G, a7, fmaf(W, a7, acc[6]));
    acc[7] = fmaf(-Hh, a8, fmaf(Wp, a8, acc[7]));
}

__device__ __forceinline__ void wls_acc(const float4* __restrict__ f8, int j, float U, float V, float W, float Wp,
                                        float m1, float m2, const float4& oa, const float4& ob, float* acc) {
    const float4 ra = __ldg(f8 + 2 * (size_t)j);
    const float4 rb = __ldg(f8 + 2 * (size_t)j + 1);
    wls_acc_diff(ra.x - oa.x, ra.y - oa.y, ra.z - oa.z, ra.w - oa.w, rb.x - ob.x, rb.y - ob.y, rb.z - ob.z,
                 rb.w - ob.w, U, V, W, Wp, m1, m2, acc);
}

// RBF-FD value of population k_src of the stencil at the point whose
// weights are row r of node p (centred on the node's own value, the weights
// sum to one)
template <int KQ>
__device__ __forceinline__ float rbf_general(const Stencil& S, const float4* __restrict__ f8, int p, int r,
                                             int k_src) {
    const float own = pop(f8, p, k_src);
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
        const int4 id = __ldg(S.idx + (size_t)q * S.n_pad + p);
        const float4 w = __ldg(S.Wr + (size_t)(r * KQ + q) * S.n_pad + p);
        acc = fmaf(w.x, pop(f8, id.x, k_src) - own, acc);
        acc = fmaf(w.y, pop(f8, id.y, k_src) - own, acc);
        acc = fmaf(w.z, pop(f8, id.z, k_src) - own, acc);
        acc = fmaf(w.w, pop(f8, id.w, k_src) - own, acc);
    }
    return own + acc;
}

template <int KQ>
__device__ __forceinline__ float wls_general(const Stencil& S, const float4* __restrict__ f8, int p, int k_src,
                                             const float* pb) {
    const float own = pop(f8, p, k_src);
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
        const int4 id = __ldg(S.idx + (size_t)q * S.n_pad + p);
        float4 m[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) m[a] = __ldg(S.M + (size_t)(a * KQ + q) * S.n_pad + p);
        const int ids[4] = {id.x, id.y, id.z, id.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float* mc = reinterpret_cast<const float*>(m);
            float tcol[6], mm[6];
#pragma unroll
            for (int a = 0; a < 6; ++a) tcol[a] = mc[4 * a + c];
            unbasis(tcol, mm);
            float w = 0.f;
#pragma unroll
            for (int a = 0; a < 6; ++a) w = fmaf(pb[a], mm[a], w);
            acc = fmaf(w, pop(f8, ids[c], k_src) - own, acc);
        }
    }
    return own + acc;
}

__device__ __forceinline__ void lag_block(const Stencil& S, int p, int* ids) {
    const int4 i0 = __ldg(S.idx + p);
    const int4 i1 = __ldg(S.idx + (size_t)S.n_pad + p);
    const int4 i2 = __ldg(S.idx + 2 * (size_t)S.n_pad + p);
    ids[0] = i0.x; ids[1] = i0.y; ids[2] = i0.z; ids[3] = i0.w;
    ids[4] = i1.x; ids[5] = i1.y; ids[6] = i1.z; ids[7] = i1.w;
    ids[8] = i2.x;
}

// Error-free FP32 transforms (Knuth TwoSum, FMA-based product error).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (hi, lo) + (hi, lo), not renormalised
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& sh, float& sl) {
    float e;
    two_sum(ah, bh, sh, e);
    sl = e + al + bl;
}

// Moments of the streamed populations g[0..8] (shifted), then the TRT update
// (Eq. (3)-(5); BGK when omega_m == omega_p) of the pairs (k, k') = (1,3),
// (2,4), (5,7), (6,8) selected by bit pr of pair_mask, and of k = 0 when
// do_rest is set.  Lanes that share a node split the pairs between them.
//
// The update is formed as an increment g*_k = g_k + Delta_k computed only
// from small quantities, so FP32 keeps mass and momentum to round-off of the
// non-equilibrium part: the momentum-sized parts -- the pair differences
// g_k - g_k' and J = rho u = sum g e + F/2 -- are carried as exact (hi, lo)
// pairs, and the antisymmetric non-equilibrium part
//   g_k^- - g_k^{eq-} = (g_k - g_k')/2 - 3 w_k e_k . J
// is evaluated from them before rounding.  (With a plain FP32 u = j/rho +
// g/2 the rounding of u acts as a steady momentum source that the slow
// viscous modes amplify to ~1e-5 relative error in a Poiseuille channel.)
__device__ __forceinline__ void collide_pairs(float* g, const Collide& C, unsigned pair_mask, bool do_rest) {
    float dr = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) dr += g[k];
    const float rho = 1.0f + dr;
    // exact pair differences d_pr = g_k - g_k'
    float dh[4], dl[4];
    two_sum(g[1], -g[3], dh[0], dl[0]);
    two_sum(g[2], -g[4], dh[1], dl[1]);
    two_sum(g[5], -g[7], dh[2], dl[2]);
    two_sum(g[6], -g[8], dh[3], dl[3]);
    const float Fx = rho * C.ax, Fy = rho * C.ay;
    // J = rho u: Jx = d13 + d57 - d68 + Fx/2, Jy = d24 + d57 + d68 + Fy/2
    float jxh, jxl, jyh, jyl;
    df_add(dh[0], dl[0], dh[2], dl[2], jxh, jxl);
    df_add(jxh, jxl, -dh[3], -dl[3], jxh, jxl);
    df_add(jxh, jxl, 0.5f * Fx, 0.f, jxh, jxl);
    df_add(dh[1], dl[1], dh[2], dl[2], jyh, jyl);
    df_add(jyh, jyl, dh[3], dl[3], jyh, jyl);
    df_add(jyh, jyl, 0.5f * Fy, 0.f, jyh, jyl);
    const float inv = 1.0f / rho;
    const float ux = jxh * inv, uy = jyh * inv;
    const float usq = ux * ux + uy * uy;
    const float ua = ux * C.ax + uy * C.ay;
    if (do_rest) {
        const float e0 = (4.0f / 9.0f) * (dr - rho * 1.5f * usq);
        const float s0 = (4.0f / 9.0f) * rho * (-3.0f * ua);
        g[0] = g[0] + (-C.omega_p * (g[0] - e0) + C.src_p * s0);
    }
#pragma unroll
    for (int pr = 0; pr < 4; ++pr) {
        if (!((pair_mask >> pr) & 1u)) continue;
        const int k = pr < 2 ? pr + 1 : pr + 3;
        const int kp = k + 2;
        const float w = w_of(k);
        const float ex = ex_of(k), ey = ey_of(k);
        const float eu = ex * ux + ey * uy, ea = ex * C.ax + ey * C.ay;
        const float gp = 0.5f * (g[k] + g[kp]);
        const float ep = w * (dr + rho * (4.5f * eu * eu - 1.5f * usq));
        // e_k . J as (hi, lo)
        float eh, el;
        if (pr == 0) { eh = jxh; el = jxl; }
        else if (pr == 1) { eh = jyh; el = jyl; }
        else if (pr == 2) df_add(jxh, jxl, jyh, jyl, eh, el);
        else df_add(-jxh, -jxl, jyh, jyl, eh, el);
        // g^- - g^{eq-} = c (a d - e.J): a = 3/2, c = 1/3 on the axes; a = 6, c = 1/12 on the diagonals
        const float af = pr < 2 ? 1.5f : 6.0f;
        const float cf = pr < 2 ? (1.0f / 3.0f) : (1.0f / 12.0f);
        const float pa = __fmul_rn(af, dh[pr]);
        const float pe = __fmaf_rn(af, dh[pr], -pa);
        const float A = __fsub_rn(pa, eh) + ((pe + af * dl[pr]) - el);
        const float nm = cf * A;
        const float sp = w * rho * (9.0f * eu * ea - 3.0f * ua);
        const float sm = w * rho * 3.0f * ea;
        const float rp = -C.omega_p * (gp - ep) + C.src_p * sp;
        const float rm = -C.omega_m * nm + C.src_m * sm;
        g[k] = g[k] + (rp + rm);
        g[kp] = g[kp] + (rp - rm);
    }
}

// tau = 1: contribution of arriving direction k to the mass / momentum change.
// The departure values are the node's own (dr, u) plus small interpolated
// increments (a, bx, by); sk = k, or k' on a bounce-back link.  The large
// term 3 w e . (rho u) of the own node cancels between opposite directions
// and is kept out of the sums (its momentum, rho u, is added back
// analytically); a link flips its sign, hence the -2 L term.  Accumulates
// into dm (mass change), mx, my (momentum change).
__device__ __forceinline__ void tau1_accumulate(int k, int sk, bool is_link, float a, float bx, float by,
                                                float rhox, float uxx, float uyx, const Collide& C, float& dm,
                                                float& mx, float& my) {
    const float rd = rhox + a;
    const float udx = uxx + bx, udy = uyx + by;
    const float cx = a * uxx + rhox * bx + a * bx;
    const float cy = a * uyx + rhox * by + a * by;
    const float ex = ex_of(sk), ey = ey_of(sk), w = w_of(sk);
    const float eu = ex * udx + ey * udy, usq = udx * udx + udy * udy;
    const float ea = ex * C.ax + ey * C.ay;
    float R = w * (a + 3.0f * (ex * cx + ey * cy) + rd * (4.5f * eu * eu - 1.5f * usq)) +
              0.5f * w * rd * (3.0f * ea - 3.0f * (udx * C.ax + udy * C.ay) + 9.0f * eu * ea);
    if (is_link) R -= 2.0f * 3.0f * w_of(k) * (ex_of(k) * rhox * uxx + ey_of(k) * rhox * uyx);
    dm += R;
    mx += R * ex_of(k);
    my += R * ey_of(k);
}

template <int LPN>
__device__ __forceinline__ void collide_part(float* g, const Collide& C, int h) {
    if (LPN == 1) collide_pairs(g, C, 0xFu, true);
    else collide_pairs(g, C, h == 0 ? 0x3u : 0xCu, h == 0);
}

}  // namespace dev
}  // namespace mlbm
