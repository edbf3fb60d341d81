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
#include <cstdio>

#include "device_common.cuh"
#include "kernels.h"

namespace mlbm {
namespace dev {

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

// TRT collision of shifted populations g[0..8] in place (BGK when omega_m == omega_p)
__device__ __forceinline__ void collide(float* g, const Collide& C) {
    float dr = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) dr += g[k];
    const float rho = 1.0f + dr;
    const float jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
    const float jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
    const float inv = 1.0f / rho;
    const float ux = jx * inv + 0.5f * C.ax, uy = jy * inv + 0.5f * C.ay;
    const float usq = ux * ux + uy * uy;
    const float ua = ux * C.ax + uy * C.ay;
    // k = 0
    {
        const float e0 = (4.0f / 9.0f) * (dr - rho * 1.5f * usq);
        const float s0 = (4.0f / 9.0f) * rho * (-3.0f * ua);
        g[0] = g[0] - C.omega_p * (g[0] - e0) + C.src_p * s0;
    }
    // pairs (k, k') = (1,3), (2,4), (5,7), (6,8)
#pragma unroll
    for (int pr = 0; pr < 4; ++pr) {
        const int k = pr < 2 ? pr + 1 : pr + 3;
        const int kp = k + 2;
        const float w = w_of(k);
        const float ex = ex_of(k), ey = ey_of(k);
        const float eu = ex * ux + ey * uy, ea = ex * C.ax + ey * C.ay;
        const float ep = w * (dr + rho * (4.5f * eu * eu - 1.5f * usq));
        const float em = w * rho * 3.0f * eu;
        const float sp = w * rho * (9.0f * eu * ea - 3.0f * ua);
        const float sm = w * rho * 3.0f * ea;
        const float gp = 0.5f * (g[k] + g[kp]), gm = 0.5f * (g[k] - g[kp]);
        const float rp = -C.omega_p * (gp - ep) + C.src_p * sp;
        const float rm = -C.omega_m * (gm - em) + C.src_m * sm;
        g[k] = g[k] + rp + rm;
        g[kp] = g[kp] + rp - rm;
    }
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

// Accumulate one stencil node's contribution for the 8 moving directions.
// m0..m5: the node's column of M (units of s).  Weight of direction k is
// p(-e_k)^T m with p = [1, x, y, x^2, x y, y^2].
__device__ __forceinline__ void wls_acc(const float4* __restrict__ f8, int j, float m0, float m1, float m2, float m3,
                                        float m4, float m5, float* acc) {
    const float4 a = __ldg(f8 + 2 * (size_t)j);
    const float4 b = __ldg(f8 + 2 * (size_t)j + 1);
    const float A = m0 + m3, B = m0 + m5;
    const float Cc = A + m5;
    const float D = Cc + m4, E = Cc - m4;
    const float G = m1 + m2, Hh = m1 - m2;
    acc[0] = fmaf(A - m1, a.x, acc[0]);
    acc[1] = fmaf(B - m2, a.y, acc[1]);
    acc[2] = fmaf(A + m1, a.z, acc[2]);
    acc[3] = fmaf(B + m2, a.w, acc[3]);
    acc[4] = fmaf(D - G, b.x, acc[4]);
    acc[5] = fmaf(E + Hh, b.y, acc[5]);
    acc[6] = fmaf(D + G, b.z, acc[6]);
    acc[7] = fmaf(E - Hh, b.w, acc[7]);
}

template <int KQ>
__device__ __forceinline__ float wls_general(const Stencil& S, const float4* __restrict__ f8, int p, int k_src,
                                             const float* pb) {
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
            float w = 0.f;
#pragma unroll
            for (int a = 0; a < 6; ++a) w = fmaf(pb[a], mc[4 * a + c], w);
            acc = fmaf(w, pop(f8, ids[c], k_src), acc);
        }
    }
    return acc;
}

__device__ __forceinline__ void lag_block(const Stencil& S, int p, int* ids) {
    const int4 i0 = __ldg(S.idx + p);
    const int4 i1 = __ldg(S.idx + (size_t)S.n_pad + p);
    const int4 i2 = __ldg(S.idx + 2 * (size_t)S.n_pad + p);
    ids[0] = i0.x; ids[1] = i0.y; ids[2] = i0.z; ids[3] = i0.w;
    ids[4] = i1.x; ids[5] = i1.y; ids[6] = i1.z; ids[7] = i1.w;
    ids[8] = i2.x;
}

// ------------------------------------------------------------ BGK / TRT
template <int KQ>
__global__ void __launch_bounds__(256) bgk_step_kernel(Stencil S, const float4* __restrict__ f8in,
                                                       const float* __restrict__ f0in, float4* __restrict__ f8out,
                                                       float* __restrict__ f0out, Collide C) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S.n) return;
    const uint8_t meta = S.meta[p];
    const int kind = meta & 3;
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
        if (kind == 0) {
#pragma unroll
            for (int q = 0; q < KQ; ++q) {
                const int4 id = ld_stream(S.idx + (size_t)q * S.n_pad + p);
                float4 m[6];
#pragma unroll
                for (int a = 0; a < 6; ++a) m[a] = ld_stream(S.M + (size_t)(a * KQ + q) * S.n_pad + p);
                wls_acc(f8in, id.x, m[0].x, m[1].x, m[2].x, m[3].x, m[4].x, m[5].x, acc);
                wls_acc(f8in, id.y, m[0].y, m[1].y, m[2].y, m[3].y, m[4].y, m[5].y, acc);
                wls_acc(f8in, id.z, m[0].z, m[1].z, m[2].z, m[3].z, m[4].z, m[5].z, acc);
                wls_acc(f8in, id.w, m[0].w, m[1].w, m[2].w, m[3].w, m[4].w, m[5].w, acc);
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
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const int j = ids[b * 3 + a];
                    const float4 fa = __ldg(f8in + 2 * (size_t)j);
                    const float4 fb = __ldg(f8in + 2 * (size_t)j + 1);
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
        if (meta & 4) {
            const LinkRec L = S.links[S.link_slot[p]];
            float over[8];
#pragma unroll
            for (int k = 1; k < 9; ++k) {
                over[k - 1] = acc[k - 1];
                if (!((L.mask >> k) & 1u)) continue;
                const int kp = opp_of(k);
                if (S.bb_mode == 0) {
                    over[k - 1] = pop(f8in, p, kp);
                } else if (kind == 0) {
                    float pb[6];
                    basis_at(k, L.t[k - 1], pb);
                    over[k - 1] = wls_general<KQ>(S, f8in, p, kp, pb);
                } else {
                    int ids[9];
                    lag_block(S, p, ids);
                    const float tt = L.t[k - 1];
                    float lx[3], ly[3];
                    lag3(tt * r * ex_of(k) - cx, lx[0], lx[1], lx[2]);
                    lag3(tt * r * ey_of(k) - cy, ly[0], ly[1], ly[2]);
                    float v = 0.f;
#pragma unroll
                    for (int b = 0; b < 3; ++b)
#pragma unroll
                        for (int a = 0; a < 3; ++a) v = fmaf(lx[a] * ly[b], pop(f8in, ids[b * 3 + a], kp), v);
                    over[k - 1] = v;
                }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = over[k];
        }
        g[0] = f0in[p];
#pragma unroll
        for (int k = 1; k < 9; ++k) g[k] = acc[k - 1];
        collide(g, C);
    }
    f8out[2 * (size_t)p] = make_float4(g[1], g[2], g[3], g[4]);
    f8out[2 * (size_t)p + 1] = make_float4(g[5], g[6], g[7], g[8]);
    f0out[p] = g[0];
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

template <int KQ>
__global__ void __launch_bounds__(256) tau1_step_kernel(Stencil S, const float4* __restrict__ in,
                                                        float4* __restrict__ out, Collide C) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S.n) return;
    const uint8_t meta = S.meta[p];
    const int kind = meta & 3;
    if (kind == 2) {
        out[p] = S.eqv[p];
        return;
    }
    const float4 me = in[p];
    float c[3][6];
    float4 v9[9];
    float r = 0.f, cx = 0.f, cy = 0.f;
    if (kind == 0) {
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int a = 0; a < 6; ++a) c[f][a] = 0.f;
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            const int4 id = ld_stream(S.idx + (size_t)q * S.n_pad + p);
            float4 m[6];
#pragma unroll
            for (int a = 0; a < 6; ++a) m[a] = ld_stream(S.M + (size_t)(a * KQ + q) * S.n_pad + p);
            const int ids[4] = {id.x, id.y, id.z, id.w};
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const float4 v = __ldg(in + ids[cc]);
                const float* mc = reinterpret_cast<const float*>(m);
#pragma unroll
                for (int a = 0; a < 6; ++a) {
                    const float ma = mc[4 * a + cc];
                    c[0][a] = fmaf(ma, v.x, c[0][a]);
                    c[1][a] = fmaf(ma, v.y, c[1][a]);
                    c[2][a] = fmaf(ma, v.z, c[2][a]);
                }
            }
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
    // k = 0 from the node itself
    const float rho0 = 1.0f + me.x;
    float dr = geq(0, me.x, rho0, me.y, me.z) + 0.5f * src(0, rho0, me.y, me.z, C.ax, C.ay);
    float jx = 0.f, jy = 0.f;
#pragma unroll
    for (int k = 1; k < 9; ++k) {
        const bool is_link = (L.mask >> k) & 1u;
        const int sk = is_link ? opp_of(k) : k;
        float d[3];
        if (is_link && S.bb_mode == 0) {
            d[0] = me.x; d[1] = me.y; d[2] = me.z;
        } else {
            const float tt = is_link ? L.t[k - 1] : -1.0f;
            if (kind == 0) {
                float pb[6];
                basis_at(k, tt, pb);
                eval_coeffs(c, pb, d);
            } else {
                float lx[3], ly[3];
                lag3(tt * r * ex_of(k) - cx, lx[0], lx[1], lx[2]);
                lag3(tt * r * ey_of(k) - cy, ly[0], ly[1], ly[2]);
                d[0] = d[1] = d[2] = 0.f;
#pragma unroll
                for (int b = 0; b < 3; ++b)
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float w = lx[a] * ly[b];
                        const float4 v = v9[b * 3 + a];
                        d[0] = fmaf(w, v.x, d[0]);
                        d[1] = fmaf(w, v.y, d[1]);
                        d[2] = fmaf(w, v.z, d[2]);
                    }
            }
        }
        const float rd = 1.0f + d[0];
        const float fk = geq(sk, d[0], rd, d[1], d[2]) + 0.5f * src(sk, rd, d[1], d[2], C.ax, C.ay);
        dr += fk;
        jx += fk * ex_of(k);
        jy += fk * ey_of(k);
    }
    const float rho = 1.0f + dr;
    const float inv = 1.0f / rho;
    out[p] = make_float4(dr, jx * inv + 0.5f * C.ax, jy * inv + 0.5f * C.ay, 0.f);
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
                                 const float* __restrict__ f0, float ax, float ay, float* __restrict__ rho_o,
                                 float* __restrict__ ux_o, float* __restrict__ uy_o, double* __restrict__ ru) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
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
// 2 f_k(t+1, x) e_{k'} area_x / s^2, per-block FP64 partials (fixed order).
template <int KQ>
__global__ void __launch_bounds__(128) force_kernel(Stencil S, int model, int n_link_nodes,
                                                    const int* __restrict__ link_nodes,
                                                    const float* __restrict__ area_over_s2,
                                                    const float4* __restrict__ st8, const float4* __restrict__ ruv,
                                                    Collide C, double* __restrict__ partial) {
    double fx = 0.0, fy = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_link_nodes; e += gridDim.x * blockDim.x) {
        const int p = link_nodes[e];
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
                val += w_of(kp);
            } else {
                float d[3];
                if (S.bb_mode == 0) {
                    const float4 me = ruv[p];
                    d[0] = me.x; d[1] = me.y; d[2] = me.z;
                } else if (kind == 0) {
                    float pb[6];
                    basis_at(k, L.t[k - 1], pb);
                    d[0] = d[1] = d[2] = 0.f;
                    for (int q = 0; q < KQ; ++q) {
                        const int4 id = S.idx[(size_t)q * S.n_pad + p];
                        const int ids[4] = {id.x, id.y, id.z, id.w};
                        for (int c = 0; c < 4; ++c) {
                            float w = 0.f;
                            for (int aa = 0; aa < 6; ++aa) {
                                const float4 m = S.M[(size_t)(aa * KQ + q) * S.n_pad + p];
                                const float mc = c == 0 ? m.x : (c == 1 ? m.y : (c == 2 ? m.z : m.w));
                                w = fmaf(pb[aa], mc, w);
                            }
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
                val = geq(kp, d[0], rd, d[1], d[2]) + 0.5f * src(kp, rd, d[1], d[2], C.ax, C.ay) + w_of(kp);
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

// sum |u - u_prev|^2, sum |u|^2 over masked nodes, then copy u into u_prev
__global__ void __launch_bounds__(kRedThreads) change_partial(int64_t n, const float* __restrict__ ux,
                                                               const float* __restrict__ uy,
                                                               float* __restrict__ px, float* __restrict__ py,
                                                               const uint8_t* __restrict__ mask,
                                                               double* __restrict__ partial) {
    double d = 0, m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float u = ux[i], v = uy[i];
        if (!mask || mask[i]) {
            const double du = (double)u - px[i], dv = (double)v - py[i];
            d += du * du + dv * dv;
            m += (double)u * u + (double)v * v;
        }
        px[i] = u;
        py[i] = v;
    }
    __shared__ double sd[kRedThreads], sm[kRedThreads];
    sd[threadIdx.x] = d;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int h = kRedThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sd[threadIdx.x] += sd[threadIdx.x + h];
            sm[threadIdx.x] += sm[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * (size_t)blockIdx.x] = sd[0];
        partial[2 * (size_t)blockIdx.x + 1] = sm[0];
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

cudaError_t launch_bgk_step(const dev::Stencil& S, const float4* f8in, const float* f0in, float4* f8out,
                            float* f0out, const dev::Collide& C, int block, cudaStream_t st) {
    if (S.n == 0) return cudaSuccess;
    MLBM_DISPATCH_KQ(S.Kq, (dev::bgk_step_kernel<KQC><<<blocks_for(S.n, block), block, 0, st>>>(S, f8in, f0in, f8out, f0out, C)));
    return cudaGetLastError();
}

cudaError_t launch_tau1_step(const dev::Stencil& S, const float4* in, float4* out, const dev::Collide& C, int block,
                             cudaStream_t st) {
    if (S.n == 0) return cudaSuccess;
    MLBM_DISPATCH_KQ(S.Kq, (dev::tau1_step_kernel<KQC><<<blocks_for(S.n, block), block, 0, st>>>(S, in, out, C)));
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
                                const float4* ruv, float ax, float ay, float* rho, float* ux, float* uy, double* ru,
                                cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (model == 0)
        dev::macroscopics_bgk<<<blocks_for(n, 256), 256, 0, st>>>(n, perm, f8, f0, ax, ay, rho, ux, uy, ru);
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
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1024));
}

cudaError_t launch_reduce_fields(const float* rho, const float* ux, const float* uy, const float* area,
                                 const uint8_t* mask, int64_t n, double* partial, double* out, cudaStream_t st) {
    const int nb = reduce_blocks(n);
    dev::reduce_fields_partial<<<nb, dev::kRedThreads, 0, st>>>(n, rho, ux, uy, area, mask, partial);
    dev::reduce_fields_final<<<1, dev::kRedThreads, 0, st>>>(nb, partial, out);
    return cudaGetLastError();
}

cudaError_t launch_change(const float* ux, const float* uy, float* px, float* py, const uint8_t* mask, int64_t n,
                          double* partial, double* out, cudaStream_t st) {
    const int nb = reduce_blocks(n);
    dev::change_partial<<<nb, dev::kRedThreads, 0, st>>>(n, ux, uy, px, py, mask, partial);
    dev::sum_pairs<<<1, 32, 0, st>>>(nb, partial, out);
    return cudaGetLastError();
}

}  // namespace mlbm
