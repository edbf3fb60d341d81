// State I/O, macroscopic fields, the momentum-exchange force and the FP64
// reductions; the step kernels are in kernels_bgk.cu, kernels_tau1.cu,
// kernels_rbf.cu, kernels_ring1.cu and kernels_tma.cu.
//
// All population values are stored minus their weight omega_k (and rho as
// rho - 1) so that FP32 keeps the small deviations that carry the flow.
#include <cstdio>

#include "device_common.cuh"
#include "kernels.h"
#include "launch_util.cuh"

namespace mlbm {
namespace dev {

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
    if (S.Kq > 8) {
        MLBM_DISPATCH_KQ_RBF(S.Kq, (dev::force_kernel<KQC><<<nb, 128, 0, st>>>(S, model, n_link_nodes, link_nodes, area_over_s2, f8, ruv, C, partial)));
    } else {
        MLBM_DISPATCH_KQ(S.Kq, (dev::force_kernel<KQC><<<nb, 128, 0, st>>>(S, model, n_link_nodes, link_nodes, area_over_s2, f8, ruv, C, partial)));
    }
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
