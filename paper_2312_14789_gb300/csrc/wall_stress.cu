// Wall force by integrating the fluid stress along the wall nodes: an
// alternative to the momentum exchange over bounce-back links, for node sets
// whose walls carry nodes on the surface.
#include <cmath>

#include "kernels.h"

namespace mlbm {
namespace dev {

// (rho - 1, ux, uy) of node p from the current state; BGK velocities carry
// the half-force shift of the collision's moments
__device__ __forceinline__ void node_state(int model, const float4* __restrict__ f8, const float* __restrict__ f0,
                                           const float4* __restrict__ ruv, float ax, float ay, int p, double& dr,
                                           double& ux, double& uy) {
    if (model == 0) {
        const float4 a = f8[2 * (size_t)p], b = f8[2 * (size_t)p + 1];
        const double d = (double)f0[p] + ((double)a.x + a.y + a.z + a.w) + ((double)b.x + b.y + b.z + b.w);
        const double jx = ((double)a.x - a.z) + ((double)b.x - b.y) + ((double)b.w - b.z);
        const double jy = ((double)a.y - a.w) + ((double)b.x + b.y) - ((double)b.z + b.w);
        dr = d;
        ux = jx / (1.0 + d) - 0.5 * ax;
        uy = jy / (1.0 + d) - 0.5 * ay;
    } else {
        const float4 s = ruv[p];
        dr = s.x;
        ux = s.y;
        uy = s.z;
    }
}

// one thread per wall node: velocity gradient from the node's least-squares
// fit (the x and y rows of the stored matrix, in lattice units of s), stress
// sigma = -(rho - 1)/3 I + rho nu (grad u + grad u^T), traction sigma n ds / s;
// a node that is not a least-squares node gets NaN (reported by the host)
template <int KQ>
__global__ void __launch_bounds__(128) wall_traction(Stencil S, int model, const float4* __restrict__ f8,
                                                     const float* __restrict__ f0, const float4* __restrict__ ruv,
                                                     float ax, float ay, double nu, double inv_s,
                                                     const int* __restrict__ pos, const double* __restrict__ nrm,
                                                     const double* __restrict__ ds, int m, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int p = pos[i];
    if ((S.meta[p] & 3) != 0) {
        out[2 * i] = out[2 * i + 1] = nan("");
        return;
    }
    double dr, ux, uy;
    node_state(model, f8, f0, ruv, ax, ay, p, dr, ux, uy);
    double uxx = 0, uxy = 0, uyx = 0, uyy = 0;
    for (int q = 0; q < KQ; ++q) {
        const int4 id = S.idx[(size_t)q * S.n_pad + p];
        const float4 gx = S.M[(size_t)(4 * KQ + q) * S.n_pad + p];
        const float4 gy = S.M[(size_t)(5 * KQ + q) * S.n_pad + p];
        const int ids[4] = {id.x, id.y, id.z, id.w};
        const float wx[4] = {gx.x, gx.y, gx.z, gx.w};
        const float wy[4] = {gy.x, gy.y, gy.z, gy.w};
        for (int c = 0; c < 4; ++c) {
            double drj, uxj, uyj;
            node_state(model, f8, f0, ruv, ax, ay, ids[c], drj, uxj, uyj);
            const double du = uxj - ux, dv = uyj - uy;
            uxx += wx[c] * du;
            uxy += wy[c] * du;
            uyx += wx[c] * dv;
            uyy += wy[c] * dv;
        }
    }
    const double rho = 1.0 + dr, pr = dr / 3.0;
    const double sxx = -pr + 2.0 * rho * nu * uxx;
    const double syy = -pr + 2.0 * rho * nu * uyy;
    const double sxy = rho * nu * (uxy + uyx);
    const double nx = nrm[2 * i], ny = nrm[2 * i + 1], l = ds[i] * inv_s;
    out[2 * i] = (sxx * nx + sxy * ny) * l;
    out[2 * i + 1] = (sxy * nx + syy * ny) * l;
}

}  // namespace dev

#define MLBM_WS_DISPATCH(KQ, ...)                                \
    switch (KQ) {                                                \
        case 2: { constexpr int KQC = 2; __VA_ARGS__; } break;   \
        case 3: { constexpr int KQC = 3; __VA_ARGS__; } break;   \
        case 4: { constexpr int KQC = 4; __VA_ARGS__; } break;   \
        case 5: { constexpr int KQC = 5; __VA_ARGS__; } break;   \
        case 6: { constexpr int KQC = 6; __VA_ARGS__; } break;   \
        case 7: { constexpr int KQC = 7; __VA_ARGS__; } break;   \
        case 8: { constexpr int KQC = 8; __VA_ARGS__; } break;   \
        default: return cudaErrorInvalidValue;                   \
    }

cudaError_t launch_wall_traction(const dev::Stencil& S, int model, const float4* f8, const float* f0,
                                 const float4* ruv, float ax, float ay, double nu, double s, const int* pos,
                                 const double* nrm, const double* ds, int m, double* out, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    const int blocks = (m + 127) / 128;
    MLBM_WS_DISPATCH(S.Kq, (dev::wall_traction<KQC><<<blocks, 128, 0, st>>>(S, model, f8, f0, ruv, ax, ay, nu,
                                                                            1.0 / s, pos, nrm, ds, m, out)));
    return cudaGetLastError();
}

}  // namespace mlbm
