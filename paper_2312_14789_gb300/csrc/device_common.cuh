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
};

struct Collide {
    float omega_p, omega_m;  // 1/tau+, 1/tau-
    float src_p, src_m;      // 1 - 1/(2 tau+), 1 - 1/(2 tau-)
    float ax, ay;            // body acceleration
};

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

}  // namespace dev
}  // namespace mlbm
