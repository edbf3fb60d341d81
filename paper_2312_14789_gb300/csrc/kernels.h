// Host-side launchers of the kernels in kernels.cu.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace mlbm {

cudaError_t launch_bgk_step(const dev::Stencil& S, const float4* f8in, const float* f0in, float4* f8out,
                            float* f0out, const dev::Collide& C, int variant, cudaStream_t st);
// wall tractions of the listed wall nodes (device positions pos[m], normals
// nrm[m][2], wall lengths ds[m]) into out[m][2], FP64 (wall_stress.cu)
cudaError_t launch_wall_traction(const dev::Stencil& S, int model, const float4* f8, const float* f0,
                                 const float4* ruv, float ax, float ay, double nu, double s, const int* pos,
                                 const double* nrm, const double* ds, int m, double* out, cudaStream_t st);
// raises the dynamic shared-memory limit of the staged step kernel (variant 22)
cudaError_t prepare_staged_step(int Kq, int stage_max);
// BGK variants 0-3 (kernels_bgk_generic.cu)
cudaError_t launch_bgk_step_generic(const dev::Stencil& S, const float4* f8in, const float* f0in, float4* f8out,
                                    float* f0out, const dev::Collide& C, int variant, cudaStream_t st);
// BGK variants 14-19 and 22 (kernels_bgk_alt.cu)
cudaError_t launch_bgk_step_alt(const dev::Stencil& S, const float4* f8in, const float* f0in, float4* f8out,
                                float* f0out, const dev::Collide& C, int variant, cudaStream_t st);
// RBF-FD stencils (kernels_rbf.cu); launch_bgk_step / launch_tau1_step hand
// contexts with per-direction weights to these
cudaError_t launch_bgk_step_rbf(const dev::Stencil& S, const float4* f8in, const float* f0in, float4* f8out,
                                float* f0out, const dev::Collide& C, int variant, cudaStream_t st);
cudaError_t launch_tau1_step_rbf(const dev::Stencil& S, const float4* in, float4* out, const dev::Collide& C,
                                 int variant, cudaStream_t st);
cudaError_t launch_tau1_step(const dev::Stencil& S, const float4* in, float4* out, const dev::Collide& C, int variant,
                             cudaStream_t st);
cudaError_t launch_set_bgk(int n, const int* perm, const double* f, float4* f8, float* f0, cudaStream_t st);
cudaError_t launch_get_bgk(int n, const int* perm, const float4* f8, const float* f0, double* f, cudaStream_t st);
cudaError_t launch_set_bgk_equilibrium(int n, const int* perm, const double* ru, float4* f8, float* f0,
                                       cudaStream_t st);
cudaError_t launch_set_tau1(int n, const int* perm, const double* ru, float4* s, cudaStream_t st);
// tau = 1: holds the m nodes' states fixed in later steps by making them
// equilibrium-kind nodes whose record is their current state (run to steady
// state of a batch: samples that have converged)
cudaError_t launch_freeze_tau1(int m, uint8_t* meta, float4* eqv, const float4* state, cudaStream_t st);
cudaError_t launch_get_tau1(int n, const int* perm, const float4* s, double* ru, cudaStream_t st);
cudaError_t launch_macroscopics(int model, int n, const int* perm, const float4* f8, const float* f0,
                                const float4* ruv, float ax, float ay, const uint16_t* node_sample,
                                const dev::Collide* coll, float* rho, float* ux, float* uy, double* ru,
                                cudaStream_t st);
// persistent bulk-copy pipelined step (kernels_tma.cu), variants 4..7
bool tma_supported(int Kq);
cudaError_t launch_step_tma(int variant, int model, const dev::Stencil& S, const float4* f8in, const float* f0in,
                            float4* f8out, float* f0out, const float4* rin, float4* rout, const dev::Collide& C,
                            int* err, const dev::Wait& W, cudaStream_t st);
// persistent one-lane-per-node step with a bulk-copy ring of stencil rows
// (kernels.cu), variants 27..29
cudaError_t launch_step_ring1(int variant, int model, const dev::Stencil& S, const float4* f8in, const float* f0in,
                              float4* f8out, float* f0out, const float4* rin, float4* rout, const dev::Collide& C,
                              int* err, const dev::Wait& W, cudaStream_t st);
int force_blocks(int n_link_nodes);
cudaError_t launch_force(const dev::Stencil& S, int model, int n_link_nodes, const int* link_nodes,
                         const float* area_over_s2, const float4* f8, const float4* ruv, const dev::Collide& C,
                         double* partial, double* out, cudaStream_t st);
// the FP64 reductions never use more than this many partial-sum blocks
constexpr int kReduceMaxBlocks = 1024;
int reduce_blocks(int64_t n);
cudaError_t launch_reduce_fields(const float* rho, const float* ux, const float* uy, const float* area,
                                 const uint8_t* mask, int64_t n, double* partial, double* out, cudaStream_t st);
// per sample: sum |u - u_prev|^2, sum |u|^2 and the count of nodes with a
// non-positive density or non-finite field (3 doubles into out); u -> u_prev
cudaError_t launch_change(const float* rho, const float* ux, const float* uy, float* px, float* py,
                          const uint8_t* mask, int64_t n, double* partial, double* out, cudaStream_t st);

// warm start (features.cu)
cudaError_t launch_warm_check(int n, const int* perm, const uint16_t* node_sample, const uint8_t* meta,
                              const float* Y, int no, const double* scale_u, const double* scale_rho, float umax,
                              float drho_max, int* flag, cudaStream_t st);
cudaError_t launch_warm_drho(int n, const int* perm, const uint16_t* node_sample, const uint8_t* meta,
                             const float* Y, int no, const double* scale_rho, float* drho, cudaStream_t st);
cudaError_t launch_warm_fill(int n, const int* perm, const uint16_t* node_sample, const uint8_t* meta,
                             const float4* eqv, const float* Y, int no, const double* scale_u, const float* drho,
                             const double* drho_mean, const int* flag, double* ru, cudaStream_t st);

}  // namespace mlbm
