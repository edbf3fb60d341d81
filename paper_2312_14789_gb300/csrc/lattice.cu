// Lattice LBM on a regular nx x ny grid: the comparison method of the paper
// (Sec. 2.1, Eq. (1)-(3): streaming by one lattice spacing per step, then
// collision), with the same FP32 collision as the meshless step (shifted
// populations g = f - w, TRT/BGK with the second-order source, conservative
// pair form).  Cells are fluid, solid (half-way bounce-back on the links
// that come from a solid cell: g_k(x) = g*_k'(x)) or equilibrium (g =
// g^eq(rho_b, u_b) every step).  Layout: one plane of n = nx ny floats per
// population (k = 0..8), row-major cells, two buffers; a step is one pull
// kernel, thread per cell.
#include <cmath>
#include <string>
#include <vector>

#include "kernels.h"
#include "mlbm_internal.h"

namespace mlbm {
namespace dev {

enum : uint8_t { kCellFluid = 0, kCellSolid = 1, kCellEq = 2 };

__global__ void __launch_bounds__(256) lattice_step(int nx, int ny, int px, int py,
                                                    const uint8_t* __restrict__ cell,
                                                    const float4* __restrict__ eqv, const float* __restrict__ fin,
                                                    float* __restrict__ fout, Collide C) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= nx) return;
    const size_t n = (size_t)nx * ny;
    const size_t i = (size_t)y * nx + x;
    const uint8_t c = cell[i];
    float g[9];
    if (c == kCellSolid) {
        return;
    } else if (c == kCellEq) {
        const float4 e = eqv[i];
        eq_populations(e.x, e.y, e.z, g);
    } else {
        g[0] = fin[i];
#pragma unroll
        for (int k = 1; k < 9; ++k) {
            int sx = x - ex_of(k), sy = y - ey_of(k);
            bool inside = true;
            if (sx < 0 || sx >= nx) {
                if (px) sx = (sx + nx) % nx;
                else inside = false;
            }
            if (sy < 0 || sy >= ny) {
                if (py) sy = (sy + ny) % ny;
                else inside = false;
            }
            const size_t j = (size_t)sy * nx + sx;
            // a link from outside a non-periodic side or from a solid cell bounces back
            if (!inside || cell[j] == kCellSolid) g[k] = fin[(size_t)opp_of(k) * n + i];
            else g[k] = fin[(size_t)k * n + j];
        }
        collide_pairs(g, C, 0xFu, true);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) fout[(size_t)k * n + i] = g[k];
}

// momentum exchange on the bounce-back links of the state `st` (post
// collision): a link (x, k) whose source x - e_k is solid receives
// g*_k'(x), and the body takes 2 g*_k'(x) e_k' (populations relative to the
// rest state, as for the meshless wall force)
__global__ void __launch_bounds__(256) lattice_force(int nx, int ny, int px, int py,
                                                     const uint8_t* __restrict__ cell, const float* __restrict__ st,
                                                     double* __restrict__ partial) {
    const size_t n = (size_t)nx * ny;
    double fx = 0.0, fy = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (cell[i] != kCellFluid) continue;
        const int x = (int)(i % nx), y = (int)(i / nx);
        for (int k = 1; k < 9; ++k) {
            int sx = x - ex_of(k), sy = y - ey_of(k);
            if (sx < 0 || sx >= nx) {
                if (!px) continue;
                sx = (sx + nx) % nx;
            }
            if (sy < 0 || sy >= ny) {
                if (!py) continue;
                sy = (sy + ny) % ny;
            }
            if (cell[(size_t)sy * nx + sx] != kCellSolid) continue;
            const int kp = opp_of(k);
            const double v = st[(size_t)kp * n + i];
            fx += 2.0 * v * ex_of(kp);
            fy += 2.0 * v * ey_of(kp);
        }
    }
    __shared__ double sx_[256], sy_[256];
    sx_[threadIdx.x] = fx;
    sy_[threadIdx.x] = fy;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sx_[threadIdx.x] += sx_[threadIdx.x + h];
            sy_[threadIdx.x] += sy_[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = sx_[0];
        partial[2 * blockIdx.x + 1] = sy_[0];
    }
}

__global__ void lattice_sum_pairs(int nb, const double* __restrict__ partial, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nb; ++i) {
        a += partial[2 * i];
        b += partial[2 * i + 1];
    }
    out[0] = a;
    out[1] = b;
}

// populations (FP64, [n][9], unshifted) <-> state planes (FP32, shifted)
__global__ void lattice_set(size_t n, const double* __restrict__ f, float* __restrict__ st) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int k = 0; k < 9; ++k) st[(size_t)k * n + i] = (float)(f[9 * i + k] - (double)w_of(k));
}

__global__ void lattice_get(size_t n, const float* __restrict__ st, double* __restrict__ f) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int k = 0; k < 9; ++k) f[9 * i + k] = (double)st[(size_t)k * n + i] + (double)w_of(k);
}

}  // namespace dev
}  // namespace mlbm

using namespace mlbm;

struct mlbm_lattice {
    int nx = 0, ny = 0, px = 0, py = 0;
    mlbm_params params{};
    dev::Collide C{};
    uint8_t* cell = nullptr;
    float4* eqv = nullptr;
    float* f[2] = {nullptr, nullptr};
    double* io = nullptr;
    double* partial = nullptr;
    double* small = nullptr;
    int cur = 0;
    int64_t steps = 0;
    cudaStream_t stream = nullptr;
};

namespace {
#define LAT_CUDA(call)                                                                                        \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess) return set_error(MLBM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
constexpr int kForceBlocks = 264;

void free_lattice(mlbm_lattice* L) {
    if (!L) return;
    cudaFree(L->cell);
    cudaFree(L->eqv);
    cudaFree(L->f[0]);
    cudaFree(L->f[1]);
    cudaFree(L->io);
    cudaFree(L->partial);
    cudaFree(L->small);
    if (L->stream) cudaStreamDestroy(L->stream);
    delete L;
}
}  // namespace

extern "C" {

mlbm_status mlbm_lattice_init(mlbm_lattice** out, int nx, int ny, int periodic_x, int periodic_y,
                              const uint8_t* cell, const double* eq_values, const mlbm_params* p) {
    clear_error();
    // rows map to the grid's y dimension (at most 65535)
    if (!out || !cell || !p || nx < 1 || ny < 1 || ny > 65535 || (int64_t)nx * ny > (int64_t(1) << 31) - 1)
        return set_error(MLBM_E_INVALID, "lattice_init: bad arguments (1 <= ny <= 65535, nx ny < 2^31)");
    *out = nullptr;
    if (p->model != MLBM_MODEL_BGK || !(p->tau > 0.5) || (p->tau_minus > 0 && !(p->tau_minus > 0.5)) ||
        !std::isfinite(p->gx) || !std::isfinite(p->gy))
        return set_error(MLBM_E_INVALID, "lattice_init: BGK/TRT parameters with tau > 1/2 needed");
    const size_t n = (size_t)nx * ny;
    bool has_eq = false;
    for (size_t i = 0; i < n; ++i) {
        if (cell[i] > 2) return set_error(MLBM_E_INVALID, "lattice_init: cell types are 0, 1, 2");
        has_eq |= cell[i] == 2;
    }
    if (has_eq && !eq_values) return set_error(MLBM_E_INVALID, "lattice_init: equilibrium cells need eq_values");
    auto* L = new (std::nothrow) mlbm_lattice;
    if (!L) return set_error(MLBM_E_OOM, "lattice_init: out of host memory");
    L->nx = nx;
    L->ny = ny;
    L->px = periodic_x != 0;
    L->py = periodic_y != 0;
    L->params = *p;
    const double tp = p->tau, tm = p->tau_minus > 0 ? p->tau_minus : p->tau;
    L->C.omega_p = (float)(1.0 / tp);
    L->C.omega_m = (float)(1.0 / tm);
    L->C.src_p = (float)(1.0 - 0.5 / tp);
    L->C.src_m = (float)(1.0 - 0.5 / tm);
    L->C.ax = (float)p->gx;
    L->C.ay = (float)p->gy;
    std::vector<float4> he(n, make_float4(0, 0, 0, 0));
    if (eq_values)
        for (size_t i = 0; i < n; ++i)
            if (cell[i] == 2)
                he[i] = make_float4((float)(eq_values[3 * i] - 1.0), (float)eq_values[3 * i + 1],
                                    (float)eq_values[3 * i + 2], 0.f);
    cudaError_t e = cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&L->cell, n);
    if (e == cudaSuccess) e = cudaMalloc(&L->eqv, n * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&L->f[0], 9 * n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&L->f[1], 9 * n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&L->io, 9 * n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&L->partial, 2 * kForceBlocks * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&L->small, 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(L->cell, cell, n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L->eqv, he.data(), n * sizeof(float4), cudaMemcpyHostToDevice);
    // rest state (shifted populations zero), equilibrium cells at their values
    if (e == cudaSuccess) e = cudaMemset(L->f[0], 0, 9 * n * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(L->f[1], 0, 9 * n * sizeof(float));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        free_lattice(L);
        return set_error(MLBM_E_CUDA, std::string("lattice_init: ") + cudaGetErrorString(e));
    }
    *out = L;
    return MLBM_OK;
}

void mlbm_lattice_destroy(mlbm_lattice* L) { free_lattice(L); }

mlbm_status mlbm_lattice_step(mlbm_lattice* L, int64_t n_steps) {
    if (!L || n_steps < 0) return set_error(MLBM_E_INVALID, "lattice_step: bad arguments");
    const dim3 block(256), grid((L->nx + 255) / 256, L->ny);
    for (int64_t s = 0; s < n_steps; ++s) {
        dev::lattice_step<<<grid, block, 0, L->stream>>>(L->nx, L->ny, L->px, L->py, L->cell, L->eqv, L->f[L->cur],
                                                         L->f[1 - L->cur], L->C);
        L->cur = 1 - L->cur;
    }
    LAT_CUDA(cudaGetLastError());
    L->steps += n_steps;
    return MLBM_OK;
}

mlbm_status mlbm_lattice_time_steps(mlbm_lattice* L, int64_t n_steps, double* ms) {
    if (!L || n_steps < 1 || !ms) return set_error(MLBM_E_INVALID, "lattice_time_steps: bad arguments");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LAT_CUDA(cudaEventCreate(&e0));
    LAT_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, L->stream);
    mlbm_status st = mlbm_lattice_step(L, n_steps);
    cudaEventRecord(e1, L->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MLBM_OK) return st;
    if (e != cudaSuccess) return set_error(MLBM_E_CUDA, std::string("lattice_time_steps: ") + cudaGetErrorString(e));
    *ms = t;
    return MLBM_OK;
}

mlbm_status mlbm_lattice_sync(mlbm_lattice* L) {
    if (!L) return set_error(MLBM_E_INVALID, "lattice_sync: NULL lattice");
    LAT_CUDA(cudaStreamSynchronize(L->stream));
    return MLBM_OK;
}

mlbm_status mlbm_lattice_set_populations(mlbm_lattice* L, const double* f) {
    if (!L || !f) return set_error(MLBM_E_INVALID, "lattice_set_populations: NULL argument");
    const size_t n = (size_t)L->nx * L->ny;
    LAT_CUDA(cudaMemcpyAsync(L->io, f, 9 * n * sizeof(double), cudaMemcpyHostToDevice, L->stream));
    dev::lattice_set<<<(unsigned)((n + 255) / 256), 256, 0, L->stream>>>(n, L->io, L->f[L->cur]);
    LAT_CUDA(cudaGetLastError());
    LAT_CUDA(cudaStreamSynchronize(L->stream));
    L->steps = 0;
    return MLBM_OK;
}

mlbm_status mlbm_lattice_get_populations(mlbm_lattice* L, double* f) {
    if (!L || !f) return set_error(MLBM_E_INVALID, "lattice_get_populations: NULL argument");
    const size_t n = (size_t)L->nx * L->ny;
    dev::lattice_get<<<(unsigned)((n + 255) / 256), 256, 0, L->stream>>>(n, L->f[L->cur], L->io);
    LAT_CUDA(cudaGetLastError());
    LAT_CUDA(cudaMemcpyAsync(f, L->io, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    LAT_CUDA(cudaStreamSynchronize(L->stream));
    return MLBM_OK;
}

mlbm_status mlbm_lattice_force(mlbm_lattice* L, double* fx, double* fy) {
    if (!L) return set_error(MLBM_E_INVALID, "lattice_force: NULL lattice");
    dev::lattice_force<<<kForceBlocks, 256, 0, L->stream>>>(L->nx, L->ny, L->px, L->py, L->cell, L->f[L->cur],
                                                            L->partial);
    dev::lattice_sum_pairs<<<1, 32, 0, L->stream>>>(kForceBlocks, L->partial, L->small);
    LAT_CUDA(cudaGetLastError());
    double h[2];
    LAT_CUDA(cudaMemcpyAsync(h, L->small, 16, cudaMemcpyDeviceToHost, L->stream));
    LAT_CUDA(cudaStreamSynchronize(L->stream));
    if (fx) *fx = h[0];
    if (fy) *fy = h[1];
    return MLBM_OK;
}

}  // extern "C"
