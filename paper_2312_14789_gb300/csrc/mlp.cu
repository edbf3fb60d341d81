// Warm-start MLP 16 -> 64 -> 64 -> 64 -> n_out (n_out <= 3, ReLU), BF16 tensor-core GEMMs with
// FP32 accumulation (mma.sync m16n8k16), training by hand-written backward
// kernels and Adam.
//
// Parameters are kept in FP32 ("master") in the packed order W1[16][64], b1,
// W2[64][64], b2, W3[64][64], b3, W4[64][n_out], b4 (y = x W + b per layer); the
// kernels convert the weights to BF16 in shared memory.  Rounding points:
// the features and every hidden activation (after bias and ReLU) are rounded
// to BF16 where they become an MMA operand; the output error and every hidden
// error likewise.  Accumulation and biases are FP32.
//
// Forward: one warp per 16-row tile; a layer's FP32 accumulator fragments are
// re-packed in registers as the next layer's A fragments.
// Gradients: blocks of 4 warps take 64-row chunks: each warp runs its 16 rows
// forward and back through the layers (dX = dZ W^T), staging activations and
// errors transposed ([feature][row], BF16) in shared memory; then the block
// computes dW = H^T dZ for the chunk with MMAs whose K dimension is the 64
// rows, each output tile owned by one warp (no atomics), and adds the bias
// sums.  Each block writes its FP32 partial gradient; a second kernel adds
// the partials in block order, so the result is reproducible run to run.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"
#include "mlbm_internal.h"

namespace mlbm {
namespace mlp {

constexpr int kIn = 16, kH = 64, kMaxOut = 3;
// packed offsets
constexpr int oW1 = 0, oB1 = oW1 + kIn * kH, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kH * kH, oW4 = oB3 + kH;
// offset of b4 and parameter count for `no` outputs (9538 for no = 2)
__host__ __device__ constexpr int off_b4(int no) { return oW4 + kH * no; }
__host__ __device__ constexpr int param_count(int no) { return off_b4(no) + no; }
static_assert(param_count(2) == 9538, "packing");

// padded shared-memory strides (BF16 elements) that keep fragment loads free of bank conflicts
constexpr int kS16 = 24, kS64 = 72;

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Forward weights, transposed [out][in] BF16, padded strides; biases FP32.
struct FwdSmem {
    __nv_bfloat16 wt1[kH * kS16];
    __nv_bfloat16 wt2[kH * kS64];
    __nv_bfloat16 wt3[kH * kS64];
    __nv_bfloat16 wt4[8 * kS64];  // outputs padded to 8
    float b1[kH], b2[kH], b3[kH], b4[8];
};

__device__ void load_fwd(const float* __restrict__ P, int no, FwdSmem& s) {
    for (int i = threadIdx.x; i < kH * kS16; i += blockDim.x) {
        const int n = i / kS16, k = i % kS16;
        s.wt1[i] = __float2bfloat16_rn(k < kIn ? P[oW1 + k * kH + n] : 0.f);
    }
    for (int i = threadIdx.x; i < kH * kS64; i += blockDim.x) {
        const int n = i / kS64, k = i % kS64;
        s.wt2[i] = __float2bfloat16_rn(k < kH ? P[oW2 + k * kH + n] : 0.f);
        s.wt3[i] = __float2bfloat16_rn(k < kH ? P[oW3 + k * kH + n] : 0.f);
    }
    for (int i = threadIdx.x; i < 8 * kS64; i += blockDim.x) {
        const int n = i / kS64, k = i % kS64;
        s.wt4[i] = __float2bfloat16_rn((k < kH && n < no) ? P[oW4 + k * no + n] : 0.f);
    }
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        s.b1[i] = P[oB1 + i];
        s.b2[i] = P[oB2 + i];
        s.b3[i] = P[oB3 + i];
    }
    if (threadIdx.x < 8) s.b4[threadIdx.x] = (int)threadIdx.x < no ? P[off_b4(no) + threadIdx.x] : 0.f;
}

// Row of the data set that minibatch row r reads: r itself (seed 0), else a
// splitmix64 hash of (seed, step, r) reduced modulo n_data.
__device__ __forceinline__ int64_t data_row(int64_t r, int64_t n_data, uint64_t seed, uint64_t step) {
    if (seed == 0) return r;
    uint64_t z = seed ^ (step * 0xD1B54A32D192ED03ull) ^ ((uint64_t)r * 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (int64_t)(z % (uint64_t)n_data);
}

// A fragment of the feature tile (rows g, g + 8 of the warp's 16 rows);
// src0 / src1: data rows of those two rows, -1 for padding
__device__ __forceinline__ void load_x(const float* __restrict__ X, int64_t src0, int64_t src1, int t, uint32_t* a) {
    float v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = 0.f;
    if (src0 >= 0) {
        const float* x = X + src0 * kIn;
        v[0] = x[2 * t]; v[1] = x[2 * t + 1];
        v[4] = x[2 * t + 8]; v[5] = x[2 * t + 9];
    }
    if (src1 >= 0) {
        const float* x = X + src1 * kIn;
        v[2] = x[2 * t]; v[3] = x[2 * t + 1];
        v[6] = x[2 * t + 8]; v[7] = x[2 * t + 9];
    }
    a[0] = pack2(v[0], v[1]);
    a[1] = pack2(v[2], v[3]);
    a[2] = pack2(v[4], v[5]);
    a[3] = pack2(v[6], v[7]);
}

// one hidden layer: A (k-tiles of the input) -> ReLU(A W + b) packed as the
// next A fragments
template <int KT>
__device__ __forceinline__ void hidden_layer(const uint32_t (*a)[4], const __nv_bfloat16* wt, int stride,
                                             const float* bias, int g, int t, uint32_t (*out)[4]) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float bl = bias[8 * nt + 2 * t], bh = bias[8 * nt + 2 * t + 1];
        float d[4] = {bl, bh, bl, bh};
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) {
            const __nv_bfloat16* w = wt + (8 * nt + g) * stride + 16 * kt + 2 * t;
            mma(d, a[kt], ld32(w), ld32(w + 8));
        }
        const float r0 = fmaxf(d[0], 0.f), r1 = fmaxf(d[1], 0.f), r2 = fmaxf(d[2], 0.f), r3 = fmaxf(d[3], 0.f);
        out[nt >> 1][(nt & 1) * 2 + 0] = pack2(r0, r1);
        out[nt >> 1][(nt & 1) * 2 + 1] = pack2(r2, r3);
    }
}

__device__ __forceinline__ void output_layer(const uint32_t (*a)[4], const FwdSmem& s, int g, int t, float* d) {
    const float bl = s.b4[2 * t], bh = s.b4[2 * t + 1];
    d[0] = bl; d[1] = bh; d[2] = bl; d[3] = bh;
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        const __nv_bfloat16* w = s.wt4 + g * kS64 + 16 * kt + 2 * t;
        mma(d, a[kt], ld32(w), ld32(w + 8));
    }
}

__global__ void __launch_bounds__(128) forward_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                      int64_t n, int no, float* __restrict__ Y) {
    __shared__ FwdSmem s;
    load_fwd(P, no, s);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t tiles = (n + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * 4 + warp; tile < tiles; tile += (int64_t)gridDim.x * 4) {
        const int64_t row0 = tile * 16;
        uint32_t a1[1][4], a2[4][4], a3[4][4], a4[4][4];
        load_x(X, row0 + g < n ? row0 + g : -1, row0 + g + 8 < n ? row0 + g + 8 : -1, t, a1[0]);
        hidden_layer<1>(a1, s.wt1, kS16, s.b1, g, t, a2);
        hidden_layer<4>(a2, s.wt2, kS64, s.b2, g, t, a3);
        hidden_layer<4>(a3, s.wt3, kS64, s.b3, g, t, a4);
        float d[4];
        output_layer(a4, s, g, t, d);
        // this lane holds output columns 2t, 2t + 1 of rows g, g + 8
        const int c0 = 2 * t, c1 = 2 * t + 1;
        if (row0 + g < n) {
            if (c0 < no) Y[(row0 + g) * no + c0] = d[0];
            if (c1 < no) Y[(row0 + g) * no + c1] = d[1];
        }
        if (row0 + g + 8 < n) {
            if (c0 < no) Y[(row0 + g + 8) * no + c0] = d[2];
            if (c1 < no) Y[(row0 + g + 8) * no + c1] = d[3];
        }
    }
}

// ------------------------------------------------------------ gradients
constexpr int kChunk = 64;  // rows per block iteration (4 warps x 16)

struct BwdSmem {
    FwdSmem f;
    // row-major [in][out] BF16 weights for dX = dZ W^T
    __nv_bfloat16 w2[kH * kS64];
    __nv_bfloat16 w3[kH * kS64];
    __nv_bfloat16 w4[kH * kS16];  // outputs padded to 16
    // staging, transposed [feature][row] BF16
    __nv_bfloat16 h0[kIn * kS64];
    __nv_bfloat16 h1[kH * kS64], h2[kH * kS64], h3[kH * kS64];
    __nv_bfloat16 dz1[kH * kS64], dz2[kH * kS64], dz3[kH * kS64];
    __nv_bfloat16 dy[8 * kS64];
    // FP32 gradient accumulators of the block
    float gw1[kIn * kH], gw2[kH * kH], gw3[kH * kH], gw4[kH * 8];
    float gb1[kH], gb2[kH], gb3[kH], gb4[8];
    double loss[4];
};

// write a warp's 16-row fragment of a [rows x 64] matrix (FP32 accumulator
// layout, 8 n-tiles) into transposed staging [col][row], BF16
__device__ __forceinline__ void stage_t(__nv_bfloat16* dst, const float (*v)[4], int rbase, int g, int t) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int c = 8 * nt + 2 * t;
        dst[c * kS64 + rbase + g] = __float2bfloat16_rn(v[nt][0]);
        dst[(c + 1) * kS64 + rbase + g] = __float2bfloat16_rn(v[nt][1]);
        dst[c * kS64 + rbase + g + 8] = __float2bfloat16_rn(v[nt][2]);
        dst[(c + 1) * kS64 + rbase + g + 8] = __float2bfloat16_rn(v[nt][3]);
    }
}

// unpack A fragments (4 k-tiles, BF16 pairs) of a [rows x 64] activation to FP32 accumulator layout
__device__ __forceinline__ void unpack_a(const uint32_t (*a)[4], float (*v)[4]) {
#pragma unroll
    for (int kt = 0; kt < 4; ++kt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int nt = 2 * kt + h;
            __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&a[kt][2 * h]);
            __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&a[kt][2 * h + 1]);
            v[nt][0] = __low2float(lo); v[nt][1] = __high2float(lo);
            v[nt][2] = __low2float(hi); v[nt][3] = __high2float(hi);
        }
}

// dA = dZ W^T for a layer with 64 inputs: dz (A fragments over the layer's
// outputs, KT k-tiles), w row-major [in][out] with the given stride
template <int KT>
__device__ __forceinline__ void back_layer(const uint32_t (*dz)[4], const __nv_bfloat16* w, int stride, int g, int t,
                                           float (*da)[4]) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) {
            const __nv_bfloat16* p = w + (8 * nt + g) * stride + 16 * kt + 2 * t;
            mma(d, dz[kt], ld32(p), ld32(p + 8));
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) da[nt][i] = d[i];
    }
}

// dZ = dA * [H > 0], rounded to BF16 and packed as A fragments
__device__ __forceinline__ void mask_pack(float (*da)[4], const float (*h)[4], uint32_t (*out)[4]) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
        for (int i = 0; i < 4; ++i) da[nt][i] = h[nt][i] > 0.f ? da[nt][i] : 0.f;
        out[nt >> 1][(nt & 1) * 2 + 0] = pack2(da[nt][0], da[nt][1]);
        out[nt >> 1][(nt & 1) * 2 + 1] = pack2(da[nt][2], da[nt][3]);
    }
}

// dW tile (16 x 8) += H^T dZ over the chunk's 64 rows; h: [feat][row], dz: [out][row]
__device__ __forceinline__ void dw_tile(const __nv_bfloat16* h, const __nv_bfloat16* dz, int mt, int nt, int g, int t,
                                        float* d) {
#pragma unroll
    for (int kt = 0; kt < kChunk / 16; ++kt) {
        const __nv_bfloat16* ap = h + (16 * mt + g) * kS64 + 16 * kt + 2 * t;
        const uint32_t a[4] = {ld32(ap), ld32(ap + 8 * kS64), ld32(ap + 8), ld32(ap + 8 * kS64 + 8)};
        const __nv_bfloat16* bp = dz + (8 * nt + g) * kS64 + 16 * kt + 2 * t;
        mma(d, a, ld32(bp), ld32(bp + 8));
    }
}

// n rows of the minibatch, drawn from n_data rows of (X, T) by data_row
__global__ void __launch_bounds__(128) grad_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                   const float* __restrict__ T, int no, int64_t n, int64_t n_data,
                                                   uint64_t seed, uint64_t step, float inv_n2,
                                                   float* __restrict__ partial, double* __restrict__ loss_partial) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    BwdSmem& s = *reinterpret_cast<BwdSmem*>(smem_raw);
    load_fwd(P, no, s.f);
    for (int i = threadIdx.x; i < kH * kS64; i += blockDim.x) {
        const int r = i / kS64, c = i % kS64;
        s.w2[i] = __float2bfloat16_rn(c < kH ? P[oW2 + r * kH + c] : 0.f);
        s.w3[i] = __float2bfloat16_rn(c < kH ? P[oW3 + r * kH + c] : 0.f);
    }
    for (int i = threadIdx.x; i < kH * kS16; i += blockDim.x) {
        const int r = i / kS16, c = i % kS16;
        s.w4[i] = __float2bfloat16_rn(c < no ? P[oW4 + r * no + c] : 0.f);
    }
    for (int i = threadIdx.x; i < kIn * kH; i += blockDim.x) s.gw1[i] = 0.f;
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) { s.gw2[i] = 0.f; s.gw3[i] = 0.f; }
    for (int i = threadIdx.x; i < kH * 8; i += blockDim.x) s.gw4[i] = 0.f;
    for (int i = threadIdx.x; i < kH; i += blockDim.x) { s.gb1[i] = 0.f; s.gb2[i] = 0.f; s.gb3[i] = 0.f; }
    if (threadIdx.x < 8) s.gb4[threadIdx.x] = 0.f;
    if (threadIdx.x < 4) s.loss[threadIdx.x] = 0.0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    double my_loss = 0.0;
    const int64_t chunks = (n + kChunk - 1) / kChunk;
    for (int64_t ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
        const int64_t row0 = ch * kChunk + warp * 16;
        const int rb = warp * 16;
        // ---- forward for the warp's 16 rows, keeping every activation
        uint32_t a1[1][4], a2[4][4], a3[4][4], a4[4][4];
        const int64_t r0 = row0 + g, r1 = row0 + g + 8;
        const int64_t src0 = r0 < n ? data_row(r0, n_data, seed, step) : -1;
        const int64_t src1 = r1 < n ? data_row(r1, n_data, seed, step) : -1;
        load_x(X, src0, src1, t, a1[0]);
        hidden_layer<1>(a1, s.f.wt1, kS16, s.f.b1, g, t, a2);
        hidden_layer<4>(a2, s.f.wt2, kS64, s.f.b2, g, t, a3);
        hidden_layer<4>(a3, s.f.wt3, kS64, s.f.b3, g, t, a4);
        float y[4];
        output_layer(a4, s.f, g, t, y);
        // ---- output error dY = 2 (Y - T) / n (zero on padding rows and
        // columns); this lane holds columns 2t, 2t + 1 of rows g, g + 8
        float dy[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = 2 * t + (q & 1);
            const int64_t src = q < 2 ? src0 : src1;
            if (c < no && src >= 0) {
                const float e = y[q] - T[src * no + c];
                my_loss += (double)e * e;
                dy[q] = inv_n2 * e;
            }
        }
        // staging of the inputs of every layer and of dY
        {
            float v[8][4];
            unpack_a(a2, v);
            stage_t(s.h1, v, rb, g, t);
            unpack_a(a3, v);
            stage_t(s.h2, v, rb, g, t);
            unpack_a(a4, v);
            stage_t(s.h3, v, rb, g, t);
            // features: rows g, g+8; cols 2t, 2t+1, 2t+8, 2t+9
            const __nv_bfloat162* xa = reinterpret_cast<const __nv_bfloat162*>(a1[0]);
            s.h0[(2 * t) * kS64 + rb + g] = xa[0].x; s.h0[(2 * t + 1) * kS64 + rb + g] = xa[0].y;
            s.h0[(2 * t) * kS64 + rb + g + 8] = xa[1].x; s.h0[(2 * t + 1) * kS64 + rb + g + 8] = xa[1].y;
            s.h0[(2 * t + 8) * kS64 + rb + g] = xa[2].x; s.h0[(2 * t + 9) * kS64 + rb + g] = xa[2].y;
            s.h0[(2 * t + 8) * kS64 + rb + g + 8] = xa[3].x; s.h0[(2 * t + 9) * kS64 + rb + g + 8] = xa[3].y;
            // dY (cols 0..7, only 0 and 1 non-zero)
            s.dy[(2 * t) * kS64 + rb + g] = __float2bfloat16_rn(dy[0]);
            s.dy[(2 * t + 1) * kS64 + rb + g] = __float2bfloat16_rn(dy[1]);
            s.dy[(2 * t) * kS64 + rb + g + 8] = __float2bfloat16_rn(dy[2]);
            s.dy[(2 * t + 1) * kS64 + rb + g + 8] = __float2bfloat16_rn(dy[3]);
        }
        // ---- back through the layers: dZ3 = (dY W4^T) * [H3 > 0], ...
        uint32_t ady[1][4] = {{pack2(dy[0], dy[1]), pack2(dy[2], dy[3]), 0u, 0u}};
        float da[8][4], hv[8][4];
        uint32_t dz3[4][4], dz2[4][4], dz1[4][4];
        back_layer<1>(ady, s.w4, kS16, g, t, da);
        unpack_a(a4, hv);
        mask_pack(da, hv, dz3);
        stage_t(s.dz3, da, rb, g, t);
        back_layer<4>(dz3, s.w3, kS64, g, t, da);
        unpack_a(a3, hv);
        mask_pack(da, hv, dz2);
        stage_t(s.dz2, da, rb, g, t);
        back_layer<4>(dz2, s.w2, kS64, g, t, da);
        unpack_a(a2, hv);
        mask_pack(da, hv, dz1);
        stage_t(s.dz1, da, rb, g, t);
        __syncthreads();
        // ---- weight gradients of the chunk: 76 output tiles, warp w takes w, w+4, ...
        for (int tile = warp; tile < 76; tile += 4) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            float* gw;
            int ld, mt, nt, ncols;
            if (tile < 8) {  // dW1 [16][64]
                mt = 0; nt = tile; gw = s.gw1; ld = kH; ncols = kH;
                dw_tile(s.h0, s.dz1, mt, nt, g, t, d);
            } else if (tile < 40) {  // dW2 [64][64]
                mt = (tile - 8) >> 3; nt = (tile - 8) & 7; gw = s.gw2; ld = kH; ncols = kH;
                dw_tile(s.h1, s.dz2, mt, nt, g, t, d);
            } else if (tile < 72) {  // dW3
                mt = (tile - 40) >> 3; nt = (tile - 40) & 7; gw = s.gw3; ld = kH; ncols = kH;
                dw_tile(s.h2, s.dz3, mt, nt, g, t, d);
            } else {  // dW4 [64][8]
                mt = tile - 72; nt = 0; gw = s.gw4; ld = 8; ncols = 8;
                dw_tile(s.h3, s.dy, mt, nt, g, t, d);
            }
            const int r = 16 * mt + g, c = 8 * nt + 2 * t;
            if (c < ncols) {
                gw[r * ld + c] += d[0];
                gw[r * ld + c + 1] += d[1];
                gw[(r + 8) * ld + c] += d[2];
                gw[(r + 8) * ld + c + 1] += d[3];
            }
        }
        // ---- bias gradients: column sums of the BF16 errors over the chunk
        for (int c = threadIdx.x; c < 3 * kH + no; c += blockDim.x) {
            const __nv_bfloat16* src;
            float* dst;
            if (c < kH) { src = s.dz1 + c * kS64; dst = &s.gb1[c]; }
            else if (c < 2 * kH) { src = s.dz2 + (c - kH) * kS64; dst = &s.gb2[c - kH]; }
            else if (c < 3 * kH) { src = s.dz3 + (c - 2 * kH) * kS64; dst = &s.gb3[c - 2 * kH]; }
            else { src = s.dy + (c - 3 * kH) * kS64; dst = &s.gb4[c - 3 * kH]; }
            float acc = 0.f;
            for (int r = 0; r < kChunk; ++r) acc += __bfloat162float(src[r]);
            *dst += acc;
        }
        __syncthreads();
    }
    // ---- loss of the block (fixed order), then the block's partial gradient
    for (int o = 16; o > 0; o >>= 1) my_loss += __shfl_xor_sync(0xffffffffu, my_loss, o);
    if (lane == 0) s.loss[warp] = my_loss;
    __syncthreads();
    float* out = partial + (size_t)blockIdx.x * param_count(no);
    for (int i = threadIdx.x; i < kIn * kH; i += blockDim.x) out[oW1 + i] = s.gw1[i];
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) {
        out[oW2 + i] = s.gw2[i];
        out[oW3 + i] = s.gw3[i];
    }
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        out[oB1 + i] = s.gb1[i];
        out[oB2 + i] = s.gb2[i];
        out[oB3 + i] = s.gb3[i];
        for (int j = 0; j < no; ++j) out[oW4 + i * no + j] = s.gw4[i * 8 + j];
    }
    if ((int)threadIdx.x < no) out[off_b4(no) + threadIdx.x] = s.gb4[threadIdx.x];
    if (threadIdx.x == 0) loss_partial[blockIdx.x] = (s.loss[0] + s.loss[1]) + (s.loss[2] + s.loss[3]);
}

__global__ void sum_partials(int nb, int kp, const float* __restrict__ partial, const double* __restrict__ loss_partial,
                             float* __restrict__ grad, double* __restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kp) {
        float acc = 0.f;
        for (int b = 0; b < nb; ++b) acc += partial[(size_t)b * kp + i];
        grad[i] = acc;
    }
    if (i == 0) {
        double l = 0.0;
        for (int b = 0; b < nb; ++b) l += loss_partial[b];
        *loss = l;
    }
}

// Adam (Kingma & Ba), bias-corrected, on the FP32 master parameters
__global__ void adam_kernel(int kp, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ grad, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kp) return;
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace mlp
}  // namespace mlbm

using namespace mlbm;

struct mlbm_mlp {
    float* p = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;
    float* partial = nullptr;
    double* loss_partial = nullptr;
    double* loss = nullptr;
    int max_blocks = 0;
    int n_out = 2;
    int kp = 0;     // parameter count
    int64_t t = 0;  // Adam step count
};

namespace {
#define MLP_CUDA(call)                                                                                \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return set_error(MLBM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double gauss(uint64_t& s) {
    const double u1 = ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}
constexpr int kMaxGradBlocks = 2 * 152;
int grad_blocks(int64_t n) {
    const int64_t chunks = (n + mlp::kChunk - 1) / mlp::kChunk;
    return (int)std::max<int64_t>(1, std::min<int64_t>(chunks, kMaxGradBlocks));
}
}  // namespace

extern "C" {

int64_t mlbm_mlp_param_count(int n_out) {
    return n_out >= 1 && n_out <= mlp::kMaxOut ? mlp::param_count(n_out) : -1;
}

int mlbm_mlp_outputs(const mlbm_mlp* m) { return m ? m->n_out : -1; }

mlbm_status mlbm_mlp_create(mlbm_mlp** out, int n_out, uint64_t seed) {
    clear_error();
    if (!out || n_out < 1 || n_out > mlp::kMaxOut) return set_error(MLBM_E_INVALID, "mlp_create: bad arguments");
    *out = nullptr;
    auto* m = new (std::nothrow) mlbm_mlp;
    if (!m) return set_error(MLBM_E_OOM, "mlp_create: out of host memory");
    m->max_blocks = kMaxGradBlocks;
    m->n_out = n_out;
    m->kp = mlp::param_count(n_out);
    cudaError_t e = cudaSuccess;
    e = e == cudaSuccess ? cudaMalloc(&m->p, m->kp * 4) : e;
    e = e == cudaSuccess ? cudaMalloc(&m->m, m->kp * 4) : e;
    e = e == cudaSuccess ? cudaMalloc(&m->v, m->kp * 4) : e;
    e = e == cudaSuccess ? cudaMalloc(&m->grad, m->kp * 4) : e;
    e = e == cudaSuccess ? cudaMalloc(&m->partial, (size_t)m->max_blocks * m->kp * 4) : e;
    e = e == cudaSuccess ? cudaMalloc(&m->loss_partial, (size_t)m->max_blocks * 8) : e;
    e = e == cudaSuccess ? cudaMalloc(&m->loss, 8) : e;
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        mlbm_mlp_destroy(m);
        return set_error(MLBM_E_CUDA, std::string("mlp_create: ") + cudaGetErrorString(e));
    }
    // He-normal weights, zero biases
    std::vector<float> h(m->kp, 0.f);
    uint64_t st = seed * 0x2545F4914F6CDD1Dull + 1;
    const int sizes[5] = {mlp::kIn, mlp::kH, mlp::kH, mlp::kH, n_out};
    int o = 0;
    for (int l = 0; l < 4; ++l) {
        const double sd = std::sqrt(2.0 / sizes[l]);
        for (int i = 0; i < sizes[l] * sizes[l + 1]; ++i) h[o + i] = (float)(sd * gauss(st));
        o += sizes[l] * sizes[l + 1] + sizes[l + 1];
    }
    mlbm_status s = mlbm_mlp_set_params(m, h.data());
    if (s != MLBM_OK) {
        std::string msg = mlbm_last_error();
        mlbm_mlp_destroy(m);
        return set_error(s, msg);
    }
    *out = m;
    return MLBM_OK;
}

void mlbm_mlp_destroy(mlbm_mlp* m) {
    if (!m) return;
    cudaFree(m->p); cudaFree(m->m); cudaFree(m->v); cudaFree(m->grad); cudaFree(m->partial);
    cudaFree(m->loss_partial); cudaFree(m->loss);
    delete m;
}

mlbm_status mlbm_mlp_set_params(mlbm_mlp* m, const float* params) {
    if (!m || !params) return set_error(MLBM_E_INVALID, "mlp_set_params: NULL argument");
    MLP_CUDA(cudaMemcpy(m->p, params, m->kp * 4, cudaMemcpyHostToDevice));
    MLP_CUDA(cudaMemset(m->m, 0, m->kp * 4));
    MLP_CUDA(cudaMemset(m->v, 0, m->kp * 4));
    m->t = 0;
    return MLBM_OK;
}

mlbm_status mlbm_mlp_get_params(mlbm_mlp* m, float* params) {
    if (!m || !params) return set_error(MLBM_E_INVALID, "mlp_get_params: NULL argument");
    MLP_CUDA(cudaMemcpy(params, m->p, m->kp * 4, cudaMemcpyDeviceToHost));
    return MLBM_OK;
}

mlbm_status mlbm_mlp_forward_device(mlbm_mlp* m, const float* X, int64_t n, float* Y, void* stream) {
    if (!m || (n > 0 && (!X || !Y)) || n < 0) return set_error(MLBM_E_INVALID, "mlp_forward: bad arguments");
    if (n == 0) return MLBM_OK;
    const int64_t tiles = (n + 15) / 16;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((tiles + 3) / 4, 152 * 8));
    mlp::forward_kernel<<<blocks, 128, 0, static_cast<cudaStream_t>(stream)>>>(m->p, X, n, m->n_out, Y);
    MLP_CUDA(cudaGetLastError());
    return MLBM_OK;
}

}  // extern "C"

namespace {
// one gradient evaluation over n minibatch rows into m->grad and the
// device loss sum m->loss
mlbm_status grad_pass(mlbm_mlp* m, const float* X, const float* T, int64_t n, int64_t n_data, uint64_t seed,
                      uint64_t step, cudaStream_t st) {
    const int nb = grad_blocks(n);
    const size_t smem = sizeof(mlp::BwdSmem);
    MLP_CUDA(cudaFuncSetAttribute(mlp::grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    mlp::grad_kernel<<<nb, 128, smem, st>>>(m->p, X, T, m->n_out, n, n_data, seed, step, (float)(2.0 / (double)n),
                                            m->partial, m->loss_partial);
    MLP_CUDA(cudaGetLastError());
    mlp::sum_partials<<<(m->kp + 255) / 256, 256, 0, st>>>(nb, m->kp, m->partial, m->loss_partial, m->grad, m->loss);
    MLP_CUDA(cudaGetLastError());
    return MLBM_OK;
}

mlbm_status read_loss(mlbm_mlp* m, int64_t n, double* loss, cudaStream_t st) {
    double h = 0;
    MLP_CUDA(cudaMemcpyAsync(&h, m->loss, 8, cudaMemcpyDeviceToHost, st));
    MLP_CUDA(cudaStreamSynchronize(st));
    *loss = h / (double)n;
    return MLBM_OK;
}
}  // namespace

extern "C" {

mlbm_status mlbm_mlp_gradients_device(mlbm_mlp* m, const float* X, const float* T, int64_t n, float* grads,
                                      double* loss, void* stream) {
    if (!m || !X || !T || n <= 0) return set_error(MLBM_E_INVALID, "mlp_gradients: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mlbm_status s = grad_pass(m, X, T, n, n, 0, 0, st);
    if (s != MLBM_OK) return s;
    if (grads) MLP_CUDA(cudaMemcpyAsync(grads, m->grad, m->kp * 4, cudaMemcpyDeviceToDevice, st));
    if (loss) return read_loss(m, n, loss, st);
    return MLBM_OK;
}

mlbm_status mlbm_mlp_train_device(mlbm_mlp* m, const float* X, const float* T, int64_t n, int64_t batch,
                                  int64_t steps, float lr, uint64_t seed, double* loss, void* stream) {
    if (!m || !X || !T || n <= 0 || batch <= 0 || steps < 0 || !(lr > 0) || (seed == 0 && batch != n))
        return set_error(MLBM_E_INVALID, "mlp_train: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int64_t k = 0; k < steps; ++k) {
        mlbm_status s = grad_pass(m, X, T, batch, n, seed, (uint64_t)m->t, st);
        if (s != MLBM_OK) return s;
        m->t += 1;
        const double c1 = 1.0 - std::pow(0.9, (double)m->t), c2 = 1.0 - std::pow(0.999, (double)m->t);
        mlp::adam_kernel<<<(m->kp + 255) / 256, 256, 0, st>>>(m->kp, m->p, m->m, m->v, m->grad, lr, 0.9f, 0.999f, 1e-8f,
                                                                (float)c1, (float)c2);
        MLP_CUDA(cudaGetLastError());
    }
    if (loss) {
        if (steps == 0) return set_error(MLBM_E_INVALID, "mlp_train: no step taken, no loss to report");
        return read_loss(m, batch, loss, st);
    }
    return MLBM_OK;
}

}  // extern "C"
