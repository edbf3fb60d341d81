// Geometry features of the learned warm start (one thread per node; FP64
// positions and displacements, FP32 geometry)
// and the kernels that turn a network prediction into an initial state.
//
// Features (16 per node, L = length scale, ell = min(8 L, min(Lx, Ly) / 2)):
//   0      clamp(d1 / L, 0, 4), d1 = distance to the nearest solid surface
//   1, 2   unit vector from that surface point to the node
//   3      clamp(d2 / L, 0, 4), d2 = distance to the second nearest solid object
//   4..7   free paths along +x, -x, +y, -y: distance to the first solid along
//          the ray, at most ell, over L
//   8      clamp(f(+y) f(-y) / L^2, 0, 16)  (the cross-stream Poiseuille
//          profile y (w - y) of a channel along x)
//   9      clamp((f(+y) + f(-y)) / L, 0, 8) (cross-stream gap width)
//   10..13 local porosity within radius rho_j = min(c_j L, min(Lx, Ly) / 2),
//          c_j = 1, 2, 4, 8: 1 - (solid area in the circle) / (pi rho_j^2),
//          disks and their periodic images as circle-circle lenses, solid
//          sides as circular segments
//   14     porosity of the box
//   15     4 (y - y0) (y1 - y) / Ly^2 (position across the box)
// Objects are visited in a fixed order (disks in input order, periodic
// images ix = -1, 0, 1 outer and iy inner around the minimum image, then the
// solid sides left, right, bottom, top); the first strictly nearer object
// sets the direction.  A ray meets a disk when its entry point lies at
// t >= -1e-4 r (a node on the surface looking into the disk sees it at 0,
// looking outward it sees no hit).
#include <cmath>
#include <string>
#include <vector>

#include "kernels.h"
#include "mlbm_internal.h"

namespace mlbm {
namespace dev {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr float kPif = 3.14159265358979f;

// area of the intersection of two circles of radii a and b, centres d apart:
// two circular segments cut by the common chord.  The chord's half-length
// comes from the product form of Heron's formula and the segment angles from
// atan2 of (half-chord, signed centre-to-chord distance), which stays well
// conditioned in FP32 near tangency and near containment (acos of a cosine
// near +-1 does not).
__device__ float lens_area(float d, float a, float b) {
    if (d >= a + b) return 0.f;
    if (d <= fabsf(a - b)) {
        const float m = fminf(a, b);
        return kPif * m * m;
    }
    const float k = fmaxf(0.f, (-d + a + b) * (d + a - b) * (d - a + b) * (d + a + b));
    const float hc = sqrtf(k) / (2.f * d);
    const float xa = (d * d + a * a - b * b) / (2.f * d);  // signed distance from centre A to the chord
    const float xb = d - xa;
    return a * a * atan2f(hc, xa) - xa * hc + b * b * atan2f(hc, xb) - xb * hc;
}

// area of the part of a circle of radius a beyond a line at signed distance h
// from its centre (half-angle from atan2 for the same reason)
__device__ float segment_area(float h, float a) {
    if (h >= a) return 0.f;
    if (h <= -a) return kPif * a * a;
    const float hc = sqrtf((a - h) * (a + h));
    return a * a * atan2f(hc, h) - h * hc;
}

constexpr int kRadii = 4;

struct FeatGeo {
    double x0, y0, lx, ly;
    int perx, pery;
    int solid[4];
    int n_disks;
    float L, ell;
    float rho[kRadii];
    float porosity;
};

// entry distance of a ray along +a (sign = +1) or -a (sign = -1) into a disk,
// da = node - centre along the ray axis, db across it (|db| <= r); the
// half-chord is formed as a product of sums, which keeps its accuracy at
// grazing incidence; INFINITY when the entry lies behind the start (by more
// than 1e-4 r, which absorbs the rounding of a start on the surface)
__device__ __forceinline__ float ray_entry(float da, float db, float r, float sign) {
    const float adb = fabsf(db);
    const float t = -sign * da - sqrtf((r - adb) * (r + adb));
    return t >= -1e-4f * r ? fmaxf(t, 0.f) : INFINITY;
}

// Displacements come from the FP64 positions (minimum image in FP64), the
// rest is FP32: the features feed a BF16 network.
__global__ void features_kernel(int64_t n, const double* __restrict__ xy, const double* __restrict__ disks,
                                FeatGeo G, float* __restrict__ X) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = xy[2 * i], y = xy[2 * i + 1];
    float d1 = INFINITY, d2 = INFINITY, nx = 0.f, ny = 0.f;
    float fp[4] = {G.ell, G.ell, G.ell, G.ell};  // +x, -x, +y, -y
    float S[kRadii] = {0.f, 0.f, 0.f, 0.f};
    auto take = [&](float d, float ux, float uy) {
        if (d < d1) {
            d2 = d1;
            d1 = d;
            nx = ux;
            ny = uy;
        } else if (d < d2) {
            d2 = d;
        }
    };
    const float reach = fmaxf(G.rho[kRadii - 1], G.ell);  // beyond it a disk cuts no circle and no ray
    const float lxf = (float)G.lx, lyf = (float)G.ly;
    for (int k = 0; k < G.n_disks; ++k) {
        const double cx = disks[3 * k], cy = disks[3 * k + 1];
        const float r = (float)disks[3 * k + 2];
        double dx0 = x - cx, dy0 = y - cy;
        if (G.perx) dx0 -= G.lx * rint(dx0 / G.lx);
        if (G.pery) dy0 -= G.ly * rint(dy0 / G.ly);
        for (int ix = -G.perx; ix <= G.perx; ++ix)
            for (int iy = -G.pery; iy <= G.pery; ++iy) {
                const float dx = (float)dx0 + ix * lxf, dy = (float)dy0 + iy * lyf;
                const float dist = sqrtf(dx * dx + dy * dy);
                const float d = dist - r;
                if (d < d2) {
                    if (d < d1) take(d, dist > 0.f ? dx / dist : 0.f, dist > 0.f ? dy / dist : 0.f);
                    else d2 = d;
                }
                if (d >= reach) continue;
                if (fabsf(dy) <= r) {
                    fp[0] = fminf(fp[0], ray_entry(dx, dy, r, 1.f));
                    fp[1] = fminf(fp[1], ray_entry(dx, dy, r, -1.f));
                }
                if (fabsf(dx) <= r) {
                    fp[2] = fminf(fp[2], ray_entry(dy, dx, r, 1.f));
                    fp[3] = fminf(fp[3], ray_entry(dy, dx, r, -1.f));
                }
#pragma unroll
                for (int j = 0; j < kRadii; ++j) S[j] += lens_area(dist, G.rho[j], r);
            }
    }
    const float h[4] = {(float)(x - G.x0), (float)(G.x0 + G.lx - x), (float)(y - G.y0), (float)(G.y0 + G.ly - y)};
    const float wn[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    const int ray_of_side[4] = {1, 0, 3, 2};  // the -x ray meets the left side, ...
    for (int sd = 0; sd < 4; ++sd) {
        if (!G.solid[sd]) continue;
        take(h[sd], wn[sd][0], wn[sd][1]);
        fp[ray_of_side[sd]] = fminf(fp[ray_of_side[sd]], fmaxf(h[sd], 0.f));
#pragma unroll
        for (int j = 0; j < kRadii; ++j) S[j] += segment_area(h[sd], G.rho[j]);
    }
    if (!(d1 < INFINITY)) d1 = 4.f * G.L;
    if (!(d2 < INFINITY)) d2 = 4.f * G.L;
    const float a = d1 / G.L, b = d2 / G.L;
    float* o = X + 16 * i;
    o[0] = fminf(fmaxf(a, 0.f), 4.f);
    o[1] = nx;
    o[2] = ny;
    o[3] = fminf(fmaxf(b, 0.f), 4.f);
#pragma unroll
    for (int j = 0; j < 4; ++j) o[4 + j] = fp[j] / G.L;
    o[8] = fminf(fp[2] * fp[3] / (G.L * G.L), 16.f);
    o[9] = fminf((fp[2] + fp[3]) / G.L, 8.f);
#pragma unroll
    for (int j = 0; j < kRadii; ++j) o[10 + j] = 1.f - S[j] / (kPif * G.rho[j] * G.rho[j]);
    o[14] = G.porosity;
    const double yy = y - G.y0;
    o[15] = (float)(4.0 * yy * (G.ly - yy) / (G.ly * G.ly));
}

// ---------------------------------------------------------------- warm start
// Y[n][no] (caller order): scaled velocity in columns 0, 1 and, when no = 3,
// scaled density deviation in column 2.
// flag[sample] |= 1 when a prediction of the sample is unusable: a
// non-finite value, a speed above umax or a density deviation above drho_max
__global__ void warm_check(int n, const int* __restrict__ perm, const uint16_t* __restrict__ node_sample,
                           const uint8_t* __restrict__ meta, const float* __restrict__ Y, int no,
                           const double* __restrict__ scale_u, const double* __restrict__ scale_rho, float umax,
                           float drho_max, int* __restrict__ flag) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    if ((meta[p] & 3) == 2) return;  // equilibrium-overwrite node
    const int smp = node_sample ? node_sample[p] : 0;
    const int64_t id = perm[p];
    const double ux = scale_u[smp] * (double)Y[no * id], uy = scale_u[smp] * (double)Y[no * id + 1];
    const double sp = sqrt(ux * ux + uy * uy);
    bool bad = !(sp <= (double)umax);
    if (no == 3) bad |= !(fabs(scale_rho[smp] * (double)Y[no * id + 2]) <= (double)drho_max);
    if (bad) atomicOr(&flag[smp], 1);
}

// scaled density deviation of every node in position order (0 on
// equilibrium-overwrite nodes), for the per-sample mean
__global__ void warm_drho(int n, const int* __restrict__ perm, const uint16_t* __restrict__ node_sample,
                          const uint8_t* __restrict__ meta, const float* __restrict__ Y, int no,
                          const double* __restrict__ scale_rho, float* __restrict__ drho) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int smp = node_sample ? node_sample[p] : 0;
    drho[p] = (meta[p] & 3) == 2 ? 0.f : (float)(scale_rho[smp] * (double)Y[no * (int64_t)perm[p] + 2]);
}

// rho_u[n][3] (caller order, FP64) of the warm start: rho = 1 + (predicted
// deviation - its area-weighted sample mean, so the sample's mass stays that
// of the rest state) and u = predicted velocity; samples flagged cold start
// from rest; equilibrium-overwrite nodes take their boundary values
__global__ void warm_fill(int n, const int* __restrict__ perm, const uint16_t* __restrict__ node_sample,
                          const uint8_t* __restrict__ meta, const float4* __restrict__ eqv,
                          const float* __restrict__ Y, int no, const double* __restrict__ scale_u,
                          const float* __restrict__ drho, const double* __restrict__ drho_mean,
                          const int* __restrict__ flag, double* __restrict__ ru) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int smp = node_sample ? node_sample[p] : 0;
    const int64_t id = perm[p];
    double* v = ru + 3 * id;
    if ((meta[p] & 3) == 2) {
        const float4 e = eqv[p];
        v[0] = 1.0 + (double)e.x;
        v[1] = e.y;
        v[2] = e.z;
        return;
    }
    const bool cold = flag[smp] != 0;
    const double sc = cold ? 0.0 : scale_u[smp];
    v[0] = (no == 3 && !cold) ? 1.0 + ((double)drho[p] - drho_mean[smp]) : 1.0;
    v[1] = sc * (double)Y[no * id];
    v[2] = sc * (double)Y[no * id + 1];
}

}  // namespace dev

cudaError_t launch_warm_check(int n, const int* perm, const uint16_t* node_sample, const uint8_t* meta,
                              const float* Y, int no, const double* scale_u, const double* scale_rho, float umax,
                              float drho_max, int* flag, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    dev::warm_check<<<(n + 255) / 256, 256, 0, st>>>(n, perm, node_sample, meta, Y, no, scale_u, scale_rho, umax,
                                                     drho_max, flag);
    return cudaGetLastError();
}

cudaError_t launch_warm_drho(int n, const int* perm, const uint16_t* node_sample, const uint8_t* meta,
                             const float* Y, int no, const double* scale_rho, float* drho, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    dev::warm_drho<<<(n + 255) / 256, 256, 0, st>>>(n, perm, node_sample, meta, Y, no, scale_rho, drho);
    return cudaGetLastError();
}

cudaError_t launch_warm_fill(int n, const int* perm, const uint16_t* node_sample, const uint8_t* meta,
                             const float4* eqv, const float* Y, int no, const double* scale_u, const float* drho,
                             const double* drho_mean, const int* flag, double* ru, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    dev::warm_fill<<<(n + 255) / 256, 256, 0, st>>>(n, perm, node_sample, meta, eqv, Y, no, scale_u, drho, drho_mean,
                                                    flag, ru);
    return cudaGetLastError();
}

}  // namespace mlbm

using namespace mlbm;

extern "C" mlbm_status mlbm_features_device(const mlbm_nodes* nodes, const mlbm_geometry* geo, double L, float* X) {
    clear_error();
    if (!nodes || !geo || !X || nodes->n < 0 || (nodes->n > 0 && !nodes->xy) || !(L > 0) ||
        (geo->n_disks > 0 && !geo->disks) || geo->n_disks < 0)
        return set_error(MLBM_E_INVALID, "features: bad arguments");
    const double lx = geo->x1 - geo->x0, ly = geo->y1 - geo->y0;
    if (!(lx > 0) || !(ly > 0)) return set_error(MLBM_E_INVALID, "features: empty box");
    const int64_t n = nodes->n;
    if (n == 0) return MLBM_OK;
    dev::FeatGeo G{};
    G.x0 = geo->x0;
    G.y0 = geo->y0;
    G.lx = lx;
    G.ly = ly;
    G.perx = geo->side[0] == MLBM_SIDE_PERIODIC && geo->side[1] == MLBM_SIDE_PERIODIC;
    G.pery = geo->side[2] == MLBM_SIDE_PERIODIC && geo->side[3] == MLBM_SIDE_PERIODIC;
    for (int k = 0; k < 4; ++k) G.solid[k] = geo->side[k] == MLBM_SIDE_SOLID;
    G.n_disks = geo->n_disks;
    G.L = (float)L;
    G.ell = (float)std::fmin(8.0 * L, 0.5 * std::fmin(lx, ly));
    const double cj[dev::kRadii] = {1.0, 2.0, 4.0, 8.0};
    for (int j = 0; j < dev::kRadii; ++j) G.rho[j] = (float)std::fmin(cj[j] * L, 0.5 * std::fmin(lx, ly));
    double solid = 0.0;
    for (int k = 0; k < geo->n_disks; ++k) solid += dev::kPi * geo->disks[3 * k + 2] * geo->disks[3 * k + 2];
    G.porosity = (float)(1.0 - solid / (lx * ly));
    double* dxy = nullptr;
    double* ddisks = nullptr;
    cudaError_t e = cudaMalloc(&dxy, (size_t)n * 2 * sizeof(double));
    if (e == cudaSuccess && geo->n_disks > 0) e = cudaMalloc(&ddisks, (size_t)geo->n_disks * 3 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(dxy, nodes->xy, (size_t)n * 2 * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && geo->n_disks > 0)
        e = cudaMemcpy(ddisks, geo->disks, (size_t)geo->n_disks * 3 * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const int64_t blocks = (n + 127) / 128;
        dev::features_kernel<<<(unsigned)blocks, 128>>>(n, dxy, ddisks, G, X);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(dxy);
    cudaFree(ddisks);
    if (e != cudaSuccess) return set_error(MLBM_E_CUDA, std::string("features: ") + cudaGetErrorString(e));
    return MLBM_OK;
}
