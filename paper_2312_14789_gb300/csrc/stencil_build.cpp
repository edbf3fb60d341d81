// Host (FP64) stencil builder behind mlbm_build_stencils.
//
// Per node, once per node set and streaming distance s (the paper's weight
// precomputation, Sec. 2.2):
//   1. K nearest nodes by a ring search over a uniform cell grid (periodic
//      sides wrap; the minimum image of every offset is used, Sec. 3.2);
//   2. the quadratic weighted least-squares matrix by Householder QR of
//      sqrt(W) P (FP64), stored in units of s;
//   3. the regular 3x3 block test for biquadratic Lagrange (Sec. 2.2);
//   4. bounce-back links by intersecting the departure segment with the
//      solids (Sec. 3.1, 3.2);
//   5. a Hilbert-curve order of the nodes so that neighbour gathers on the
//      GPU stay within a small window of memory.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>

#include "mlbm_internal.h"

namespace mlbm {
namespace {

struct Box {
    double x0, y0, x1, y1, lx, ly;
    int side[4];
    bool px, py;
};

inline double min_image(double d, double L, bool periodic) {
    if (!periodic) return d;
    if (d >= 0.5 * L) d -= L;
    if (d < -0.5 * L) d += L;
    return d;
}

// Uniform grid whose cells tile periodic extents exactly.
struct CellGrid {
    double x0 = 0, y0 = 0, cx = 1, cy = 1;
    int ncx = 1, ncy = 1;
    std::vector<int64_t> start, items;

    int cell_x(double x) const {
        int c = (int)std::floor((x - x0) / cx);
        return c < 0 ? 0 : (c >= ncx ? ncx - 1 : c);
    }
    int cell_y(double y) const {
        int c = (int)std::floor((y - y0) / cy);
        return c < 0 ? 0 : (c >= ncy ? ncy - 1 : c);
    }
};

CellGrid make_grid(const double* xy, int64_t n, const Box& b, int K) {
    CellGrid g;
    g.x0 = b.x0;
    g.y0 = b.y0;
    // about K/4 nodes per cell
    double target = std::sqrt(b.lx * b.ly / (double)n * std::max(1, K / 4));
    g.ncx = std::max(1, (int)std::floor(b.lx / target));
    g.ncy = std::max(1, (int)std::floor(b.ly / target));
    g.ncx = std::min(g.ncx, 1 << 15);
    g.ncy = std::min(g.ncy, 1 << 15);
    g.cx = b.lx / g.ncx;
    g.cy = b.ly / g.ncy;
    int64_t nc = (int64_t)g.ncx * g.ncy;
    g.start.assign(nc + 1, 0);
    std::vector<int64_t> cell(n);
    for (int64_t i = 0; i < n; ++i) {
        cell[i] = (int64_t)g.cell_y(xy[2 * i + 1]) * g.ncx + g.cell_x(xy[2 * i]);
        g.start[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < nc; ++c) g.start[c + 1] += g.start[c];
    g.items.resize(n);
    std::vector<int64_t> fill(g.start.begin(), g.start.end() - 1);
    for (int64_t i = 0; i < n; ++i) g.items[fill[cell[i]]++] = i;  // ids ascending per cell
    return g;
}

// K nearest of node i ordered by (d2, id), self included.
void knn_one(const CellGrid& g, const double* xy, const Box& b, int64_t i, int K, int64_t* id, double* d2,
             double* off) {
    const double xi = xy[2 * i], yi = xy[2 * i + 1];
    const int ci = g.cell_x(xi), cj = g.cell_y(yi);
    int cnt = 0;
    const int rmax = std::max(g.ncx, g.ncy) + 1;
    const double cmin = std::min(g.cx, g.cy);
    for (int r = 0; r <= rmax; ++r) {
        for (int dy = -r; dy <= r; ++dy) {
            int yy = cj + dy;
            if (b.py) {
                yy %= g.ncy;
                if (yy < 0) yy += g.ncy;
            } else if (yy < 0 || yy >= g.ncy) {
                continue;
            }
            const bool edge_row = (dy == -r || dy == r);
            for (int dx = -r; dx <= r; dx += (edge_row ? 1 : 2 * r)) {
                int xx = ci + dx;
                if (b.px) {
                    xx %= g.ncx;
                    if (xx < 0) xx += g.ncx;
                } else if (xx < 0 || xx >= g.ncx) {
                    if (r == 0) break;
                    continue;
                }
                const int64_t c = (int64_t)yy * g.ncx + xx;
                for (int64_t e = g.start[c]; e < g.start[c + 1]; ++e) {
                    const int64_t j = g.items[e];
                    const double ox = min_image(xy[2 * j] - xi, b.lx, b.px);
                    const double oy = min_image(xy[2 * j + 1] - yi, b.ly, b.py);
                    const double dd = ox * ox + oy * oy;
                    if (cnt == K && (dd > d2[K - 1] || (dd == d2[K - 1] && j > id[K - 1]))) continue;
                    bool dup = false;
                    for (int m = 0; m < cnt; ++m)
                        if (id[m] == j) { dup = true; break; }
                    if (dup) continue;
                    int pos = (cnt == K) ? K - 1 : cnt;
                    while (pos > 0 && (d2[pos - 1] > dd || (d2[pos - 1] == dd && id[pos - 1] > j))) {
                        d2[pos] = d2[pos - 1];
                        id[pos] = id[pos - 1];
                        off[2 * pos] = off[2 * pos - 2];
                        off[2 * pos + 1] = off[2 * pos - 1];
                        --pos;
                    }
                    d2[pos] = dd;
                    id[pos] = j;
                    off[2 * pos] = ox;
                    off[2 * pos + 1] = oy;
                    if (cnt < K) ++cnt;
                }
                if (r == 0) break;
            }
        }
        // every unvisited node sits at least r cells away
        if (cnt == K) {
            const double reach = r * cmin;
            if (d2[K - 1] < reach * reach) break;
        }
    }
}

// The n_l nearest nodes of the point x_i + (dx, dy), ordered by (d2, id):
// offsets by the periodic minimum image from node i, the squared distance
// measured from the point (RBF-FD stencils per Lagrangian point).
void knn_point(const CellGrid& g, const double* xy, const Box& b, int64_t i, double dx, double dy, int n_l,
               int64_t* id, double* d2, double* off) {
    const double xi = xy[2 * i], yi = xy[2 * i + 1];
    double qx = xi + dx, qy = yi + dy;
    if (b.px) qx = b.x0 + std::fmod(std::fmod(qx - b.x0, b.lx) + b.lx, b.lx);
    if (b.py) qy = b.y0 + std::fmod(std::fmod(qy - b.y0, b.ly) + b.ly, b.ly);
    const int ci = g.cell_x(qx), cj = g.cell_y(qy);
    int cnt = 0;
    const int rmax = std::max(g.ncx, g.ncy) + 1;
    const double cmin = std::min(g.cx, g.cy);
    for (int r = 0; r <= rmax; ++r) {
        for (int ddy = -r; ddy <= r; ++ddy) {
            int yy = cj + ddy;
            if (b.py) {
                yy %= g.ncy;
                if (yy < 0) yy += g.ncy;
            } else if (yy < 0 || yy >= g.ncy) {
                continue;
            }
            const bool edge_row = (ddy == -r || ddy == r);
            for (int ddx = -r; ddx <= r; ddx += (edge_row ? 1 : 2 * r)) {
                int xx = ci + ddx;
                if (b.px) {
                    xx %= g.ncx;
                    if (xx < 0) xx += g.ncx;
                } else if (xx < 0 || xx >= g.ncx) {
                    if (r == 0) break;
                    continue;
                }
                const int64_t c = (int64_t)yy * g.ncx + xx;
                for (int64_t e = g.start[c]; e < g.start[c + 1]; ++e) {
                    const int64_t j = g.items[e];
                    const double ox = min_image(xy[2 * j] - xi, b.lx, b.px);
                    const double oy = min_image(xy[2 * j + 1] - yi, b.ly, b.py);
                    const double ex = ox - dx, ey = oy - dy;
                    const double dd = ex * ex + ey * ey;
                    if (cnt == n_l && (dd > d2[n_l - 1] || (dd == d2[n_l - 1] && j > id[n_l - 1]))) continue;
                    bool dup = false;
                    for (int m = 0; m < cnt; ++m)
                        if (id[m] == j) { dup = true; break; }
                    if (dup) continue;
                    int pos = (cnt == n_l) ? n_l - 1 : cnt;
                    while (pos > 0 && (d2[pos - 1] > dd || (d2[pos - 1] == dd && id[pos - 1] > j))) {
                        d2[pos] = d2[pos - 1];
                        id[pos] = id[pos - 1];
                        off[2 * pos] = off[2 * pos - 2];
                        off[2 * pos + 1] = off[2 * pos - 1];
                        --pos;
                    }
                    d2[pos] = dd;
                    id[pos] = j;
                    off[2 * pos] = ox;
                    off[2 * pos + 1] = oy;
                    if (cnt < n_l) ++cnt;
                }
                if (r == 0) break;
            }
        }
        if (cnt == n_l) {
            const double reach = r * cmin;
            if (d2[n_l - 1] < reach * reach) break;
        }
    }
}

// Quadratic WLS by Householder QR.  Returns 0, or 2 when cond(R)^2 > 1e12.
int wls_qr(const double* off, int K, double s, double sigma_factor, double* M) {
    double rK = 0;
    for (int j = 0; j < K; ++j) rK = std::max(rK, std::sqrt(off[2 * j] * off[2 * j] + off[2 * j + 1] * off[2 * j + 1]));
    if (!(rK > 0)) return 2;
    const double sig2 = (sigma_factor * rK) * (sigma_factor * rK);
    double A[32][6], sw[32];
    for (int j = 0; j < K; ++j) {
        const double x = off[2 * j], y = off[2 * j + 1];
        sw[j] = std::sqrt(std::exp(-(x * x + y * y) / sig2));
        const double u = x / rK, v = y / rK;
        const double p[6] = {1.0, u, v, u * u, u * v, v * v};
        for (int a = 0; a < 6; ++a) A[j][a] = sw[j] * p[a];
    }
    double V[6][32];  // Householder vectors
    for (int c = 0; c < 6; ++c) {
        double nrm = 0;
        for (int j = c; j < K; ++j) nrm += A[j][c] * A[j][c];
        nrm = std::sqrt(nrm);
        if (nrm == 0) return 2;
        const double alpha = A[c][c] > 0 ? -nrm : nrm;
        double vv = 0;
        for (int j = 0; j < K; ++j) V[c][j] = 0;
        for (int j = c; j < K; ++j) V[c][j] = A[j][c];
        V[c][c] -= alpha;
        for (int j = c; j < K; ++j) vv += V[c][j] * V[c][j];
        if (vv == 0) return 2;
        for (int col = c; col < 6; ++col) {
            double dot = 0;
            for (int j = c; j < K; ++j) dot += V[c][j] * A[j][col];
            const double f = 2.0 * dot / vv;
            for (int j = c; j < K; ++j) A[j][col] -= f * V[c][j];
        }
        const double vn = std::sqrt(vv);
        for (int j = c; j < K; ++j) V[c][j] /= vn;  // unit vector: H = I - 2 v v^T
    }
    // R = A[0:6][0:6] (upper), its inverse by back substitution
    double Ri[6][6] = {};
    for (int c = 0; c < 6; ++c) {
        if (A[c][c] == 0) return 2;
        Ri[c][c] = 1.0 / A[c][c];
        for (int r = c - 1; r >= 0; --r) {
            double acc = 0;
            for (int m = r + 1; m <= c; ++m) acc += A[r][m] * Ri[m][c];
            Ri[r][c] = -acc / A[r][r];
        }
    }
    double nR = 0, nRi = 0;
    for (int c = 0; c < 6; ++c) {
        double a = 0, b = 0;
        for (int r = 0; r <= c; ++r) { a += std::fabs(A[r][c]); b += std::fabs(Ri[r][c]); }
        nR = std::max(nR, a);
        nRi = std::max(nRi, b);
    }
    if ((nR * nRi) * (nR * nRi) > 1e12) return 2;
    // Q1 = H_0 ... H_5 [I_6; 0]  (K x 6)
    double Q[32][6];
    for (int j = 0; j < K; ++j)
        for (int a = 0; a < 6; ++a) Q[j][a] = (j == a) ? 1.0 : 0.0;
    for (int c = 5; c >= 0; --c)
        for (int col = 0; col < 6; ++col) {
            double dot = 0;
            for (int j = c; j < K; ++j) dot += V[c][j] * Q[j][col];
            for (int j = c; j < K; ++j) Q[j][col] -= 2.0 * dot * V[c][j];
        }
    // M~ = R^-1 Q1^T diag(sqrt w), rows scaled by (s / rK)^deg
    static const int deg[6] = {0, 1, 1, 2, 2, 2};
    for (int a = 0; a < 6; ++a) {
        const double sc = std::pow(s / rK, deg[a]);
        for (int j = 0; j < K; ++j) {
            double acc = 0;
            for (int m = a; m < 6; ++m) acc += Ri[a][m] * Q[j][m];
            M[a * K + j] = acc * sw[j] * sc;
        }
    }
    return 0;
}

// RBF-FD weights of the stencil for the value at (dx, dy) (Sec. 2.2): the
// cubic polyharmonic spline with quadratic augmentation.  The saddle-point
// system [Phi P; P^T 0] [w; l] = [phi(|o_i - d|); p(d)] is solved by LU with
// partial pivoting in FP64, coordinates scaled by the largest offset (the
// weights are scale-free).  Returns 0, or 2 for a numerically singular
// system (smallest pivot below 1e-13 of the largest).
int rbf_weights(const double* off, int K, double dx, double dy, double* w) {
    const int N = K + 6;
    double rK = 0;
    for (int j = 0; j < K; ++j) rK = std::max(rK, std::hypot(off[2 * j], off[2 * j + 1]));
    if (!(rK > 0)) return 2;
    double A[38][38], b[38], u[32], v[32];
    for (int j = 0; j < K; ++j) {
        u[j] = off[2 * j] / rK;
        v[j] = off[2 * j + 1] / rK;
    }
    const double du = dx / rK, dv = dy / rK;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) A[i][j] = 0.0;
    for (int i = 0; i < K; ++i) {
        for (int j = 0; j < K; ++j) {
            const double r = std::hypot(u[i] - u[j], v[i] - v[j]);
            A[i][j] = r * r * r;
        }
        const double p[6] = {1.0, u[i], v[i], u[i] * u[i], u[i] * v[i], v[i] * v[i]};
        for (int a = 0; a < 6; ++a) A[i][K + a] = A[K + a][i] = p[a];
        const double r = std::hypot(u[i] - du, v[i] - dv);
        b[i] = r * r * r;
    }
    const double pd[6] = {1.0, du, dv, du * du, du * dv, dv * dv};
    for (int a = 0; a < 6; ++a) b[K + a] = pd[a];
    double pmax = 0, pmin = 1e300;
    for (int c = 0; c < N; ++c) {
        int piv = c;
        for (int r = c + 1; r < N; ++r)
            if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
        if (piv != c) {
            for (int j = 0; j < N; ++j) std::swap(A[c][j], A[piv][j]);
            std::swap(b[c], b[piv]);
        }
        const double d = A[c][c];
        pmax = std::max(pmax, std::fabs(d));
        pmin = std::min(pmin, std::fabs(d));
        if (d == 0.0) return 2;
        for (int r = c + 1; r < N; ++r) {
            const double m = A[r][c] / d;
            if (m == 0.0) continue;
            for (int j = c; j < N; ++j) A[r][j] -= m * A[c][j];
            b[r] -= m * b[c];
        }
    }
    if (pmin < 1e-13 * pmax) return 2;
    double x[38];
    for (int r = N - 1; r >= 0; --r) {
        double acc = b[r];
        for (int j = r + 1; j < N; ++j) acc -= A[r][j] * x[j];
        x[r] = acc / A[r][r];
    }
    for (int j = 0; j < K; ++j) w[j] = x[j];
    return 0;
}

// Departure offsets and which directions interpolate (simple bounce-back
// links copy the node's own population instead).
void departures(double s, uint16_t mask, const double* q, int bb_mode, double* dx, double* dy, bool* use) {
    use[0] = false;
    for (int k = 1; k < 9; ++k) {
        if (mask & (1u << k)) {
            if (bb_mode == MLBM_BB_SIMPLE) {
                use[k] = false;
                dx[k] = dy[k] = 0;
                continue;
            }
            const double t = 1.0 - 2.0 * q[k];
            dx[k] = t * s * kEx[k];
            dy[k] = t * s * kEy[k];
        } else {
            dx[k] = -s * kEx[k];
            dy[k] = -s * kEy[k];
        }
        use[k] = true;
    }
}

// Axis-aligned 3x3 block (spacing h = nearest non-zero offset) centred on
// x + h e_m, m tried in D2Q9 order, containing every departure point.
bool find_block(const double* off, int K, const double* dx, const double* dy, const bool* use, double tol,
                int8_t* slot, double* h_out, uint8_t* center) {
    double h = 0;
    for (int j = 0; j < K; ++j) {
        const double r = std::sqrt(off[2 * j] * off[2 * j] + off[2 * j + 1] * off[2 * j + 1]);
        if (r > 0 && (h == 0 || r < h)) h = r;
    }
    if (h == 0) return false;
    for (int m = 0; m < 9; ++m) {
        const double cx = kEx[m] * h, cy = kEy[m] * h;
        bool ok = true;
        for (int k = 1; k < 9 && ok; ++k)
            if (use[k] && (std::fabs(dx[k] - cx) > h * (1.0 + tol) || std::fabs(dy[k] - cy) > h * (1.0 + tol)))
                ok = false;
        int8_t sl[9];
        for (int b = 0; b < 3 && ok; ++b)
            for (int a = 0; a < 3 && ok; ++a) {
                const double px = cx + (a - 1) * h, py = cy + (b - 1) * h;
                int found = -1;
                for (int j = 0; j < K; ++j)
                    if (std::fabs(off[2 * j] - px) <= tol * h && std::fabs(off[2 * j + 1] - py) <= tol * h) {
                        found = j;
                        break;
                    }
                if (found < 0) ok = false;
                else sl[b * 3 + a] = (int8_t)found;
            }
        if (ok) {
            std::memcpy(slot, sl, 9);
            *h_out = h;
            *center = (uint8_t)m;
            return true;
        }
    }
    return false;
}

// Bounce-back links of node (x, y).  Returns 0, or 8 when the node is inside
// a solid.
// Disks binned by the cells of a uniform grid over the box that their circle
// (and each periodic image's), grown by `reach`, overlaps.  A departure
// segment from a node is at most sqrt(2) s long, so with reach > sqrt(2) s a
// disk that can meet it, or contains or touches the node, is listed in the
// node's cell: testing those disks gives the result of testing all of them.
struct DiskGrid {
    double x0 = 0, y0 = 0, x1 = 0, y1 = 0, c = 1;
    int ncx = 0, ncy = 0;
    std::vector<int> start, items;
    // the disks to test for a node at (x, y): ids[0..*n), or all disks when
    // the node lies outside the grid (ids = nullptr)
    const int* at(double x, double y, int* n) const {
        if (ncx == 0 || !(x >= x0 && x <= x1 && y >= y0 && y <= y1)) return nullptr;
        const int i = std::min(ncx - 1, (int)std::floor((x - x0) / c));
        const int j = std::min(ncy - 1, (int)std::floor((y - y0) / c));
        const int k = j * ncx + i;
        *n = start[k + 1] - start[k];
        return items.data() + start[k];
    }
};

DiskGrid make_disk_grid(const Box& b, const double* disks, int nd, double reach) {
    DiskGrid g;
    if (nd == 0) return g;
    double rmax = 0;
    for (int d = 0; d < nd; ++d) rmax = std::max(rmax, disks[3 * d + 2]);
    g.x0 = b.x0;
    g.y0 = b.y0;
    g.x1 = b.x1;
    g.y1 = b.y1;
    g.c = std::max({2.0 * reach, 0.5 * rmax, std::max(b.lx, b.ly) / 2048.0});
    g.ncx = std::max(1, (int)std::ceil(b.lx / g.c));
    g.ncy = std::max(1, (int)std::ceil(b.ly / g.c));
    std::vector<std::vector<int>> cells((size_t)g.ncx * g.ncy);
    for (int d = 0; d < nd; ++d)
        for (int ix = -1; ix <= 1; ++ix) {
            if (ix != 0 && !b.px) continue;
            for (int iy = -1; iy <= 1; ++iy) {
                if (iy != 0 && !b.py) continue;
                const double cx = disks[3 * d] + ix * b.lx, cy = disks[3 * d + 1] + iy * b.ly;
                const double r = disks[3 * d + 2] + reach;
                const double lo_x = cx - r, hi_x = cx + r, lo_y = cy - r, hi_y = cy + r;
                if (hi_x < g.x0 || lo_x > g.x1 || hi_y < g.y0 || lo_y > g.y1) continue;
                const int i0 = std::max(0, (int)std::floor((lo_x - g.x0) / g.c));
                const int i1 = std::min(g.ncx - 1, (int)std::floor((hi_x - g.x0) / g.c));
                const int j0 = std::max(0, (int)std::floor((lo_y - g.y0) / g.c));
                const int j1 = std::min(g.ncy - 1, (int)std::floor((hi_y - g.y0) / g.c));
                for (int j = j0; j <= j1; ++j)
                    for (int i = i0; i <= i1; ++i) cells[(size_t)j * g.ncx + i].push_back(d);
            }
        }
    g.start.assign(cells.size() + 1, 0);
    for (size_t k = 0; k < cells.size(); ++k) {
        std::sort(cells[k].begin(), cells[k].end());
        cells[k].erase(std::unique(cells[k].begin(), cells[k].end()), cells[k].end());
        g.start[k + 1] = g.start[k] + (int)cells[k].size();
    }
    g.items.reserve((size_t)g.start.back());
    for (const auto& v : cells) g.items.insert(g.items.end(), v.begin(), v.end());
    return g;
}

// Bounce-back links of a node: for each direction, the fraction q of the
// departure segment at which it first meets a solid side or disk (every
// periodic image of the disks `ids` lists; all nd disks when ids is NULL).
int links_of(double x, double y, double s, const Box& b, const double* disks, const int* ids, int nd,
             uint16_t* mask, double* q) {
    const double tol = 1e-9 * s;
    *mask = 0;
    for (int k = 0; k < 9; ++k) q[k] = 0;
    for (int k = 1; k < 9; ++k) {
        const double vx = -s * kEx[k], vy = -s * kEy[k];
        double best = 2.0;
        auto side_hit = [&](double dist, double speed) -> int {
            // dist: distance from the node to the wall along the inward normal,
            // speed > 0: approach rate per unit t
            if (dist < -tol) return 8;
            const double t = dist <= tol ? 0.0 : dist / speed;
            if (t < 1.0 && t < best) best = t;
            return 0;
        };
        if (b.side[2] == MLBM_SIDE_SOLID && vy < 0 && side_hit(y - b.y0, -vy)) return 8;
        if (b.side[3] == MLBM_SIDE_SOLID && vy > 0 && side_hit(b.y1 - y, vy)) return 8;
        if (b.side[0] == MLBM_SIDE_SOLID && vx < 0 && side_hit(x - b.x0, -vx)) return 8;
        if (b.side[1] == MLBM_SIDE_SOLID && vx > 0 && side_hit(b.x1 - x, vx)) return 8;
        for (int m = 0; m < nd; ++m) {
            const int d = ids ? ids[m] : m;
            for (int ix = -1; ix <= 1; ++ix) {
                if (ix != 0 && !b.px) continue;
                for (int iy = -1; iy <= 1; ++iy) {
                    if (iy != 0 && !b.py) continue;
                    const double cxd = disks[3 * d] + ix * b.lx, cyd = disks[3 * d + 1] + iy * b.ly;
                    const double R = disks[3 * d + 2];
                    const double rx = x - cxd, ry = y - cyd;
                    const double dist = std::sqrt(rx * rx + ry * ry);
                    if (dist < R * (1.0 - 1e-9)) return 8;
                    const double bb = rx * vx + ry * vy;
                    if (dist <= R * (1.0 + 1e-9)) {
                        if (bb < 0) best = 0.0;
                        continue;
                    }
                    const double aa = vx * vx + vy * vy;
                    const double cc = rx * rx + ry * ry - R * R;
                    const double disc = bb * bb - aa * cc;
                    if (disc <= 0) continue;
                    const double t = (-bb - std::sqrt(disc)) / aa;
                    if (t >= 0 && t < 1.0 && t < best) best = t;
                }
            }
        }
        if (best < 1.0) {
            *mask |= (uint16_t)(1u << k);
            q[k] = best;
        }
    }
    return 0;
}

// Morton (Z-order) index: the bits of x and y interleaved.
uint64_t morton_index(uint32_t x, uint32_t y) {
    uint64_t d = 0;
    for (int b = 0; b < 32; ++b) d |= ((uint64_t)((x >> b) & 1u) << (2 * b)) | ((uint64_t)((y >> b) & 1u) << (2 * b + 1));
    return d;
}

uint64_t hilbert_index(uint32_t x, uint32_t y, int order);

// Position -> caller id for a node order (MLBM_ORDER_*).  Keys come from the
// positions scaled to [0, 2^16) over the box; ties keep the caller's order.
// Rows: strips of height ~ the mean node spacing times 8, left to right in
// each strip.
std::vector<int64_t> order_nodes(const std::vector<double>& xy, double x0, double y0, double lx, double ly,
                                 int order) {
    const int64_t n = (int64_t)(xy.size() / 2);
    std::vector<int64_t> perm(n);
    std::iota(perm.begin(), perm.end(), 0);
    if (order == MLBM_ORDER_INPUT) return perm;
    std::vector<uint64_t> key(n);
    const int bits = 16;
    const double scale = (double)((1u << bits) - 1);
    const double strip = 8.0 * std::sqrt(lx * ly / std::max<int64_t>(n, 1));
    const int64_t n_strips = std::max<int64_t>(1, (int64_t)std::ceil(ly / strip));
    for (int64_t i = 0; i < n; ++i) {
        double u = (xy[2 * i] - x0) / lx, v = (xy[2 * i + 1] - y0) / ly;
        u = std::min(1.0, std::max(0.0, u));
        v = std::min(1.0, std::max(0.0, v));
        const uint32_t ux = (uint32_t)(u * scale), vy = (uint32_t)(v * scale);
        if (order == MLBM_ORDER_MORTON) {
            key[i] = morton_index(ux, vy);
        } else if (order == MLBM_ORDER_ROWS) {
            const int64_t row = std::min<int64_t>(n_strips - 1, (int64_t)(v * n_strips));
            key[i] = ((uint64_t)row << 32) | ux;
        } else {
            key[i] = hilbert_index(ux, vy, bits);
        }
    }
    std::stable_sort(perm.begin(), perm.end(), [&](int64_t a, int64_t c) { return key[a] < key[c]; });
    return perm;
}

// Hilbert index of (x, y) in [0, 2^order)^2.
uint64_t hilbert_index(uint32_t x, uint32_t y, int order) {
    uint64_t d = 0;
    for (uint32_t sq = 1u << (order - 1); sq > 0; sq >>= 1) {
        const uint32_t rx = (x & sq) ? 1 : 0;
        const uint32_t ry = (y & sq) ? 1 : 0;
        d += (uint64_t)sq * sq * ((3 * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = sq - 1 - x;
                y = sq - 1 - y;
            }
            std::swap(x, y);
        }
    }
    return d;
}

}  // namespace
}  // namespace mlbm

using namespace mlbm;

extern "C" mlbm_status mlbm_build_stencils(const mlbm_nodes* nodes, const mlbm_geometry* geo, int K, double s,
                                           double sigma_factor, int bb_mode, int use_lagrange,
                                           mlbm_stencils** out) {
    return mlbm_build_stencils_ex(nodes, geo, K, s, sigma_factor, bb_mode, use_lagrange, MLBM_INTERP_WLS, out);
}

namespace {

// The builder.  K is the node's own stencil (least-squares fit, Lagrange
// detection); for MLBM_INTERP_RBF_POINTS every interpolating direction gets
// the n_l nearest nodes of its departure point and the node's device stencil
// is their union, k_max slots wide.
mlbm_status build_impl(const mlbm_nodes* nodes, const mlbm_geometry* geo, int K, double s, double sigma_factor,
                       int bb_mode, int use_lagrange, int interp, int n_l, int k_max, mlbm_stencils** out) {
    clear_error();
    if (interp != MLBM_INTERP_WLS && interp != MLBM_INTERP_RBF && interp != MLBM_INTERP_RBF_POINTS)
        return set_error(MLBM_E_INVALID, "build_stencils: bad interpolant");
    if (!out) return set_error(MLBM_E_INVALID, "build_stencils: out is NULL");
    *out = nullptr;
    if (!nodes || !geo || !nodes->xy || !nodes->node_class)
        return set_error(MLBM_E_INVALID, "build_stencils: nodes, geometry, xy and node_class are required");
    const int64_t n = nodes->n;
    if (n < 1 || n > (int64_t(1) << 31) - 1) return set_error(MLBM_E_INVALID, "build_stencils: bad node count");
    if (K < 6 || K > 32 || K % 4 != 0 || K > n)
        return set_error(MLBM_E_INVALID, "build_stencils: K must be a multiple of 4 in [8, 32] and <= n");
    const bool points = interp == MLBM_INTERP_RBF_POINTS;
    if (points && (n_l < 7 || n_l > 32 || n_l > n || k_max < K || k_max > 64 || k_max % 4 != 0))
        return set_error(MLBM_E_INVALID,
                         "build_stencils: n_l must be in [7, 32] and <= n, k_max a multiple of 4 in [K, 64]");
    const int Kw = points ? k_max : K;  // device stencil width
    if (use_lagrange && K < 9) return set_error(MLBM_E_INVALID, "build_stencils: Lagrange needs K >= 9");
    if (!(s > 0) || !(sigma_factor > 0)) return set_error(MLBM_E_INVALID, "build_stencils: s and sigma must be > 0");
    if (bb_mode != MLBM_BB_SIMPLE && bb_mode != MLBM_BB_INTERPOLATED)
        return set_error(MLBM_E_INVALID, "build_stencils: bad bb_mode");
    Box b;
    b.x0 = geo->x0; b.y0 = geo->y0; b.x1 = geo->x1; b.y1 = geo->y1;
    b.lx = b.x1 - b.x0; b.ly = b.y1 - b.y0;
    for (int i = 0; i < 4; ++i) {
        b.side[i] = geo->side[i];
        if (b.side[i] < 0 || b.side[i] > 2) return set_error(MLBM_E_INVALID, "build_stencils: bad side type");
    }
    if (!(b.lx > 0) || !(b.ly > 0)) return set_error(MLBM_E_INVALID, "build_stencils: empty box");
    if ((b.side[0] == MLBM_SIDE_PERIODIC) != (b.side[1] == MLBM_SIDE_PERIODIC) ||
        (b.side[2] == MLBM_SIDE_PERIODIC) != (b.side[3] == MLBM_SIDE_PERIODIC))
        return set_error(MLBM_E_INVALID, "build_stencils: periodic sides must come in pairs");
    b.px = b.side[0] == MLBM_SIDE_PERIODIC;
    b.py = b.side[2] == MLBM_SIDE_PERIODIC;
    if (geo->n_disks < 0 || (geo->n_disks > 0 && !geo->disks))
        return set_error(MLBM_E_INVALID, "build_stencils: bad disks");
    for (int64_t i = 0; i < n; ++i) {
        if (nodes->node_class[i] > MLBM_NODE_EQ) return set_error(MLBM_E_INVALID, "build_stencils: bad node class");
        if (nodes->node_class[i] == MLBM_NODE_EQ && !nodes->eq_values)
            return set_error(MLBM_E_INVALID, "build_stencils: equilibrium nodes need eq_values");
        if (!std::isfinite(nodes->xy[2 * i]) || !std::isfinite(nodes->xy[2 * i + 1]))
            return set_error(MLBM_E_INVALID, "build_stencils: non-finite coordinate");
    }
    const auto t0 = std::chrono::steady_clock::now();
    auto* st = new (std::nothrow) mlbm_stencils;
    if (!st) return set_error(MLBM_E_OOM, "build_stencils: out of host memory");
    HostStencils& H = st->h;
    H.n = n;
    H.K = Kw;
    H.s = s;
    H.bb_mode = bb_mode;
    H.interp = interp;
    H.box_area = b.lx * b.ly;
    const double* xy = nodes->xy;
    const CellGrid grid = make_grid(xy, n, b, K);
    const DiskGrid disk_grid = make_disk_grid(b, geo->disks, geo->n_disks, 1.5 * s);

    // caller-order work arrays (nid, Mc, Wc in the device stencil width Kw)
    std::vector<int64_t> nid((size_t)n * Kw);
    std::vector<double> off((size_t)n * K * 2);
    std::vector<double> Mc((size_t)n * 6 * Kw, 0.0);
    std::vector<double> Wc(interp != MLBM_INTERP_WLS ? (size_t)n * 8 * Kw : 0, 0.0);
    std::vector<uint8_t> kind(n), center(n, 0);
    std::vector<double> lagh(n, 0.0), qc((size_t)n * 9, 0.0);
    std::vector<int8_t> slot((size_t)n * 9, 0);
    std::vector<uint16_t> mask(n, 0);
    int64_t bad_node = -1;
    int bad_code = 0;
#pragma omp parallel
    {
        std::vector<double> d2(std::max(K, n_l)), pd2(std::max(n_l, 1)), poff(2 * std::max(n_l, 1)),
            pw(std::max(n_l, 1)), Mown(6 * K);
        std::vector<int64_t> own(K), pid(std::max(n_l, 1)), uni;
        std::vector<std::vector<int64_t>> memb(9);
        std::vector<std::vector<double>> wdir(9);
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) {
            int64_t* nrow = &nid[(size_t)i * Kw];
            knn_one(grid, xy, b, i, K, own.data(), d2.data(), &off[(size_t)i * K * 2]);
            for (int j = 0; j < Kw; ++j) nrow[j] = j < K ? own[j] : i;  // padding: the node itself
            if (nodes->node_class[i] == MLBM_NODE_EQ) {
                kind[i] = kKindEq;
                continue;
            }
            int n_ids = geo->n_disks;
            const int* ids = disk_grid.at(xy[2 * i], xy[2 * i + 1], &n_ids);
            if (!ids) n_ids = geo->n_disks;
            int code = links_of(xy[2 * i], xy[2 * i + 1], s, b, geo->disks, ids, n_ids, &mask[i], &qc[(size_t)i * 9]);
            if (code) {
#pragma omp critical
                { if (bad_node < 0 || i < bad_node) { bad_node = i; bad_code = code; } }
                continue;
            }
            double dx[9], dy[9];
            bool use[9];
            departures(s, mask[i], &qc[(size_t)i * 9], bb_mode, dx, dy, use);
            if (use_lagrange && find_block(&off[(size_t)i * K * 2], K, dx, dy, use, 1e-9, &slot[(size_t)i * 9],
                                           &lagh[i], &center[i])) {
                kind[i] = kKindLagrange;
                continue;
            }
            kind[i] = kKindWls;
            code = wls_qr(&off[(size_t)i * K * 2], K, s, sigma_factor, Mown.data());
            if (!points)
                for (int a = 0; a < 6; ++a)
                    for (int j = 0; j < K; ++j) Mc[((size_t)i * 6 + a) * Kw + j] = Mown[(size_t)a * K + j];
            if (!code && interp == MLBM_INTERP_RBF)
                for (int k = 1; k < 9 && !code; ++k)
                    if (use[k])
                        code = rbf_weights(&off[(size_t)i * K * 2], K, dx[k], dy[k], &Wc[((size_t)i * 8 + k - 1) * K]);
            if (!code && points) {
                // the n_l nearest nodes of every departure point and their
                // weights there; the device stencil is the union with the node
                uni.assign(1, i);
                for (int k = 1; k < 9 && !code; ++k) {
                    memb[k].clear();
                    if (!use[k]) continue;
                    knn_point(grid, xy, b, i, dx[k], dy[k], n_l, pid.data(), pd2.data(), poff.data());
                    code = rbf_weights(poff.data(), n_l, dx[k], dy[k], pw.data());
                    memb[k].assign(pid.begin(), pid.begin() + n_l);
                    wdir[k].assign(pw.begin(), pw.begin() + n_l);
                    uni.insert(uni.end(), pid.begin(), pid.begin() + n_l);
                }
                if (!code) {
                    std::sort(uni.begin(), uni.end());
                    uni.erase(std::unique(uni.begin(), uni.end()), uni.end());
                    if ((int)uni.size() > Kw) code = 9;
                }
                if (!code) {
                    for (int j = 0; j < Kw; ++j) nrow[j] = j < (int)uni.size() ? uni[j] : i;
                    for (int k = 1; k < 9; ++k) {
                        double* row = &Wc[((size_t)i * 8 + k - 1) * Kw];
                        if (!use[k]) {  // simple bounce-back: the kernel copies the node's own value
                            continue;
                        }
                        for (int m = 0; m < n_l; ++m) {
                            const int u = (int)(std::lower_bound(uni.begin(), uni.end(), memb[k][m]) - uni.begin());
                            row[u] = wdir[k][m];
                        }
                    }
                }
            }
            if (code) {
#pragma omp critical
                { if (bad_node < 0 || i < bad_node) { bad_node = i; bad_code = code; } }
            }
        }
    }
    if (bad_node >= 0) {
        delete st;
        if (bad_code == 8)
            return set_error(MLBM_E_GEOMETRY, "build_stencils: node " + std::to_string(bad_node) + " lies inside a solid");
        if (bad_code == 9)
            return set_error(MLBM_E_INVALID, "build_stencils: the departure stencils of node " +
                                                 std::to_string(bad_node) + " hold more than k_max nodes");
        return set_error(MLBM_E_SINGULAR_STENCIL,
                         "build_stencils: degenerate least-squares stencil at node " + std::to_string(bad_node));
    }

    // node order (Hilbert by default)
    H.xy.assign(xy, xy + 2 * (size_t)n);
    H.bx0 = b.x0;
    H.by0 = b.y0;
    H.blx = b.lx;
    H.bly = b.ly;
    H.order = MLBM_ORDER_HILBERT;
    H.perm = order_nodes(H.xy, b.x0, b.y0, b.lx, b.ly, H.order);
    H.inv.resize(n);
    for (int64_t p = 0; p < n; ++p) H.inv[H.perm[p]] = p;

    H.idx.resize((size_t)n * Kw);
    H.M.assign((size_t)n * 6 * Kw, 0.0);
    H.Wr.assign(interp != MLBM_INTERP_WLS ? (size_t)n * 8 * Kw : 0, 0.0);
    H.kind.resize(n);
    H.center.resize(n);
    H.lag_h.resize(n);
    H.lag_slot.resize((size_t)n * 9);
    H.link_mask.resize(n);
    H.q.resize((size_t)n * 9);
    H.eqv.assign((size_t)n * 3, 0.0);
    H.area.resize(n);
    mlbm_stencil_info& I = H.info;
    I = mlbm_stencil_info{};
    I.n = n;
    I.K = Kw;
    I.s = s;
    int64_t n_wls = 0, n_lag = 0, n_eq = 0, n_link_nodes = 0, n_links = 0;
#pragma omp parallel for schedule(static, 4096) reduction(+ : n_wls, n_lag, n_eq, n_link_nodes, n_links)
    for (int64_t p = 0; p < n; ++p) {
        const int64_t i = H.perm[p];
        for (int j = 0; j < Kw; ++j) H.idx[(size_t)p * Kw + j] = (int32_t)H.inv[nid[(size_t)i * Kw + j]];
        std::memcpy(&H.M[(size_t)p * 6 * Kw], &Mc[(size_t)i * 6 * Kw], sizeof(double) * 6 * Kw);
        if (!Wc.empty()) std::memcpy(&H.Wr[(size_t)p * 8 * Kw], &Wc[(size_t)i * 8 * Kw], sizeof(double) * 8 * Kw);
        H.kind[p] = kind[i];
        H.center[p] = center[i];
        H.lag_h[p] = lagh[i];
        std::memcpy(&H.lag_slot[(size_t)p * 9], &slot[(size_t)i * 9], 9);
        H.link_mask[p] = mask[i];
        std::memcpy(&H.q[(size_t)p * 9], &qc[(size_t)i * 9], sizeof(double) * 9);
        if (kind[i] == kKindEq)
            for (int c = 0; c < 3; ++c) H.eqv[(size_t)p * 3 + c] = nodes->eq_values[(size_t)i * 3 + c];
        H.area[p] = nodes->area ? nodes->area[i] : 1.0;
        if (kind[i] == kKindWls) n_wls++;
        else if (kind[i] == kKindLagrange) n_lag++;
        else n_eq++;
        if (mask[i]) {
            n_link_nodes++;
            for (int k = 1; k < 9; ++k) n_links += (mask[i] >> k) & 1;
        }
    }
    I.n_wls = n_wls;
    I.n_lagrange = n_lag;
    I.n_eq = n_eq;
    I.n_link_nodes = n_link_nodes;
    I.n_links = n_links;
    I.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = st;
    return MLBM_OK;
}

}  // namespace

extern "C" mlbm_status mlbm_build_stencils_ex(const mlbm_nodes* nodes, const mlbm_geometry* geo, int K, double s,
                                              double sigma_factor, int bb_mode, int use_lagrange, int interp,
                                              mlbm_stencils** out) {
    if (interp == MLBM_INTERP_RBF_POINTS)
        return set_error(MLBM_E_INVALID, "build_stencils_ex: stencils per departure point need "
                                         "mlbm_build_stencils_points");
    return build_impl(nodes, geo, K, s, sigma_factor, bb_mode, use_lagrange, interp, 0, K, out);
}

extern "C" mlbm_status mlbm_build_stencils_points(const mlbm_nodes* nodes, const mlbm_geometry* geo, int n_l,
                                                  int k_max, double s, int bb_mode, int use_lagrange,
                                                  mlbm_stencils** out) {
    return build_impl(nodes, geo, 16, s, 0.7071067811865476, bb_mode, use_lagrange, MLBM_INTERP_RBF_POINTS, n_l,
                      k_max, out);
}

extern "C" void mlbm_stencils_free(mlbm_stencils* st) { delete st; }

extern "C" mlbm_status mlbm_stencils_info(const mlbm_stencils* st, mlbm_stencil_info* info) {
    if (!st || !info) return set_error(MLBM_E_INVALID, "stencils_info: NULL argument");
    *info = st->h.info;
    return MLBM_OK;
}

extern "C" mlbm_status mlbm_stencils_export(const mlbm_stencils* st, int64_t* idx, double* M, int32_t* kind,
                                            int32_t* link_mask, double* q, double* lag_h, int32_t* lag_center) {
    if (!st) return set_error(MLBM_E_INVALID, "stencils_export: NULL stencils");
    const HostStencils& H = st->h;
    const int K = H.K;
    for (int64_t p = 0; p < H.n; ++p) {
        const int64_t i = H.perm[p];
        if (idx)
            for (int j = 0; j < K; ++j) idx[(size_t)i * K + j] = H.perm[H.idx[(size_t)p * K + j]];
        if (M) std::memcpy(&M[(size_t)i * 6 * K], &H.M[(size_t)p * 6 * K], sizeof(double) * 6 * K);
        if (kind) kind[i] = H.kind[p];
        if (link_mask) link_mask[i] = H.link_mask[p];
        if (q) std::memcpy(&q[(size_t)i * 9], &H.q[(size_t)p * 9], sizeof(double) * 9);
        if (lag_h) lag_h[i] = H.lag_h[p];
        if (lag_center) lag_center[i] = H.center[p];
    }
    return MLBM_OK;
}

extern "C" mlbm_status mlbm_stencils_set_order(mlbm_stencils* st, int order) {
    clear_error();
    if (!st || order < MLBM_ORDER_HILBERT || order > MLBM_ORDER_INPUT)
        return set_error(MLBM_E_INVALID, "stencils_set_order: bad arguments");
    HostStencils& H = st->h;
    if (H.order == order) return MLBM_OK;
    if ((int64_t)H.xy.size() != 2 * H.n)
        return set_error(MLBM_E_INVALID, "stencils_set_order: these stencils carry no node positions");
    const int64_t n = H.n;
    const int K = H.K;
    std::vector<int64_t> perm = order_nodes(H.xy, H.bx0, H.by0, H.blx, H.bly, order);
    std::vector<int64_t> inv(n);
    for (int64_t p = 0; p < n; ++p) inv[perm[p]] = p;
    // new position q takes what sat at old position H.inv[perm[q]]; neighbour
    // positions are mapped through the caller ids
    auto move = [&](auto& v, size_t w) {
        auto old = v;
        for (int64_t q = 0; q < n; ++q) {
            const int64_t o = H.inv[perm[q]];
            std::copy(old.begin() + (size_t)o * w, old.begin() + (size_t)(o + 1) * w, v.begin() + (size_t)q * w);
        }
    };
    {
        std::vector<int32_t> old = H.idx;
        for (int64_t q = 0; q < n; ++q) {
            const int64_t o = H.inv[perm[q]];
            for (int j = 0; j < K; ++j) H.idx[(size_t)q * K + j] = (int32_t)inv[H.perm[old[(size_t)o * K + j]]];
        }
    }
    move(H.M, (size_t)6 * K);
    if (!H.Wr.empty()) move(H.Wr, (size_t)8 * K);
    move(H.kind, 1);
    move(H.center, 1);
    move(H.lag_h, 1);
    move(H.lag_slot, 9);
    move(H.link_mask, 1);
    move(H.q, 9);
    move(H.eqv, 3);
    move(H.area, 1);
    if (!H.s_node.empty()) move(H.s_node, 1);
    H.perm = std::move(perm);
    H.inv = std::move(inv);
    H.order = order;
    return MLBM_OK;
}

extern "C" int mlbm_stencils_order(const mlbm_stencils* st) { return st ? st->h.order : -1; }

extern "C" mlbm_status mlbm_stencils_export_weights(const mlbm_stencils* st, double* W) {
    if (!st || !W) return set_error(MLBM_E_INVALID, "stencils_export_weights: NULL argument");
    const HostStencils& H = st->h;
    if (H.interp == MLBM_INTERP_WLS) return set_error(MLBM_E_INVALID, "stencils_export_weights: not RBF-FD stencils");
    const int K = H.K;
    for (int64_t p = 0; p < H.n; ++p) {
        const int64_t i = H.perm[p];
        std::memset(&W[(size_t)i * 9 * K], 0, sizeof(double) * K);
        std::memcpy(&W[((size_t)i * 9 + 1) * K], &H.Wr[(size_t)p * 8 * K], sizeof(double) * 8 * K);
    }
    return MLBM_OK;
}
