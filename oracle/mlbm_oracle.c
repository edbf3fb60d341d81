/*
 * FP64 CPU oracle of the meshless lattice Boltzmann (MLBM) time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code with the
 * CUDA path (no headers, constants, tables or helpers); both read the same
 * seeded node sets and nothing else.
 *
 * Plain, slow and direct: every loop follows the paper's equations in the
 * order they are written, in double precision (long double for the least
 * squares normal equations).  Paper: Strzelczyk & Matyka, "Modeling inertial
 * flows with meshless Lattice Boltzmann Method" (arXiv 2312.14789).
 *
 *   Eq. (1)  lattice streaming, Eq. (2) D2Q9 streaming vectors e_k
 *   Eq. (3)  TRT collision, Eq. (4) symmetric/antisymmetric parts
 *   Eq. (6)  nu = c_s^2 (tau+ - 1/2)
 *   Eq. (7)  equilibrium f^eq, Eq. (8) weights omega_k
 *   Eq. (9)  moments rho, u
 *   Eq. (10)-(11)  LBM1 (tau = 1)
 *   Sec. 2.2, Eq. (12)  semi-Lagrangian meshless streaming
 *           f_k(t+1, x) = f_k^post(t, x + dx_{k'}) ~ sum_i w_i^k f_k^post(t, x_i)
 *   Sec. 2.2 biquadratic Lagrange interpolation on regular 3x3 stencils
 *   Eq. (14)-(15)  MLBM1: macroscopic fields interpolated to the departure
 *           points, equilibria summed there
 *   Sec. 3.1 simple bounce-back where the departure point lies in the solid;
 *           equilibrium overwrite on straight inflow/outflow/side boundaries
 *   Sec. 3.2, Eq. (22) interpolated bounce-back with boundary nodes on the
 *           wall, f_k(t+1, x) = f_{k'}^post(t, x + dx_k); periodic sides by
 *           periodic stencil search; body force with a second-order source
 *
 * Readings where the paper is silent (listed with reasons in the design
 * notes): the interpolant is a second-order Gaussian-weighted least squares
 * fit over the K nearest nodes of the Eulerian node; ties in the neighbour
 * search go to the lower node id; the interpolated bounce-back for a wall at
 * fraction q of the streaming distance uses the departure point
 * x + (1 - 2q) s e_k (q = 0 gives the paper's wall-node rule).
 *
 * Parity pins for every function here live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- D2Q9 --- */
/* Eq. (2): e_k in the paper's order */
static const int OEX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int OEY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* k' with e_{k'} = -e_k */
static const int OOPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* omega_k, Eq. (8) */
static double oomega(int k) {
    if (k == 0) return 4.0 / 9.0;
    if (k <= 4) return 1.0 / 9.0;
    return 1.0 / 36.0;
}
static const double CS2 = 1.0 / 3.0; /* c_s^2, c_s = 1/sqrt(3) */

int oracle_ex(int k) { return OEX[k]; }
int oracle_ey(int k) { return OEY[k]; }
int oracle_opp(int k) { return OOPP[k]; }
double oracle_omega(int k) { return oomega(k); }

/* Eq. (7) */
double oracle_feq(int k, double rho, double ux, double uy) {
    double eu = OEX[k] * ux + OEY[k] * uy;
    double uu = ux * ux + uy * uy;
    return oomega(k) * rho * (1.0 + eu / CS2 + (eu * eu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/*
 * Body-force source, second order in velocity (Guo et al. form):
 *   S_k = omega_k [ (e_k - u) / c_s^2 + (e_k . u) e_k / c_s^4 ] . F,  F = rho g.
 * Its zeroth moment is 0 and its first moment is F.
 */
double oracle_source(int k, double rho, double ux, double uy, double gx, double gy) {
    double Fx = rho * gx, Fy = rho * gy;
    double eu = OEX[k] * ux + OEY[k] * uy;
    double ax = (OEX[k] - ux) / CS2 + eu * OEX[k] / (CS2 * CS2);
    double ay = (OEY[k] - uy) / CS2 + eu * OEY[k] / (CS2 * CS2);
    return oomega(k) * (ax * Fx + ay * Fy);
}

/*
 * Eq. (9) with the force correction: rho = sum f, rho u = sum f e + F/2.
 */
void oracle_moments(const double* f, double gx, double gy, double* rho, double* ux, double* uy) {
    double r = 0, mx = 0, my = 0;
    for (int k = 0; k < 9; ++k) { r += f[k]; mx += f[k] * OEX[k]; my += f[k] * OEY[k]; }
    *rho = r;
    *ux = mx / r + 0.5 * gx;
    *uy = my / r + 0.5 * gy;
}

/*
 * Eq. (3)-(4), TRT collision (BGK when tau_m == tau_p), plus the source split
 * the same way: (1 - 1/(2 tau+)) S^+ + (1 - 1/(2 tau-)) S^-.
 * f: pre-collision populations of one node; out: post-collision.
 */
void oracle_collide(const double* f, double tau_p, double tau_m, double gx, double gy, double* out) {
    double rho, ux, uy;
    oracle_moments(f, gx, gy, &rho, &ux, &uy);
    double feq[9], S[9];
    for (int k = 0; k < 9; ++k) {
        feq[k] = oracle_feq(k, rho, ux, uy);
        S[k] = oracle_source(k, rho, ux, uy, gx, gy);
    }
    for (int k = 0; k < 9; ++k) {
        int kp = OOPP[k];
        double fp = 0.5 * (f[k] + f[kp]), fm = 0.5 * (f[k] - f[kp]);
        double ep = 0.5 * (feq[k] + feq[kp]), em = 0.5 * (feq[k] - feq[kp]);
        double sp = 0.5 * (S[k] + S[kp]), sm = 0.5 * (S[k] - S[kp]);
        out[k] = f[k] - (fp - ep) / tau_p - (fm - em) / tau_m
               + (1.0 - 0.5 / tau_p) * sp + (1.0 - 0.5 / tau_m) * sm;
    }
}

/* ------------------------------------------------------- neighbour search --- */
/* minimum image on a periodic side: offset wrapped into [-L/2, L/2) */
static double omin_image(double d, double L, int periodic) {
    if (!periodic) return d;
    if (d >= 0.5 * L) d -= L;
    if (d < -0.5 * L) d += L;
    return d;
}

/*
 * Brute-force K nearest neighbours of each target node among all n nodes,
 * self included (distance 0), ordered by (d^2, node id).  Offsets x_j - x use
 * the minimum image across periodic sides (Sec. 3.2: periodic stencil search).
 * box = {x0, y0, x1, y1}.  Returns 0, or 1 when K > n.
 */
int oracle_knn(const double* xy, int64_t n, const double* box, int periodic_x, int periodic_y, int K,
               const int64_t* targets, int64_t nt, int64_t* idx_out, double* off_out) {
    if (K > n || K < 1) return 1;
    double Lx = box[2] - box[0], Ly = box[3] - box[1];
#pragma omp parallel
    {
    double* bd = (double*)malloc(sizeof(double) * K);
    int64_t* bi = (int64_t*)malloc(sizeof(int64_t) * K);
#pragma omp for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        double xi = xy[2 * i], yi = xy[2 * i + 1];
        int cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            double dx = omin_image(xy[2 * j] - xi, Lx, periodic_x);
            double dy = omin_image(xy[2 * j + 1] - yi, Ly, periodic_y);
            double d2 = dx * dx + dy * dy;
            /* insertion into the sorted list of the best K so far */
            if (cnt == K) {
                double wd = bd[K - 1];
                int64_t wi = bi[K - 1];
                if (d2 > wd || (d2 == wd && j > wi)) continue;
                cnt--;
            }
            int pos = cnt;
            while (pos > 0 && (bd[pos - 1] > d2 || (bd[pos - 1] == d2 && bi[pos - 1] > j))) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                pos--;
            }
            bd[pos] = d2;
            bi[pos] = j;
            cnt++;
        }
        for (int m = 0; m < K; ++m) {
            int64_t j = bi[m];
            idx_out[t * K + m] = j;
            off_out[2 * (t * K + m)] = omin_image(xy[2 * j] - xi, Lx, periodic_x);
            off_out[2 * (t * K + m) + 1] = omin_image(xy[2 * j + 1] - yi, Ly, periodic_y);
        }
    }
    free(bd);
    free(bi);
    }
    return 0;
}

/* ------------------------------------------------------ weighted LSQ fit --- */
/* quadratic basis p(r) = [1, x, y, x^2, x y, y^2] */
static void obasis(double x, double y, double* p) {
    p[0] = 1.0; p[1] = x; p[2] = y; p[3] = x * x; p[4] = x * y; p[5] = y * y;
}
static const int ODEG[6] = {0, 1, 1, 2, 2, 2};

/*
 * Second-order weighted least squares through the K stencil nodes
 * (offsets off[K][2] from the Eulerian node).  Gaussian weights
 * W_j = exp(-|r_j|^2 / sigma^2), sigma = sigma_factor * r_K with r_K the
 * largest stencil offset.  With P the K x 6 basis matrix,
 *     M = (P^T W P)^{-1} P^T W              (6 x K),
 * so that the fitted polynomial's coefficients are c = M f and its value at
 * offset d is p(d)^T M f.  The normal equations are solved in long double by
 * Gauss-Jordan elimination with partial pivoting, on offsets divided by r_K.
 *
 * Output M_out[6][K] is in streaming-distance units: row i is multiplied by
 * s^deg(i), so that the value at offset d equals p(d/s)^T M_out f.
 * Returns 0, or 2 when the 1-norm condition number of the (scaled) normal
 * matrix exceeds 1e12 (a degenerate stencil).
 */
int oracle_wls_matrix(const double* off, int K, double s, double sigma_factor, double* M_out) {
    double rK = 0;
    for (int j = 0; j < K; ++j) {
        double r = sqrt(off[2 * j] * off[2 * j] + off[2 * j + 1] * off[2 * j + 1]);
        if (r > rK) rK = r;
    }
    if (!(rK > 0)) return 2;
    double sigma = sigma_factor * rK;
    long double A[6][12];
    long double B[6][64];
    if (K > 64) return 1;
    for (int a = 0; a < 6; ++a) {
        for (int b = 0; b < 12; ++b) A[a][b] = 0;
        for (int j = 0; j < K; ++j) B[a][j] = 0;
    }
    for (int j = 0; j < K; ++j) {
        double x = off[2 * j], y = off[2 * j + 1];
        double w = exp(-(x * x + y * y) / (sigma * sigma));
        double p[6];
        obasis(x / rK, y / rK, p);
        for (int a = 0; a < 6; ++a) {
            for (int b = 0; b < 6; ++b) A[a][b] += (long double)w * p[a] * p[b];
            B[a][j] = (long double)w * p[a];
        }
    }
    /* augmented [A | I] -> [I | A^-1] */
    long double norm_a = 0;
    for (int b = 0; b < 6; ++b) {
        long double cs = 0;
        for (int a = 0; a < 6; ++a) cs += fabsl(A[a][b]);
        if (cs > norm_a) norm_a = cs;
    }
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) A[a][6 + b] = (a == b) ? 1.0L : 0.0L;
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        for (int r = c + 1; r < 6; ++r)
            if (fabsl(A[r][c]) > fabsl(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0L) return 2;
        if (piv != c)
            for (int b = 0; b < 12; ++b) { long double t = A[c][b]; A[c][b] = A[piv][b]; A[piv][b] = t; }
        long double d = A[c][c];
        for (int b = 0; b < 12; ++b) A[c][b] /= d;
        for (int r = 0; r < 6; ++r) {
            if (r == c) continue;
            long double m = A[r][c];
            if (m == 0.0L) continue;
            for (int b = 0; b < 12; ++b) A[r][b] -= m * A[c][b];
        }
    }
    long double norm_inv = 0;
    for (int b = 0; b < 6; ++b) {
        long double cs = 0;
        for (int a = 0; a < 6; ++a) cs += fabsl(A[a][6 + b]);
        if (cs > norm_inv) norm_inv = cs;
    }
    if (norm_a * norm_inv > 1e12L) return 2;
    for (int a = 0; a < 6; ++a) {
        double scale = pow(s / rK, ODEG[a]);
        for (int j = 0; j < K; ++j) {
            long double acc = 0;
            for (int b = 0; b < 6; ++b) acc += A[a][6 + b] * B[b][j];
            M_out[a * K + j] = (double)(acc * scale);
        }
    }
    return 0;
}

/* ------------------------------------------------ biquadratic Lagrange --- */
/* 1D quadratic Lagrange basis on nodes {-1, 0, 1}, evaluated at t */
static void olagrange3(double t, double* l) {
    l[0] = 0.5 * t * (t - 1.0);
    l[1] = (1.0 - t) * (1.0 + t);
    l[2] = 0.5 * t * (t + 1.0);
}

/*
 * Regular-stencil test (Sec. 2.2: biquadratic Lagrange where the nine nodes
 * around a departure point form a square lattice, RBF-FD-like fit
 * elsewhere).  h is the smallest non-zero stencil offset.  Candidate blocks
 * are the axis-aligned 3x3 blocks {c + h(a, b)}, a, b in {-1, 0, 1}, with
 * centre c = x + h e_m tried in the D2Q9 order m = 0..8 (the centred block
 * first).  A block is taken when all nine of its points are stencil members
 * (each within tol * h) and every departure point the node interpolates at
 * (dep_x[k], dep_y[k] for the directions with use[k] set) lies inside it
 * (|offset from c| <= h (1 + tol) per axis).
 * On success returns 1, slot[(b+1)*3 + (a+1)] = stencil position of
 * c + h(a, b), *h_out = h and *center_out = m.
 */
int oracle_lagrange_detect(const double* off, int K, double tol, const double* dep_x, const double* dep_y,
                           const int* use, int* slot, double* h_out, int* center_out) {
    double h = 0;
    for (int j = 0; j < K; ++j) {
        double r = sqrt(off[2 * j] * off[2 * j] + off[2 * j + 1] * off[2 * j + 1]);
        if (r > 0 && (h == 0 || r < h)) h = r;
    }
    if (h == 0) return 0;
    for (int m = 0; m < 9; ++m) {
        double cx = OEX[m] * h, cy = OEY[m] * h;
        int ok = 1;
        for (int k = 1; k < 9 && ok; ++k) {
            if (!use[k]) continue;
            if (fabs(dep_x[k] - cx) > h * (1.0 + tol) || fabs(dep_y[k] - cy) > h * (1.0 + tol)) ok = 0;
        }
        for (int b = -1; b <= 1 && ok; ++b)
            for (int a = -1; a <= 1 && ok; ++a) {
                int found = -1;
                for (int j = 0; j < K; ++j) {
                    double dx = off[2 * j] - (cx + a * h), dy = off[2 * j + 1] - (cy + b * h);
                    if (fabs(dx) <= tol * h && fabs(dy) <= tol * h) { found = j; break; }
                }
                if (found < 0) ok = 0;
                else slot[(b + 1) * 3 + (a + 1)] = found;
            }
        if (ok) {
            *h_out = h;
            *center_out = m;
            return 1;
        }
    }
    return 0;
}

/* departure offsets of Eq. (12) and of the bounce-back rules, per direction:
   use[k] = 0 for simple bounce-back links (no interpolation) */
static void odepartures(double s, const int* link, const double* q, int bb_mode, double* dx, double* dy,
                        int* use) {
    use[0] = 0; dx[0] = dy[0] = 0;
    for (int k = 1; k < 9; ++k) {
        if (link[k]) {
            if (bb_mode == 0) { use[k] = 0; dx[k] = dy[k] = 0; continue; }
            double t = 1.0 - 2.0 * q[k];
            dx[k] = t * s * OEX[k];
            dy[k] = t * s * OEY[k];
        } else {
            dx[k] = -s * OEX[k];
            dy[k] = -s * OEY[k];
        }
        use[k] = 1;
    }
}

/* ----------------------------------------------------- boundary links --- */
/*
 * For each direction k = 1..8, does the departure segment from x to
 * x - s e_k enter a solid?  Solids: disks (cx, cy, r), with periodic images,
 * and the sides of the box whose type is 1 (solid wall; 0 periodic, 2 open).
 * side = {left, right, bottom, top}.  q_out[k] in [0, 1) is the entry point as
 * a fraction of s along the segment; link_out[k] = 1 when it exists.
 * A node lying on a solid surface (within 1e-9 relative) has q = 0 for the
 * directions pointing into the solid.  Returns 0, or 3 when x is inside a
 * solid.
 */
int oracle_bc_links(double x, double y, double s, const double* box, const int* side,
                    const double* disks, int ndisks, int* link_out, double* q_out) {
    double Lx = box[2] - box[0], Ly = box[3] - box[1];
    double tol = 1e-9 * s;
    link_out[0] = 0; q_out[0] = 0;
    for (int k = 1; k < 9; ++k) {
        double best = 2.0;
        double vx = -s * OEX[k], vy = -s * OEY[k]; /* segment x + t v, t in [0, 1] */
        /* straight solid sides */
        if (side[2] == 1 && vy < 0) {
            double dist = y - box[1];
            if (dist < -tol) return 3;
            double t = dist <= tol ? 0.0 : dist / (-vy);
            if (t < 1.0 && t < best) best = t;
        }
        if (side[3] == 1 && vy > 0) {
            double dist = box[3] - y;
            if (dist < -tol) return 3;
            double t = dist <= tol ? 0.0 : dist / vy;
            if (t < 1.0 && t < best) best = t;
        }
        if (side[0] == 1 && vx < 0) {
            double dist = x - box[0];
            if (dist < -tol) return 3;
            double t = dist <= tol ? 0.0 : dist / (-vx);
            if (t < 1.0 && t < best) best = t;
        }
        if (side[1] == 1 && vx > 0) {
            double dist = box[2] - x;
            if (dist < -tol) return 3;
            double t = dist <= tol ? 0.0 : dist / vx;
            if (t < 1.0 && t < best) best = t;
        }
        /* disks and their periodic images */
        for (int i = 0; i < ndisks; ++i) {
            for (int ix = -1; ix <= 1; ++ix) {
                if (ix != 0 && side[0] != 0) continue;
                for (int iy = -1; iy <= 1; ++iy) {
                    if (iy != 0 && side[2] != 0) continue;
                    double cx = disks[3 * i] + ix * Lx, cy = disks[3 * i + 1] + iy * Ly, R = disks[3 * i + 2];
                    double rx = x - cx, ry = y - cy;
                    double dist = sqrt(rx * rx + ry * ry);
                    if (dist < R * (1.0 - 1e-9)) return 3;
                    double b = rx * vx + ry * vy; /* half the derivative of |r + t v|^2 at t = 0 */
                    if (dist <= R * (1.0 + 1e-9)) {
                        if (b < 0) best = 0.0;
                        continue;
                    }
                    double a = vx * vx + vy * vy;
                    double c = rx * rx + ry * ry - R * R;
                    double disc = b * b - a * c;
                    if (disc <= 0) continue;
                    double t = (-b - sqrt(disc)) / a;
                    if (t >= 0 && t < 1.0 && t < best) best = t;
                }
            }
        }
        link_out[k] = best < 1.0;
        q_out[k] = best < 1.0 ? best : 0.0;
    }
    return 0;
}

/* ---------------------------------------------- per-direction weights --- */
/*
 * Weights of Eq. (12) for one Eulerian node: for k = 1..8, w[k][j] such that
 * f_k(t+1, x) = sum_j w[k][j] f_{src[k]}^post(t, x_j).
 *   no link:                 departure offset d = -s e_k, src = k
 *   link, simple bounce-back: one-hot on the node itself, src = k'
 *   link, interpolated:      d = (1 - 2 q) s e_k, src = k'
 * interpolation by the WLS matrix (p(d/s)^T M) or, for a regular stencil,
 * biquadratic Lagrange at (d - c) / h with c the block centre.
 * self_slot: stencil position of the node itself.
 * w_out: [9][K] (row 0 unused, zero).
 */
/*
 * RBF-FD weights (Sec. 2.2: the paper's interpolant, polyharmonic spline
 * phi(r) = r^3 augmented with the quadratic monomials): for the stencil
 * offsets o_j (j < K) and an evaluation point d, the weights w solve
 *     [ Phi  P ] [ w      ]   [ phi(|o_i - d|) ]
 *     [ P^T  0 ] [ lambda ] = [ p(d)           ]
 * with Phi_ij = |o_i - o_j|^3 and P_ia = p_a(o_i), p = (1, x, y, x^2, xy, y^2);
 * then sum_j w_j f_j is the value at d of the cubic-PHS interpolant of the
 * data f_j with quadratic augmentation.  Coordinates are divided by the
 * largest offset first (the weights do not change: r^3 is homogeneous and
 * the quadratic space is closed under scaling).  Gauss-Jordan elimination
 * with partial pivoting in long double; returns 2 on a singular system.
 */
int oracle_rbf_weights(const double* off, int K, double dx, double dy, double* w_out) {
    const int N = K + 6;
    if (K > 64) return 1;
    double rK = 0;
    for (int j = 0; j < K; ++j) {
        double r = sqrt(off[2 * j] * off[2 * j] + off[2 * j + 1] * off[2 * j + 1]);
        if (r > rK) rK = r;
    }
    if (!(rK > 0)) return 2;
    long double A[70][71];
    for (int i = 0; i < N; ++i)
        for (int j = 0; j <= N; ++j) A[i][j] = 0;
    for (int i = 0; i < K; ++i) {
        const double xi = off[2 * i] / rK, yi = off[2 * i + 1] / rK;
        for (int j = 0; j < K; ++j) {
            const double ex = xi - off[2 * j] / rK, ey = yi - off[2 * j + 1] / rK;
            const double r = sqrt(ex * ex + ey * ey);
            A[i][j] = (long double)r * r * r;
        }
        double p[6];
        obasis(xi, yi, p);
        for (int a = 0; a < 6; ++a) {
            A[i][K + a] = p[a];
            A[K + a][i] = p[a];
        }
        const double qx = xi - dx / rK, qy = yi - dy / rK;
        const double rq = sqrt(qx * qx + qy * qy);
        A[i][N] = (long double)rq * rq * rq;
    }
    double pd[6];
    obasis(dx / rK, dy / rK, pd);
    for (int a = 0; a < 6; ++a) A[K + a][N] = pd[a];
    for (int c = 0; c < N; ++c) {
        int piv = c;
        for (int r = c + 1; r < N; ++r)
            if (fabsl(A[r][c]) > fabsl(A[piv][c])) piv = r;
        if (fabsl(A[piv][c]) < 1e-300L) return 2;
        if (piv != c)
            for (int b = 0; b <= N; ++b) { long double t = A[c][b]; A[c][b] = A[piv][b]; A[piv][b] = t; }
        for (int r = 0; r < N; ++r) {
            if (r == c) continue;
            long double m = A[r][c] / A[c][c];
            if (m == 0.0L) continue;
            for (int b = c; b <= N; ++b) A[r][b] -= m * A[c][b];
        }
    }
    for (int j = 0; j < K; ++j) w_out[j] = (double)(A[j][N] / A[j][j]);
    return 0;
}

void oracle_direction_weights(int K, int kind, const double* M, const int* lag_slot, double lag_h,
                              int lag_center, double s, int self_slot, const int* link, const double* q,
                              int bb_mode, double* w_out, int* src_out) {
    double dx[9], dy[9];
    int use[9];
    odepartures(s, link, q, bb_mode, dx, dy, use);
    memset(w_out, 0, sizeof(double) * 9 * K);
    src_out[0] = 0;
    for (int k = 1; k < 9; ++k) {
        src_out[k] = link[k] ? OOPP[k] : k;
        if (!use[k]) {
            w_out[k * K + self_slot] = 1.0;
            continue;
        }
        if (kind == 0) {
            double p[6];
            obasis(dx[k] / s, dy[k] / s, p);
            for (int j = 0; j < K; ++j) {
                double acc = 0;
                for (int a = 0; a < 6; ++a) acc += p[a] * M[a * K + j];
                w_out[k * K + j] = acc;
            }
        } else {
            double lx[3], ly[3];
            olagrange3(dx[k] / lag_h - OEX[lag_center], lx);
            olagrange3(dy[k] / lag_h - OEY[lag_center], ly);
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a)
                    w_out[k * K + lag_slot[b * 3 + a]] += lx[a] * ly[b];
        }
    }
}

/* ------------------------------------------------------------ MLBM step --- */
/*
 * One MLBM time step (Sec. 2.2): streaming by Eq. (12) from the
 * post-collision field f_in[n][9], then Eq. (9) moments and Eq. (3)
 * collision, for each target node.  f_0 is taken from the node itself (not
 * interpolated).  Class-2 nodes (equilibrium overwrite, Sec. 3.1) are set to
 * f^eq(rho_b, u_b) with eq_val[node] = (rho_b, ux_b, uy_b).
 * W: [nt][9][K] weights, src: [nt][9], idx: [nt][K] (node ids), per target.
 * f_out: [nt][9] post-collision populations of the targets.
 */
void oracle_mlbm_step(int64_t n, const double* f_in, int64_t nt, const int64_t* targets, int K,
                      const int64_t* idx, const double* W, const int* src, const uint8_t* node_class,
                      const double* eq_val, double tau_p, double tau_m, double gx, double gy,
                      double* f_out) {
    (void)n;
    /* small node sets run on one thread: the fork and join of a parallel
       region would cost more than the step (every node is independent, so
       the result does not depend on the thread count) */
#pragma omp parallel for schedule(static) if (nt >= 16384)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        double f[9];
        if (node_class[i] == 2) {
            for (int k = 0; k < 9; ++k)
                f_out[9 * t + k] = oracle_feq(k, eq_val[3 * i], eq_val[3 * i + 1], eq_val[3 * i + 2]);
            continue;
        }
        f[0] = f_in[9 * i + 0];
        for (int k = 1; k < 9; ++k) {
            double acc = 0;
            int sk = src[9 * t + k];
            for (int j = 0; j < K; ++j)
                acc += W[(t * 9 + k) * K + j] * f_in[9 * idx[t * K + j] + sk];
            f[k] = acc;
        }
        oracle_collide(f, tau_p, tau_m, gx, gy, f_out + 9 * t);
    }
}

/*
 * One MLBM1 time step (Eq. (14)-(15)), tau = 1: the stored state is
 * (rho, ux, uy)[n].  For k = 1..8 the density and velocity are interpolated
 * to the departure point with the same weights as Eq. (12) (velocity, not
 * momentum, is interpolated), the post-collision population there is
 * f^eq_src(rho_d, u_d) + S_src/2, and the new moments are their sums with the
 * node's own k = 0 term; rho u(t+1) = sum f e + rho g / 2.
 */
void oracle_mlbm1_step(int64_t n, const double* ru_in, int64_t nt, const int64_t* targets, int K,
                       const int64_t* idx, const double* W, const int* src, const uint8_t* node_class,
                       const double* eq_val, double gx, double gy, double* ru_out) {
    (void)n;
#pragma omp parallel for schedule(static) if (nt >= 16384)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        if (node_class[i] == 2) {
            ru_out[3 * t] = eq_val[3 * i];
            ru_out[3 * t + 1] = eq_val[3 * i + 1];
            ru_out[3 * t + 2] = eq_val[3 * i + 2];
            continue;
        }
        double f[9];
        {
            double r = ru_in[3 * i], ux = ru_in[3 * i + 1], uy = ru_in[3 * i + 2];
            f[0] = oracle_feq(0, r, ux, uy) + 0.5 * oracle_source(0, r, ux, uy, gx, gy);
        }
        for (int k = 1; k < 9; ++k) {
            double r = 0, ux = 0, uy = 0;
            for (int j = 0; j < K; ++j) {
                double w = W[(t * 9 + k) * K + j];
                int64_t m = idx[t * K + j];
                r += w * ru_in[3 * m];
                ux += w * ru_in[3 * m + 1];
                uy += w * ru_in[3 * m + 2];
            }
            int sk = src[9 * t + k];
            f[k] = oracle_feq(sk, r, ux, uy) + 0.5 * oracle_source(sk, r, ux, uy, gx, gy);
        }
        double rho = 0, mx = 0, my = 0;
        for (int k = 0; k < 9; ++k) { rho += f[k]; mx += f[k] * OEX[k]; my += f[k] * OEY[k]; }
        ru_out[3 * t] = rho;
        ru_out[3 * t + 1] = mx / rho + 0.5 * gx;
        ru_out[3 * t + 2] = my / rho + 0.5 * gy;
    }
}

/*
 * Momentum handed to the solids in the next streaming step (momentum
 * exchange over bounce-back links): for each link (x, k) the population
 * f_{k'} that would leave into the solid returns as f_k(t+1, x); the solid
 * receives (f_{k'} + f_k) e_{k'} = 2 f_k(t+1, x) e_{k'} per unit lattice
 * area, weighted by the node area in lattice units, area_x / s^2.  The rest
 * state (f_k = omega_k, uniform pressure) exerts no net force on a closed
 * body but its link sum on scattered nodes does not cancel exactly, so the
 * exchange is taken relative to it: 2 (f_k(t+1, x) - omega_k) e_{k'}.
 * For the BGK state f_in[n][9]; link_mask[t][9] marks link directions.
 */
void oracle_force_bgk(int64_t nt, const int64_t* targets, int K, const int64_t* idx, const double* W,
                      const int* src, const int* link_mask, const double* f_in, const double* area,
                      double s, double* fx, double* fy) {
    double sx = 0, sy = 0;
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        for (int k = 1; k < 9; ++k) {
            if (!link_mask[9 * t + k]) continue;
            double acc = 0;
            int sk = src[9 * t + k];
            for (int j = 0; j < K; ++j) acc += W[(t * 9 + k) * K + j] * f_in[9 * idx[t * K + j] + sk];
            double a = area[i] / (s * s);
            sx += 2.0 * (acc - oomega(k)) * OEX[OOPP[k]] * a;
            sy += 2.0 * (acc - oomega(k)) * OEY[OOPP[k]] * a;
        }
    }
    *fx = sx;
    *fy = sy;
}

/* the same for the MLBM1 state (rho, ux, uy)[n] */
void oracle_force_mlbm1(int64_t nt, const int64_t* targets, int K, const int64_t* idx, const double* W,
                        const int* src, const int* link_mask, const double* ru_in, const double* area,
                        double s, double gx, double gy, double* fx, double* fy) {
    double sx = 0, sy = 0;
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        for (int k = 1; k < 9; ++k) {
            if (!link_mask[9 * t + k]) continue;
            double r = 0, ux = 0, uy = 0;
            for (int j = 0; j < K; ++j) {
                double w = W[(t * 9 + k) * K + j];
                int64_t m = idx[t * K + j];
                r += w * ru_in[3 * m];
                ux += w * ru_in[3 * m + 1];
                uy += w * ru_in[3 * m + 2];
            }
            int sk = src[9 * t + k];
            double fk = oracle_feq(sk, r, ux, uy) + 0.5 * oracle_source(sk, r, ux, uy, gx, gy);
            double a = area[i] / (s * s);
            sx += 2.0 * (fk - oomega(k)) * OEX[OOPP[k]] * a;
            sy += 2.0 * (fk - oomega(k)) * OEY[OOPP[k]] * a;
        }
    }
    *fx = sx;
    *fy = sy;
}

/* ------------------------------------------------ per-node assembly --- */
/*
 * Everything the step needs for each target node, from its stencil
 * (idx/off from oracle_knn): the WLS matrix or the Lagrange block, the
 * bounce-back links and the per-direction weights (interp = 1: the
 * least-squares rows are replaced by RBF-FD rows at the same points).
 *   kind[t]: 0 WLS, 1 Lagrange (only when use_lagrange), 2 equilibrium node
 *            (no weights needed)
 *   status[t]: 0, or the code of the failing routine (2 degenerate stencil,
 *              3 node inside a solid)
 * Arrays are per target: M[6][K], lag_slot[9], lag_h, link[9], q[9], W[9][K],
 * src[9].
 */
void oracle_assemble(int64_t nt, const int64_t* targets, int K, const int64_t* idx, const double* off,
                     const double* xy, const uint8_t* node_class, double s, double sigma_factor,
                     int bb_mode, int use_lagrange, int interp, double lag_tol, const double* box, const int* side,
                     const double* disks, int ndisks, int* kind, double* M, int* lag_slot,
                     double* lag_h, int* lag_center, int* link, double* q, double* W, int* src,
                     int* status) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        const double* o = off + 2 * K * t;
        status[t] = 0;
        memset(M + 6 * K * t, 0, sizeof(double) * 6 * K);
        memset(W + 9 * K * t, 0, sizeof(double) * 9 * K);
        for (int a = 0; a < 9; ++a) { lag_slot[9 * t + a] = -1; link[9 * t + a] = 0; q[9 * t + a] = 0; src[9 * t + a] = a; }
        lag_h[t] = 0;
        lag_center[t] = 0;
        if (node_class[i] == 2) { kind[t] = 2; continue; }
        int self_slot = -1;
        for (int j = 0; j < K; ++j) if (idx[t * K + j] == i) { self_slot = j; break; }
        int st = oracle_bc_links(xy[2 * i], xy[2 * i + 1], s, box, side, disks, ndisks,
                                 link + 9 * t, q + 9 * t);
        if (st) { status[t] = st; kind[t] = 0; continue; }
        kind[t] = 0;
        double dx[9], dy[9];
        int use[9];
        odepartures(s, link + 9 * t, q + 9 * t, bb_mode, dx, dy, use);
        if (use_lagrange && oracle_lagrange_detect(o, K, lag_tol, dx, dy, use, lag_slot + 9 * t, lag_h + t,
                                                   lag_center + t))
            kind[t] = 1;
        else {
            st = oracle_wls_matrix(o, K, s, sigma_factor, M + 6 * K * t);
            if (st) { status[t] = st; continue; }
        }
        oracle_direction_weights(K, kind[t], M + 6 * K * t, lag_slot + 9 * t, lag_h[t], lag_center[t], s,
                                 self_slot, link + 9 * t, q + 9 * t, bb_mode, W + 9 * K * t, src + 9 * t);
        if (interp == 1 && kind[t] == 0) {
            /* RBF-FD rows replace the least-squares rows at the same points */
            for (int k = 1; k < 9; ++k) {
                if (!use[k]) continue;
                st = oracle_rbf_weights(o, K, dx[k], dy[k], W + (9 * t + k) * K);
                if (st) { status[t] = st; break; }
            }
        }
    }
}

/* ----------------------------------- RBF-FD per Lagrangian point --- */
/*
 * The paper's RBF-FD stencils (Sec. 2.2): every Lagrangian (departure) point
 * is interpolated from its own N_L nearest nodes (the paper uses N_L = 25).
 * This rewrites the rows that oracle_assemble gave the least-squares-class
 * nodes (kind 0): for every direction k = 1..8 that interpolates (all but
 * simple bounce-back links; the departure rule of oracle_assemble, so an
 * interpolated link uses its reflected point), the n_l nearest nodes of the
 * departure point x_i + d_k -- squared distance from that point, offsets by
 * the periodic minimum image from x_i, ties to the lower node id, brute
 * force -- carry the cubic-PHS + quadratic weights of oracle_rbf_weights
 * there.  The node's stencil becomes the union of the node itself and its
 * directions' stencils in increasing node id, padded to kmax slots with the
 * node itself at zero weight; every other node keeps its own K-node stencil
 * in the first K slots, padded the same way, with its rows copied.
 * idx_out [nt][kmax], w_out [nt][9][kmax] (row 0 zero).  status[t]: 3 when
 * the union has more than kmax members, 2 on a singular system.
 */
void oracle_rbf_lagrangian(int64_t nt, const int64_t* targets, const double* xy, int64_t n, const double* box,
                           int periodic_x, int periodic_y, double s, int n_l, int K, const int64_t* idx,
                           const int* kind, const int* link, const double* q, int bb_mode, const double* w_in,
                           int kmax, int64_t* idx_out, double* w_out, int* status) {
    const double Lx = box[2] - box[0], Ly = box[3] - box[1];
#pragma omp parallel
    {
    double* bd = (double*)malloc(sizeof(double) * n_l);
    int64_t* bi = (int64_t*)malloc(sizeof(int64_t) * n_l);
    double* bo = (double*)malloc(sizeof(double) * 2 * n_l);
    int64_t* uni = (int64_t*)malloc(sizeof(int64_t) * (8 * n_l + 1));
    int64_t* memb = (int64_t*)malloc(sizeof(int64_t) * 8 * n_l);
    double* wk = (double*)malloc(sizeof(double) * 8 * n_l);
#pragma omp for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        const int64_t i = targets ? targets[t] : t;
        for (int j = 0; j < kmax; ++j) idx_out[t * kmax + j] = i;
        for (int j = 0; j < 9 * kmax; ++j) w_out[t * 9 * kmax + j] = 0.0;
        if (kind[t] != 0) {
            if (K > kmax) { status[t] = 3; continue; }
            for (int j = 0; j < K; ++j) idx_out[t * kmax + j] = idx[t * K + j];
            for (int k = 0; k < 9; ++k)
                for (int j = 0; j < K; ++j) w_out[(t * 9 + k) * kmax + j] = w_in[(t * 9 + k) * K + j];
            continue;
        }
        double dx[9], dy[9];
        int use[9];
        odepartures(s, link + 9 * t, q + 9 * t, bb_mode, dx, dy, use);
        const double xi = xy[2 * i], yi = xy[2 * i + 1];
        int nu = 0;
        uni[nu++] = i;
        for (int k = 1; k < 9; ++k) {
            if (!use[k]) continue;
            int cnt = 0;
            for (int64_t j = 0; j < n; ++j) {
                const double ox = omin_image(xy[2 * j] - xi, Lx, periodic_x);
                const double oy = omin_image(xy[2 * j + 1] - yi, Ly, periodic_y);
                const double ex = ox - dx[k], ey = oy - dy[k];
                const double d2 = ex * ex + ey * ey;
                if (cnt == n_l) {
                    if (d2 > bd[n_l - 1] || (d2 == bd[n_l - 1] && j > bi[n_l - 1])) continue;
                    cnt--;
                }
                int pos = cnt;
                while (pos > 0 && (bd[pos - 1] > d2 || (bd[pos - 1] == d2 && bi[pos - 1] > j))) {
                    bd[pos] = bd[pos - 1];
                    bi[pos] = bi[pos - 1];
                    bo[2 * pos] = bo[2 * pos - 2];
                    bo[2 * pos + 1] = bo[2 * pos - 1];
                    pos--;
                }
                bd[pos] = d2;
                bi[pos] = j;
                bo[2 * pos] = ox;
                bo[2 * pos + 1] = oy;
                cnt++;
            }
            const int st = oracle_rbf_weights(bo, n_l, dx[k], dy[k], wk + (k - 1) * n_l);
            if (st) { status[t] = st; break; }
            for (int m = 0; m < n_l; ++m) {
                memb[(k - 1) * n_l + m] = bi[m];
                int seen = 0;
                for (int u = 0; u < nu; ++u) if (uni[u] == bi[m]) { seen = 1; break; }
                if (!seen) uni[nu++] = bi[m];
            }
        }
        if (status[t]) continue;
        if (nu > kmax) { status[t] = 3; continue; }
        /* union in increasing node id */
        for (int a = 1; a < nu; ++a) {
            const int64_t v = uni[a];
            int b = a;
            while (b > 0 && uni[b - 1] > v) { uni[b] = uni[b - 1]; b--; }
            uni[b] = v;
        }
        for (int u = 0; u < nu; ++u) idx_out[t * kmax + u] = uni[u];
        for (int k = 0; k < 9; ++k) {
            if (k == 0 || !use[k]) {
                /* the rest population and simple bounce-back: the rows of
                   oracle_assemble (one-hot on the node), moved to its slot */
                for (int j = 0; j < K; ++j) {
                    const double wv = w_in[(t * 9 + k) * K + j];
                    if (wv == 0.0) continue;
                    for (int u = 0; u < nu; ++u)
                        if (uni[u] == idx[t * K + j]) { w_out[(t * 9 + k) * kmax + u] += wv; break; }
                }
                continue;
            }
            for (int m = 0; m < n_l; ++m)
                for (int u = 0; u < nu; ++u)
                    if (uni[u] == memb[(k - 1) * n_l + m]) { w_out[(t * 9 + k) * kmax + u] = wk[(k - 1) * n_l + m]; break; }
        }
    }
    free(bd); free(bi); free(bo); free(uni); free(memb); free(wk);
    }
}
