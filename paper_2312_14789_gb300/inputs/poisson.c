/*
 * Seeded variable-radius Poisson-disk point sampler (Bridson-style growth from
 * an active list, with a cell grid for neighbour queries).
 *
 * This file is part of the synthetic-input generator: it places nodes in a 2D
 * box, keeps them out of solid disks and away from pre-placed boundary nodes,
 * and knows nothing about lattice Boltzmann.  Both the CUDA path and the FP64
 * oracle read the same generated node sets; neither links this code.
 *
 * Radius field: r(x, y) is bilinear over an (nrx x nry) grid spanning the box.
 * A candidate p is accepted when |p - q| >= r(p) for every placed point q
 * (minimum-image distance across periodic sides), it lies inside the box, and
 * it is at least clear_frac * r(p) outside every disk (periodic images too).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s; } rng_t;

static uint64_t splitmix64(rng_t* r) {
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double urand(rng_t* r) { return (double)(splitmix64(r) >> 11) * (1.0 / 9007199254740992.0); }

typedef struct {
    double x0, y0, x1, y1, lx, ly;
    int px, py;
    const double* rgrid; int nrx, nry;
    const double* disks; int ndisks; double clear_frac;
    /* coarse bucket grid over disks: dcell_start[c]..dcell_start[c+1] index dcell_list */
    double dcellx, dcelly; int dncx, dncy; int* dcell_start; int* dcell_list;
    double cell, cellx, celly; int ncx, ncy;
    int64_t* head; int64_t* next;
    double* pts; int64_t npts, cap;
    double rmax;
} pd_t;

static double radius_at(const pd_t* p, double x, double y) {
    double fx = (x - p->x0) / p->lx * (p->nrx - 1);
    double fy = (y - p->y0) / p->ly * (p->nry - 1);
    if (fx < 0) fx = 0; if (fy < 0) fy = 0;
    if (fx > p->nrx - 1) fx = p->nrx - 1; if (fy > p->nry - 1) fy = p->nry - 1;
    int ix = (int)fx, iy = (int)fy;
    if (ix >= p->nrx - 1) ix = p->nrx - 2; if (iy >= p->nry - 1) iy = p->nry - 2;
    if (ix < 0) ix = 0; if (iy < 0) iy = 0;
    double tx = fx - ix, ty = fy - iy;
    const double* g = p->rgrid;
    double a = g[iy * p->nrx + ix], b = g[iy * p->nrx + ix + 1];
    double c = g[(iy + 1) * p->nrx + ix], d = g[(iy + 1) * p->nrx + ix + 1];
    return (1 - ty) * ((1 - tx) * a + tx * b) + ty * ((1 - tx) * c + tx * d);
}

static double wrapd(double d, double L, int per) {
    if (!per) return d;
    if (d >= 0.5 * L) d -= L;
    if (d < -0.5 * L) d += L;
    return d;
}

static int cell_of(const pd_t* p, double x, double y, int* cx, int* cy) {
    int ix = (int)floor((x - p->x0) / p->cellx), iy = (int)floor((y - p->y0) / p->celly);
    if (ix < 0) ix = 0; if (iy < 0) iy = 0;
    if (ix >= p->ncx) ix = p->ncx - 1; if (iy >= p->ncy) iy = p->ncy - 1;
    *cx = ix; *cy = iy;
    return iy * p->ncx + ix;
}

static int add_point(pd_t* p, double x, double y) {
    if (p->npts >= p->cap) return 0;
    int cx, cy;
    int c = cell_of(p, x, y, &cx, &cy);
    p->pts[2 * p->npts] = x; p->pts[2 * p->npts + 1] = y;
    p->next[p->npts] = p->head[c];
    p->head[c] = p->npts;
    p->npts++;
    return 1;
}

/* distance test against all placed points within radius r */
static int far_from_points(const pd_t* p, double x, double y, double r) {
    int cx, cy;
    cell_of(p, x, y, &cx, &cy);
    int reachx = (int)ceil(r / p->cellx) + 1, reachy = (int)ceil(r / p->celly) + 1;
    double r2 = r * r;
    for (int dy = -reachy; dy <= reachy; ++dy) {
        int yy = cy + dy;
        if (p->py) { yy %= p->ncy; if (yy < 0) yy += p->ncy; }
        else if (yy < 0 || yy >= p->ncy) continue;
        for (int dx = -reachx; dx <= reachx; ++dx) {
            int xx = cx + dx;
            if (p->px) { xx %= p->ncx; if (xx < 0) xx += p->ncx; }
            else if (xx < 0 || xx >= p->ncx) continue;
            for (int64_t q = p->head[yy * p->ncx + xx]; q >= 0; q = p->next[q]) {
                double ddx = wrapd(p->pts[2 * q] - x, p->lx, p->px);
                double ddy = wrapd(p->pts[2 * q + 1] - y, p->ly, p->py);
                if (ddx * ddx + ddy * ddy < r2) return 0;
            }
        }
    }
    return 1;
}

static int outside_disks(const pd_t* p, double x, double y, double clear) {
    if (p->ndisks == 0) return 1;
    int ix = (int)floor((x - p->x0) / p->dcellx), iy = (int)floor((y - p->y0) / p->dcelly);
    if (ix < 0) ix = 0; if (iy < 0) iy = 0;
    if (ix >= p->dncx) ix = p->dncx - 1; if (iy >= p->dncy) iy = p->dncy - 1;
    int c = iy * p->dncx + ix;
    for (int e = p->dcell_start[c]; e < p->dcell_start[c + 1]; ++e) {
        const double* d = p->disks + 3 * p->dcell_list[e];
        double ddx = wrapd(x - d[0], p->lx, p->px);
        double ddy = wrapd(y - d[1], p->ly, p->py);
        double rr = d[2] + clear;
        if (ddx * ddx + ddy * ddy < rr * rr) return 0;
    }
    return 1;
}

static int valid(const pd_t* p, double x, double y) {
    if (x < p->x0 || x >= p->x1 || y < p->y0 || y >= p->y1) return 0;
    double r = radius_at(p, x, y);
    if (!outside_disks(p, x, y, p->clear_frac * r)) return 0;
    return far_from_points(p, x, y, r);
}

/*
 * Returns the total number of points written to out_xy (fixed points first,
 * unchanged, then the sampled ones), or -1 when max_out is too small.
 */
int64_t pd_sample(double x0, double y0, double x1, double y1, int periodic_x, int periodic_y,
                  const double* rgrid, int nrx, int nry,
                  const double* disks, int ndisks, double clear_frac,
                  const double* fixed_xy, int64_t n_fixed,
                  uint64_t seed, int k_tries, double* out_xy, int64_t max_out) {
    pd_t p;
    memset(&p, 0, sizeof(p));
    p.x0 = x0; p.y0 = y0; p.x1 = x1; p.y1 = y1; p.lx = x1 - x0; p.ly = y1 - y0;
    p.px = periodic_x; p.py = periodic_y;
    p.rgrid = rgrid; p.nrx = nrx; p.nry = nry;
    p.disks = disks; p.ndisks = ndisks; p.clear_frac = clear_frac;
    double rmin = 1e300, rmax = 0;
    for (int i = 0; i < nrx * nry; ++i) { if (rgrid[i] < rmin) rmin = rgrid[i]; if (rgrid[i] > rmax) rmax = rgrid[i]; }
    p.rmax = rmax;
    /* disk buckets: a disk is listed in every cell its (radius + 2 rmax)
       neighbourhood touches, with periodic images folded in */
    {
        double dmax = 0;
        for (int i = 0; i < ndisks; ++i) if (disks[3 * i + 2] > dmax) dmax = disks[3 * i + 2];
        /* cells at least dmin wide that tile each side exactly, so periodic
           wrapping by cell index matches the geometry */
        double dmin = dmax + 2 * rmax + 1e-9;
        p.dncx = (int)floor(p.lx / dmin); p.dncy = (int)floor(p.ly / dmin);
        if (p.dncx < 1) p.dncx = 1; if (p.dncy < 1) p.dncy = 1;
        p.dcellx = p.lx / p.dncx; p.dcelly = p.ly / p.dncy;
        int nc = p.dncx * p.dncy;
        p.dcell_start = (int*)calloc(nc + 1, sizeof(int));
        int* cnt = (int*)calloc(nc, sizeof(int));
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1) {
                int acc = 0;
                for (int c = 0; c < nc; ++c) { p.dcell_start[c] = acc; acc += cnt[c]; cnt[c] = 0; }
                p.dcell_start[nc] = acc;
                p.dcell_list = (int*)malloc(sizeof(int) * (acc > 0 ? acc : 1));
            }
            for (int i = 0; i < ndisks; ++i) {
                double cx = disks[3 * i], cy = disks[3 * i + 1], reach = disks[3 * i + 2] + 2 * rmax;
                int ax = (int)floor((cx - reach - x0) / p.dcellx), bx = (int)floor((cx + reach - x0) / p.dcellx);
                int ay = (int)floor((cy - reach - y0) / p.dcelly), by = (int)floor((cy + reach - y0) / p.dcelly);
                for (int yy = ay; yy <= by; ++yy) {
                    int wy = yy;
                    if (p.py) { wy %= p.dncy; if (wy < 0) wy += p.dncy; }
                    else if (wy < 0 || wy >= p.dncy) continue;
                    for (int xx = ax; xx <= bx; ++xx) {
                        int wx = xx;
                        if (p.px) { wx %= p.dncx; if (wx < 0) wx += p.dncx; }
                        else if (wx < 0 || wx >= p.dncx) continue;
                        int c = wy * p.dncx + wx;
                        /* skip duplicates when a small grid wraps onto itself */
                        int dup = 0;
                        if (pass == 1)
                            for (int e = p.dcell_start[c]; e < p.dcell_start[c] + cnt[c]; ++e)
                                if (p.dcell_list[e] == i) { dup = 1; break; }
                        if (pass == 0) { cnt[c]++; }
                        else if (!dup) { p.dcell_list[p.dcell_start[c] + cnt[c]++] = i; }
                    }
                }
            }
        }
        /* compact: pass 0 may have over-counted duplicates; fix starts */
        {
            int acc = 0;
            int* newlist = (int*)malloc(sizeof(int) * (p.dcell_start[nc] > 0 ? p.dcell_start[nc] : 1));
            int* newstart = (int*)calloc(nc + 1, sizeof(int));
            for (int c = 0; c < nc; ++c) {
                newstart[c] = acc;
                for (int e = 0; e < cnt[c]; ++e) newlist[acc++] = p.dcell_list[p.dcell_start[c] + e];
            }
            newstart[nc] = acc;
            free(p.dcell_list); free(p.dcell_start);
            p.dcell_list = newlist; p.dcell_start = newstart;
        }
        free(cnt);
    }
    p.cell = rmin / sqrt(2.0);
    p.ncx = (int)ceil(p.lx / p.cell); p.ncy = (int)ceil(p.ly / p.cell);
    if (p.ncx < 1) p.ncx = 1; if (p.ncy < 1) p.ncy = 1;
    p.cellx = p.lx / p.ncx; p.celly = p.ly / p.ncy;
    int64_t ncell = (int64_t)p.ncx * p.ncy;
    p.head = (int64_t*)malloc(sizeof(int64_t) * ncell);
    p.next = (int64_t*)malloc(sizeof(int64_t) * max_out);
    int64_t* active = (int64_t*)malloc(sizeof(int64_t) * max_out);
    if (!p.head || !p.next || !active) { free(p.head); free(p.next); free(active); return -1; }
    for (int64_t i = 0; i < ncell; ++i) p.head[i] = -1;
    p.pts = out_xy; p.cap = max_out;
    rng_t rng = { seed * 0x2545F4914F6CDD1Dull + 0x1234567ull };
    int64_t nact = 0;
    for (int64_t i = 0; i < n_fixed; ++i) {
        if (!add_point(&p, fixed_xy[2 * i], fixed_xy[2 * i + 1])) goto full;
        active[nact++] = p.npts - 1;
    }
    for (int restart = 0; restart < 64; ++restart) {
        if (nact == 0) {
            /* dart-throw a new seed point; stop when none fits */
            int found = 0;
            for (int t = 0; t < 20000 && !found; ++t) {
                double x = x0 + urand(&rng) * p.lx, y = y0 + urand(&rng) * p.ly;
                if (valid(&p, x, y)) {
                    if (!add_point(&p, x, y)) goto full;
                    active[nact++] = p.npts - 1;
                    found = 1;
                }
            }
            if (!found) break;
        }
        while (nact > 0) {
            int64_t ai = (int64_t)(urand(&rng) * nact);
            if (ai >= nact) ai = nact - 1;
            int64_t a = active[ai];
            double ax = p.pts[2 * a], ay = p.pts[2 * a + 1];
            double ra = radius_at(&p, ax, ay);
            int placed = 0;
            for (int t = 0; t < k_tries; ++t) {
                double ang = 2.0 * M_PI * urand(&rng);
                double rad = ra * (1.0 + urand(&rng));
                double x = ax + rad * cos(ang), y = ay + rad * sin(ang);
                if (p.px) { if (x < x0) x += p.lx; if (x >= x1) x -= p.lx; }
                if (p.py) { if (y < y0) y += p.ly; if (y >= y1) y -= p.ly; }
                if (valid(&p, x, y)) {
                    if (!add_point(&p, x, y)) goto full;
                    active[nact++] = p.npts - 1;
                    placed = 1;
                    break;
                }
            }
            if (!placed) active[ai] = active[--nact];
        }
    }
    free(p.head); free(p.next); free(active); free(p.dcell_start); free(p.dcell_list);
    return p.npts;
full:
    free(p.head); free(p.next); free(active); free(p.dcell_start); free(p.dcell_list);
    return -1;
}
