/*
 * mlbm.h -- C ABI of the GB300 meshless lattice Boltzmann (MLBM) step.
 *
 * The method (Strzelczyk & Matyka, arXiv 2312.14789): D2Q9 populations live
 * on scattered ("Eulerian") nodes; each time step streams every population
 * f_k from its departure point x - s e_k (s = streaming distance, decoupled
 * from the node spacing, Sec. 2.2-2.3), obtained by interpolating the
 * post-collision field over a stencil of neighbouring nodes (Eq. (12)),
 * then collides (BGK, or TRT Eq. (3)-(5)).  The tau = 1 variant (MLBM1,
 * Eq. (14)-(15)) stores only rho and u and interpolates those.
 *
 * Conventions for every entry point:
 *  - All pointers passed in are HOST pointers owned by the caller unless the
 *    name ends in _device; data is copied on entry, results are written to
 *    caller-owned host arrays.  The library owns the device memory of a
 *    context (cudaMalloc at mlbm_init, cudaFree at mlbm_destroy).
 *  - Node arrays are in the caller's order; the library reorders nodes
 *    internally (Hilbert curve) and undoes the permutation on output.
 *  - Units: lattice units (time step 1, population speeds |e_k| in units of
 *    the streaming distance s); lengths (xy, s, disk radii) in the caller's
 *    length unit.
 *  - Errors: every call returns an mlbm_status; on failure a message is
 *    available from mlbm_last_error() (thread-local).  No call aborts the
 *    process or traps on the device.
 *  - Streams: work is issued on the context's stream (default: a stream the
 *    context creates; see mlbm_set_stream).  Calls that return host data
 *    synchronise that stream.
 */
#ifndef MLBM_H
#define MLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MLBM_OK = 0,
    MLBM_E_INVALID = 1,          /* bad argument (null pointer, size, range) */
    MLBM_E_SINGULAR_STENCIL = 2, /* least-squares normal matrix ill-conditioned (> 1e12) */
    MLBM_E_CUDA = 3,             /* a CUDA runtime call failed, or no device */
    MLBM_E_OOM = 4,              /* host or device allocation failed */
    MLBM_E_DIVERGED = 5,         /* non-finite or non-positive density found */
    MLBM_E_TIMEOUT = 6,          /* a bounded device wait gave up */
    MLBM_E_NOT_CONVERGED = 7,    /* run_to_steady reached max_steps */
    MLBM_E_GEOMETRY = 8,         /* a node lies inside a solid */
    MLBM_E_IO = 9                /* checkpoint file could not be read or written */
} mlbm_status;

/* node classes */
enum { MLBM_NODE_FLUID = 0, MLBM_NODE_WALL = 1, MLBM_NODE_EQ = 2 };
/* box side types: periodic (the opposite side must be periodic too), solid
   wall (bounce-back), open (nothing beyond; departure points outside are
   extrapolated by the fit) */
enum { MLBM_SIDE_PERIODIC = 0, MLBM_SIDE_SOLID = 1, MLBM_SIDE_OPEN = 2 };
/* bounce-back rule on links whose departure segment enters a solid */
enum { MLBM_BB_SIMPLE = 0, MLBM_BB_INTERPOLATED = 1 };
/* collision model */
enum { MLBM_MODEL_BGK = 0, MLBM_MODEL_TAU1 = 1 };
/* interpolant of the scattered (non-Lagrange) nodes: quadratic weighted least
   squares, or RBF-FD (cubic polyharmonic spline with quadratic terms, Sec. 2.2) */
enum { MLBM_INTERP_WLS = 0, MLBM_INTERP_RBF = 1, MLBM_INTERP_RBF_POINTS = 2 };
/* device node order: Hilbert curve (default), Morton (Z) curve, strips of
   about 8 node spacings left to right, or the caller's order */
enum { MLBM_ORDER_HILBERT = 0, MLBM_ORDER_MORTON = 1, MLBM_ORDER_ROWS = 2, MLBM_ORDER_INPUT = 3 };

typedef struct mlbm_stencils mlbm_stencils;
typedef struct mlbm_ctx mlbm_ctx;

/* Node set.  xy[n][2] positions; node_class[n] in MLBM_NODE_*; eq_values
   [n][3] = (rho_b, ux_b, uy_b) used only for MLBM_NODE_EQ nodes (may be NULL
   when there are none); area[n] node areas in length units^2 (NULL: 1), used
   by the area-weighted observables and the wall force. */
typedef struct {
    int64_t n;
    const double* xy;
    const uint8_t* node_class;
    const double* eq_values;
    const double* area;
} mlbm_nodes;

/* Box [x0, x1] x [y0, y1] with side types (left, right, bottom, top) and
   solid disks[n_disks][3] = (cx, cy, r).  Disks near a periodic side also
   act through their periodic images. */
typedef struct {
    double x0, y0, x1, y1;
    int side[4];
    int n_disks;
    const double* disks;
} mlbm_geometry;

/* ---------------------------------------------------------------- stencils */
/*
 * Build everything the step needs for one node set and one streaming
 * distance s (Sec. 2.2; the precomputation the paper does once per node set):
 *  - K nearest nodes of every node, itself included, ordered by (squared
 *    distance, caller's node id); offsets use the minimum image across
 *    periodic sides (Sec. 3.2: periodic stencil search);
 *  - the 6 x K weighted least-squares matrix M = (P^T W P)^-1 P^T W of a
 *    quadratic fit, Gaussian weights exp(-r^2 / sigma^2) with
 *    sigma = sigma_factor * (largest stencil offset), solved in FP64
 *    (Householder QR) and stored in FP32 scaled to units of s;
 *  - when use_lagrange != 0, nodes whose stencil holds an axis-aligned 3x3
 *    block that contains all their departure points use biquadratic
 *    Lagrange interpolation instead (Sec. 2.2, regular parts of hybrid
 *    node sets);
 *  - bounce-back links: directions whose departure segment from x to
 *    x - s e_k enters a solid, with the entry fraction q; bb_mode selects
 *    simple bounce-back f_k = f_{k'}^post(x) (Sec. 3.1) or interpolated
 *    bounce-back at x + (1 - 2q) s e_k (Eq. (22) when q = 0);
 *  - a Hilbert-curve node order.
 * K: 6..32 and a multiple of 4 (9..32 with use_lagrange); s > 0;
 * sigma_factor > 0.  Host-only work (no GPU needed).  *out is owned by the
 * caller and released with mlbm_stencils_free.
 * Errors: MLBM_E_INVALID, MLBM_E_SINGULAR_STENCIL, MLBM_E_GEOMETRY, MLBM_E_OOM.
 */
mlbm_status mlbm_build_stencils(const mlbm_nodes* nodes, const mlbm_geometry* geo, int K, double s,
                                double sigma_factor, int bb_mode, int use_lagrange, mlbm_stencils** out);

/*
 * mlbm_build_stencils with a choice of interpolant for the scattered nodes.
 * MLBM_INTERP_RBF is the paper's RBF-FD (Sec. 2.2): the cubic polyharmonic
 * spline r^3 augmented with the six quadratic monomials, over the node's own
 * K-node stencil (the paper notes that for small streaming distances the
 * Eulerian node's stencil decides the interpolation).  For every direction
 * the weights of the value at its departure point (or at the reflected point
 * of an interpolated bounce-back link) solve the (K+6)-square saddle-point
 * system in FP64 (LU, partial pivoting); they are stored per direction, 8 K
 * FP32 weights per node.  Lagrange blocks and simple bounce-back are as for
 * the least-squares fit.  Both collision models use them (the tau = 1 model
 * interpolates rho and u with the same per-direction weights).  Errors: as
 * mlbm_build_stencils; a singular RBF-FD system gives
 * MLBM_E_SINGULAR_STENCIL.
 */
mlbm_status mlbm_build_stencils_ex(const mlbm_nodes* nodes, const mlbm_geometry* geo, int K, double s,
                                   double sigma_factor, int bb_mode, int use_lagrange, int interp,
                                   mlbm_stencils** out);

/*
 * The paper's RBF-FD with a stencil per Lagrangian point (Sec. 2.2: each
 * departure point is interpolated from its own N_L nearest nodes; the paper
 * uses N_L = 25).  For every interpolating direction of a scattered node,
 * the n_l nearest nodes of its departure point x - s e_k (of the reflected
 * point x + (1 - 2q) s e_k for an interpolated bounce-back link) -- squared
 * distance from that point, periodic minimum images, ties to the lower
 * node id -- carry the cubic-PHS + quadratic weights there (FP64 LU).  The
 * node's device stencil is the union of the node and its directions'
 * stencils, k_max slots wide (unused slots hold the node at zero weight),
 * with 8 rows of k_max FP32 weights.  Lagrange detection, links and the
 * node's own fit use its 16 nearest nodes, as mlbm_build_stencils with
 * K = 16.  n_l in [7, 32] (<= n), k_max a multiple of 4 in [16, 64].
 * Errors: as mlbm_build_stencils; MLBM_E_INVALID (naming the node) when a
 * union holds more than k_max nodes.  The scattered nodes of such stencils
 * run the RBF-FD step kernels (K = k_max); K > 32 runs variants 0-3 only.
 */
mlbm_status mlbm_build_stencils_points(const mlbm_nodes* nodes, const mlbm_geometry* geo, int n_l, int k_max,
                                       double s, int bb_mode, int use_lagrange, mlbm_stencils** out);

void mlbm_stencils_free(mlbm_stencils* st);

typedef struct {
    int64_t n;            /* nodes */
    int K;
    double s;
    int64_t n_wls;        /* nodes interpolated by the least-squares fit */
    int64_t n_lagrange;   /* nodes interpolated by biquadratic Lagrange */
    int64_t n_eq;         /* equilibrium-overwrite nodes */
    int64_t n_link_nodes; /* nodes with at least one bounce-back link */
    int64_t n_links;      /* bounce-back links */
    double build_seconds; /* host time spent in mlbm_build_stencils */
} mlbm_stencil_info;

mlbm_status mlbm_stencils_info(const mlbm_stencils* st, mlbm_stencil_info* info);

/*
 * Re-order the nodes of built stencils (the order the device arrays, and so
 * the neighbour gathers, follow): MLBM_ORDER_*.  Host-only; contexts made
 * afterwards use the new order (results in the caller's order are the same
 * up to FP32 summation order).  The paper has no counterpart (its nodes are
 * visited in input order by one CPU thread).  Errors: MLBM_E_INVALID.
 */
mlbm_status mlbm_stencils_set_order(mlbm_stencils* st, int order);
int mlbm_stencils_order(const mlbm_stencils* st);

/*
 * Copy the stencil data out in the caller's node order (for inspection and
 * tests; any pointer may be NULL to skip that array):
 *   idx[n][K]     neighbour node ids (caller's ids), search order
 *   M[n][6][K]    FP64 least-squares matrix in units of s (zero for other kinds)
 *   kind[n]       0 least squares, 1 Lagrange, 2 equilibrium node
 *   link_mask[n]  bit k set when direction k (1..8) is a bounce-back link
 *   q[n][9]       entry fractions of the links (0 elsewhere)
 *   lag_h[n]      Lagrange block spacing h (0 for other kinds)
 *   lag_center[n] block centre as a D2Q9 direction index m (c = x + h e_m)
 */
mlbm_status mlbm_stencils_export(const mlbm_stencils* st, int64_t* idx, double* M, int32_t* kind,
                                 int32_t* link_mask, double* q, double* lag_h, int32_t* lag_center);
/* RBF-FD stencils: W[n][9][K] (caller's order; columns in the stencil's
   search order, as idx of mlbm_stencils_export; row 0 and the rows of
   directions that do not interpolate are zero).  Errors: MLBM_E_INVALID. */
mlbm_status mlbm_stencils_export_weights(const mlbm_stencils* st, double* W);

/* ----------------------------------------------------------------- context */
typedef struct {
    int model;        /* MLBM_MODEL_BGK or MLBM_MODEL_TAU1 */
    double tau;       /* tau+ (viscosity nu = (tau - 1/2)/3, Eq. (6)); must be 1 for TAU1 */
    double tau_minus; /* TRT tau-; <= 0 means tau_minus = tau (BGK) */
    double gx, gy;    /* body acceleration (lattice units), second-order source */
} mlbm_params;

/*
 * Create a context on the current CUDA device: uploads the stencils, allocates
 * two state buffers and sets the state at t = 0 to the equilibrium of
 * (rho0, u0) (rho0 NULL: 1; u0 NULL: 0; u0 is [n][2]).  For MLBM_MODEL_BGK the
 * state is the post-collision populations f_k^post (FP32, stored minus the
 * weights omega_k); for MLBM_MODEL_TAU1 it is (rho, ux, uy).
 * Errors: MLBM_E_INVALID, MLBM_E_CUDA, MLBM_E_OOM.
 */
mlbm_status mlbm_init(mlbm_ctx** out, const mlbm_stencils* st, const mlbm_params* p, const double* rho0,
                      const double* u0);

void mlbm_destroy(mlbm_ctx* ctx);

/* Use a caller-owned cudaStream_t (NULL: the context's own stream). */
mlbm_status mlbm_set_stream(mlbm_ctx* ctx, void* stream);

/* Replace the state: BGK f[n][9] post-collision populations; TAU1 rho_u[n][3]. */
mlbm_status mlbm_set_populations(mlbm_ctx* ctx, const double* f);
mlbm_status mlbm_set_fields(mlbm_ctx* ctx, const double* rho_u);
/* Read the state back (BGK: f[n][9]; TAU1: rho_u[n][3]). */
mlbm_status mlbm_get_populations(mlbm_ctx* ctx, double* f);
mlbm_status mlbm_get_fields(mlbm_ctx* ctx, double* rho_u);

/*
 * Advance n_steps time steps (one fused kernel launch per step: gather,
 * interpolate to the departure points, bounce-back, moments, collision,
 * write the other buffer).  Asynchronous on the context's stream.
 */
mlbm_status mlbm_step(mlbm_ctx* ctx, int64_t n_steps);

/* Steps taken since mlbm_init (or the last state replacement / load). */
int64_t mlbm_step_count(const mlbm_ctx* ctx);

/*
 * Force of the fluid on the walls by integrating the fluid stress along the
 * given wall nodes (an alternative to the momentum exchange of mlbm_drag_lift;
 * the paper does not say how it evaluates the force of Sec. 3.1).  For each
 * listed node i (caller's order id nodes[i], a least-squares node on a wall):
 * traction sigma n_i ds_i / s with sigma = -(rho - 1)/3 I + rho nu (grad u +
 * grad u^T), nu = (tau - 1/2)/3, grad u from the node's own least-squares fit
 * (lattice units of the streaming distance s), n_i = normals[i][2] the unit
 * normal pointing out of the solid into the fluid, ds_i = ds[i] the wall
 * length the node stands for (node-spacing units).  F = sum of the tractions
 * (FP64, summed in list order) in the units of mlbm_drag_lift.  Single-sample
 * least-squares contexts only (else MLBM_E_INVALID); a listed node that is not
 * a least-squares node, or an id out of range, gives MLBM_E_INVALID.  Arrays
 * are caller-owned host memory, read during the call; m = 0 gives F = 0.
 * The context keeps a device buffer for 48 bytes per wall node, allocated on
 * the first call and grown only when a call lists more nodes than any before
 * (then MLBM_E_OOM if it cannot), so repeated calls allocate nothing.
 */
mlbm_status mlbm_wall_stress_force(mlbm_ctx* ctx, const int64_t* nodes, const double* normals, const double* ds,
                                   int64_t m, double* fx, double* fy);

/*
 * Density and velocity of the current state at every node (caller's order):
 * rho[n], u[n][2].  For BGK these are the moments the last collision used
 * (rho = sum f, rho u = sum f e - rho g / 2).  Either pointer may be NULL.
 */
mlbm_status mlbm_macroscopics(mlbm_ctx* ctx, double* rho, double* u);

/*
 * Force on all solids (momentum exchange over the bounce-back links, per unit
 * lattice area times area_x / s^2, relative to the rest state f = omega),
 * as exchanged in the next streaming step from the current state.  cd, cl = 2 F / (rho_ref u_ref^2 L_lb) with
 * L_lb = ref_length / s, rho_ref = 1.  Any output pointer may be NULL.
 */
mlbm_status mlbm_drag_lift(mlbm_ctx* ctx, double ref_length, double u_ref, double* fx, double* fy,
                           double* cd, double* cl);

/*
 * Porous-media observables (Sec. 3.2, Eq. (23), (25)) over non-equilibrium
 * nodes, FP64 area-weighted sums with a fixed summation order:
 *   u_superficial = sum(u_x A) / box area,  u_intrinsic = sum(u_x A) / sum(A),
 *   k = nu u_superficial / |g| with nu = (tau - 1/2)/3 (Darcy),
 *   tortuosity = sum(|u| A) / sum(u_x A).
 * Any output pointer may be NULL.  k is 0 when g = 0.
 */
mlbm_status mlbm_permeability(mlbm_ctx* ctx, double* k, double* u_superficial, double* u_intrinsic,
                              double* tortuosity);

/*
 * Step until the relative change of the velocity field over `window` steps,
 * ||u(t) - u(t - window)||_2 / (window ||u(t)||_2) over all nodes but the
 * equilibrium-overwrite ones, falls below tol, or max_steps is reached
 * (MLBM_E_NOT_CONVERGED).  t counts from the start of this call; the
 * criterion is evaluated every `window` steps (mlbm_run_to_steady) or every
 * `check` steps from t = window on (mlbm_run_to_steady_ex; window must be a
 * multiple of check; a ring of window / check FP32 velocity snapshots,
 * 8 bytes per node each, is allocated for the call when check < window and
 * must stay under 64 GB).  *steps_taken (may be NULL) receives the steps
 * advanced by this call.  At every evaluation (every `check` steps) the
 * fluid nodes are also checked for divergence: a density that is not
 * positive, or a non-finite density or velocity, returns MLBM_E_DIVERGED
 * (the state is left as it is for inspection).
 */
mlbm_status mlbm_run_to_steady(mlbm_ctx* ctx, double tol, int64_t window, int64_t max_steps,
                               int64_t* steps_taken);
mlbm_status mlbm_run_to_steady_ex(mlbm_ctx* ctx, double tol, int64_t window, int64_t check, int64_t max_steps,
                                  int64_t* steps_taken);

/*
 * Step until the paper's steady-state criterion holds (Sec. 3.2, porous
 * flow): with <u>(t) the superficial mean x-velocity, sum(u_x A) / box area
 * (mlbm_permeability's u_superficial; Eq. (23)), recorded every `check`
 * steps, and dn the paper's Delta n_t,
 *   Delta u(t) = |<u>(t) - <u>(t - dn)| / (|<u>(t - dn)| dt dn)
 * is evaluated every `check` steps from t = dn on (dn a multiple of check);
 * the run is steady at the first t with Delta u < threshold (the paper uses
 * threshold 1e-2, dn = 2e4).  A zero earlier mean is never steady.  dt is
 * the physical time of one step; dt = 0 selects the paper's units (sample
 * side length 1, kinematic viscosity 1): dt = nu (s / L)^2 with
 * nu = (tau - 1/2)/3 and L the side of a square of the box's area, in the
 * same length unit as s.  Divergence is checked as in mlbm_run_to_steady.
 * *steps_taken (may be NULL) receives the steps advanced by this call.
 * Single-sample contexts only (MLBM_E_INVALID otherwise; see
 * mlbm_batch_run_to_steady_mean).  Errors: MLBM_E_INVALID (threshold <= 0,
 * dn not a positive multiple of check, dt < 0), MLBM_E_DIVERGED,
 * MLBM_E_NOT_CONVERGED, MLBM_E_CUDA, MLBM_E_TIMEOUT.
 */
mlbm_status mlbm_run_to_steady_mean(mlbm_ctx* ctx, double threshold, int64_t dn, int64_t check, double dt,
                                    int64_t max_steps, int64_t* steps_taken);

/*
 * Bounded device waits.  The bulk-copy ring step variants (4..7) wait on
 * shared-memory barriers for their tile copies; each wait gives up after
 * `seconds` (default 2; accepted range [1e-4, 60]), records an error word,
 * waits (bounded again) for the copies it issued and returns, and the next
 * call that synchronises the context returns MLBM_E_TIMEOUT with the step's
 * result invalid.  The context stays usable (reload a state with
 * mlbm_set_populations / mlbm_set_fields).  No paper counterpart.
 */
mlbm_status mlbm_set_wait_limit(mlbm_ctx* ctx, double seconds);
/*
 * Test of the bounded waits: the next step launch (which must use a
 * bulk-copy ring variant, 4..7, else MLBM_E_INVALID) issues no copies for
 * the first tile of its first block, so that block's consumers wait for a
 * tile that never arrives until the wait limit runs out.  One launch only;
 * it is launched directly, never from a captured graph.  No paper counterpart.
 */
mlbm_status mlbm_test_withhold_copy(mlbm_ctx* ctx);

/* Checkpoint the state, step count and parameters to a file / restore them
   into a context built from the same stencils (node count and K checked). */
mlbm_status mlbm_save(mlbm_ctx* ctx, const char* path);
mlbm_status mlbm_load(mlbm_ctx* ctx, const char* path);

/* Average duration (ms) of the fused step kernels launched by the last
   mlbm_step call, measured with CUDA events on the context's stream when
   timing is enabled (mlbm_set_timing(ctx, 1)); -1 when not measured. */
mlbm_status mlbm_set_timing(mlbm_ctx* ctx, int enable);
double mlbm_last_step_ms(const mlbm_ctx* ctx);

/*
 * Kernel variant of the fused step (all give the same results up to FP32
 * summation order):
 *   0    one thread per node, direct loads
 *   1-3  two lanes per node (neighbour groups split, pair-shuffle reduction),
 *        1 uncapped registers, 2 / 3 capped for 3 / 4 resident blocks of 256
 *   4-7  persistent CTAs streaming the per-node matrix, indices and meta
 *        bytes through a shared-memory ring filled by bulk async copies
 *        (mbarrier pipeline), four lanes per node: 4 = 128-node tiles, 3
 *        stages; 5 = 128-node tiles, 2 stages, 2 CTAs/SM; 6 = 64-node tiles,
 *        3 stages; 7 = 64-node tiles, 2 stages
 *   8-10 persistent blocks walking node tiles that first bulk-prefetch the
 *        matrix/index/meta rows of a later tile into L2 (no shared memory):
 *        8 = two lanes per node, one round ahead; 9 = two lanes, two rounds
 *        ahead; 10 = one lane per node, one round ahead
 *   11   one lane per node, registers capped for 2 resident blocks of 256
 *   12-13 as 10 with registers capped for 2 / 3 resident blocks of 256
 *   14-17 two lanes per node split by direction half (each lane gathers the
 *        16-byte half record of its four directions): 14 = registers capped for
 *        3 resident blocks of 256, all neighbour groups unrolled; 15 = capped
 *        for 4 blocks, one group at a time; 16 = as 15, persistent with L2
 *        prefetch; 17 = capped for 4 blocks, two groups at a time (BGK only;
 *        the tau = 1 model runs variant 11 for these numbers)
 *   18-19 as 10 without the bounce-back code (fewer registers), registers
 *        capped for 2 / 3 resident blocks of 256, followed by a second kernel
 *        that recomputes every node with bounce-back links (16 lanes per node,
 *        one gather per stencil member for both the departure values and the
 *        link fits) and overwrites its output (BGK only; tau = 1 runs
 *        variant 11)
 *   20-21 as 11 (plain grid, capped for 2 blocks) and as 10 (persistent,
 *        uncapped), with the first three index rows and the rest population
 *        loaded before the node kind is read, so their latency overlaps the
 *        meta load (BGK only; tau = 1 runs variant 11).  RBF-FD stencils map
 *        10 and 12 to the persistent kernel (uncapped / capped for 2 blocks),
 *        0 to the plain uncapped kernel, 20 and 21 to the plain capped and the
 *        persistent uncapped kernel with the early loads, and the rest to the
 *        plain kernel capped for 2 blocks
 *   22   least-squares BGK with staged neighbourhoods: persistent blocks of
 *        256 threads copy the union of a 256-node tile's stencil members
 *        (32 bytes each, listed when the context is created) into shared
 *        memory with cp.async, one tile ahead of the tile they compute, and
 *        gather from there through 16-bit local indices; Lagrange and
 *        equilibrium nodes and nodes with links take the global path.
 *        Available when every tile's union has at most 1536 members (else
 *        mlbm_set_kernel_variant returns MLBM_E_INVALID and the autotuner
 *        skips it); RBF-FD stencils run the plain capped kernel and tau = 1
 *        runs variant 11 for this number
 *   23-24 other block sizes with the register budget of 12 and 11: 23 = as 12
 *        with blocks of 128 threads (128-node tiles, capped for 4 resident
 *        blocks); 24 = as 11 with blocks of 512 threads (BGK only; RBF-FD
 *        stencils run the plain capped kernel, tau = 1 runs variant 11)
 *   25-26 as 12 (persistent) and 11 (plain grid), launched with programmatic
 *        stream serialization: each step grid lets the next one be scheduled
 *        on the SM slots it frees, and the next grid prefetches its first
 *        stencil rows into L2 before it waits for the previous grid's writes
 *        (BGK and tau = 1; RBF-FD stencils run the plain capped kernel)
 *   27-29 persistent CTAs of one lane per node (the node code of 11) whose
 *        matrix, index and meta rows come from a shared-memory ring that a
 *        producer warp fills with bulk async copies, as 4-7: 27 = 128-node
 *        tiles, 2 stages, 2 CTAs/SM; 28 = 64-node tiles, 2 stages, 3 CTAs/SM;
 *        29 = 64-node tiles, 3 stages, 2 CTAs/SM (BGK and tau = 1; RBF-FD
 *        stencils run the plain capped kernel)
 * Variants 4 and up are available for K = 12, 16, 24 and 32.
 * The default is 25 when available, else 1.  mlbm_autotune times every
 * available variant for steps_per_variant steps on the context's stream
 * (state saved and restored, step count unchanged), keeps the fastest and
 * returns its per-step time in *best_ms (may be NULL).
 */
mlbm_status mlbm_set_kernel_variant(mlbm_ctx* ctx, int variant);
int mlbm_kernel_variant(const mlbm_ctx* ctx);
/* Per-step times (ms) of the last mlbm_autotune(_ex) on this context:
   ms[v] for variants v = 0 .. n-1 (-1: not timed there, or no autotune yet).
   Returns the number of variants, or -1 for a NULL context. */
int mlbm_autotune_times(const mlbm_ctx* ctx, double* ms, int n);
mlbm_status mlbm_autotune(mlbm_ctx* ctx, int steps_per_variant, double* best_ms);
/* As mlbm_autotune; with flush_l2 != 0 every timed step is preceded by a
   read of a zeroed 512 MiB temporary device buffer, so that steps are timed
   with a cold L2 that holds no dirty lines, and each step is timed on its
   own.  Returns MLBM_E_OOM if the buffer cannot be allocated. */
mlbm_status mlbm_autotune_ex(mlbm_ctx* ctx, int steps_per_variant, int flush_l2, double* best_ms);

/* ------------------------------------------------------------------ batches */
/*
 * One context over several independent samples (node sets), advanced by the
 * same fused launches: the samples' stencils are concatenated (sample i owns
 * nodes [first_i, first_i + count_i) of the context, in the caller's order of
 * that sample), each node knows its sample, and each sample has its own
 * collision parameters (tau, tau_minus, body force); the streaming distance s
 * is the one its stencils were built with.  All samples must share K, the
 * bounce-back rule and the model.  Every single-context call works on the
 * whole concatenation; the calls below give per-sample results.  Initial
 * state: rest equilibrium (rho = 1, u = 0).
 */
mlbm_status mlbm_batch_init(mlbm_ctx** out, const mlbm_stencils* const* stencils, const mlbm_params* params,
                            int n_samples);
/* number of samples (1 for a context made by mlbm_init) */
int mlbm_batch_size(const mlbm_ctx* ctx);
mlbm_status mlbm_batch_range(const mlbm_ctx* ctx, int sample, int64_t* first, int64_t* count);
/* mlbm_permeability per sample: arrays of mlbm_batch_size(ctx) entries (any may be NULL) */
mlbm_status mlbm_batch_permeability(mlbm_ctx* ctx, double* k, double* u_superficial, double* u_intrinsic,
                                    double* tortuosity);
/* mlbm_drag_lift per sample: ref_length[i], u_ref[i] inputs, outputs of
   mlbm_batch_size(ctx) entries (any may be NULL; NULL references give 0 coefficients) */
mlbm_status mlbm_batch_drag_lift(mlbm_ctx* ctx, const double* ref_length, const double* u_ref, double* fx, double* fy,
                                 double* cd, double* cl);
/* mlbm_run_to_steady with the criterion per sample; the run goes on until
   every sample has converged or max_steps is reached; steps_taken[i] is the
   step count at which sample i converged (-1: not converged).  BGK batches
   step every sample to the end.  In a tau = 1 batch a converged sample is
   held at its steady state from then on (its nodes only copy their state,
   and its criterion is no longer evaluated), so every sample ends in the
   state a single-sample run of it ends in; the batch's node kinds are the
   same after the call as before.  The same holds for
   mlbm_batch_run_to_steady_mean. */
mlbm_status mlbm_batch_run_to_steady(mlbm_ctx* ctx, double tol, int64_t window, int64_t max_steps,
                                     int64_t* steps_taken);
mlbm_status mlbm_batch_run_to_steady_ex(mlbm_ctx* ctx, double tol, int64_t window, int64_t check,
                                        int64_t max_steps, int64_t* steps_taken);
/* mlbm_run_to_steady_mean per sample (Sec. 3.2 criterion on each sample's
   own <u>); dt[i] is sample i's physical time step (NULL: the paper's units
   for every sample, as mlbm_run_to_steady_mean with dt = 0) */
mlbm_status mlbm_batch_run_to_steady_mean(mlbm_ctx* ctx, double threshold, int64_t dn, int64_t check,
                                          const double* dt, int64_t max_steps, int64_t* steps_taken);

/*
 * Autotune the node order together with the kernel variant: for every
 * MLBM_ORDER_* the stencils of all n_samples samples are re-ordered, a
 * context is made from them (mlbm_init for one sample, mlbm_batch_init
 * otherwise, with params[]), its variants are timed (mlbm_autotune_ex with
 * steps_per_variant and flush_l2) and the context is released; the stencils
 * are left in the fastest order.  best_order, best_variant and best_ms
 * (nullable) receive the winner.  Needs device memory for one context at a
 * time.  Errors: as mlbm_init / mlbm_batch_init / mlbm_autotune_ex.
 */
mlbm_status mlbm_autotune_order(mlbm_stencils* const* stencils, const mlbm_params* params, int n_samples,
                                int steps_per_variant, int flush_l2, int* best_order, int* best_variant,
                                double* best_ms);

/* mlbm_step replays chunks of 16 launches from captured CUDA graphs (one per
   starting buffer, re-captured when the variant or stream changes); enable = 0
   launches every step directly. */
mlbm_status mlbm_set_graphs(mlbm_ctx* ctx, int enable);
/* Capture and instantiate both step graphs (one per starting buffer) for the
   context's current kernel variant and stream, without running a step, so
   that a later timed mlbm_step replays graphs only.  No-op when graphs are
   off.  Errors: MLBM_E_CUDA. */
mlbm_status mlbm_prepare_graphs(mlbm_ctx* ctx);

/* ------------------------------------------------------ partitioned step */
/*
 * A node set split into n_parts contiguous ranges of its device positions
 * (the stencils' node order, Hilbert by default): partition q owns positions
 * [bounds[q], bounds[q+1]) (bounds: n_parts + 1 entries, 0 first and the
 * node count last, strictly increasing; NULL: equal counts).  The step of a
 * node reads only its stencil members' post-collision states (Sec. 2.2,
 * Eq. (12)), so each partition keeps, after its own nodes, halo slots for the
 * members it references but does not own, grouped by owning partition.
 *
 * mlbm_partition_plan (host only, no device needed) describes the split:
 * first[q], n_owned[q], n_halo[q] and halo_from[q * n_parts + o] (how many
 * of q's halo nodes partition o owns); any output may be NULL.
 * mlbm_partition_nodes lists partition `part`'s owned nodes (caller ids, in
 * its local order) and its halo nodes (caller ids, in halo-slot order); either
 * output may be NULL.  Errors: MLBM_E_INVALID (bad bounds or part).
 */
mlbm_status mlbm_partition_plan(const mlbm_stencils* st, int n_parts, const int64_t* bounds, int64_t* first,
                                int64_t* n_owned, int64_t* n_halo, int64_t* halo_from);
mlbm_status mlbm_partition_nodes(const mlbm_stencils* st, int n_parts, const int64_t* bounds, int part,
                                 int64_t* owned_ids, int64_t* halo_ids);
/*
 * The partitioned step on the current device: one context per partition (its
 * owned stencils and a state with halo slots), all on one stream.  Every
 * mlbm_part_step advances each partition once, then for every pair (owner o,
 * receiver q) packs o's new states of q's halo nodes into a buffer of o and
 * copies it into q's own halo slots (cudaMemcpyAsync), so that no step reads
 * another partition's memory; after n steps the stream is synchronised.
 * A node's arithmetic is the unpartitioned context's, in the same order, so
 * with the same kernel variant the results are bitwise equal to mlbm_init's.
 * Fields and populations are in the caller's order for all nodes (as
 * mlbm_set_fields / mlbm_get_populations); mlbm_part_permeability adds the
 * partitions' FP64 sums in partition order.  mlbm_part_info gives a
 * partition's first position, owned and halo counts and the bytes its halo
 * receives per step.  Starts at rest.  No CUDA graphs.
 * Errors: as mlbm_init, MLBM_E_INVALID for bad bounds.
 */
typedef struct mlbm_part mlbm_part;
mlbm_status mlbm_part_init(mlbm_part** out, const mlbm_stencils* st, const mlbm_params* p, int n_parts,
                           const int64_t* bounds);
void mlbm_part_destroy(mlbm_part* part);
mlbm_status mlbm_part_info(const mlbm_part* part, int q, int64_t* first, int64_t* n_owned, int64_t* n_halo,
                           int64_t* halo_bytes_per_step);
mlbm_status mlbm_part_set_kernel_variant(mlbm_part* part, int variant);
mlbm_status mlbm_part_step(mlbm_part* part, int64_t n_steps);
mlbm_status mlbm_part_set_fields(mlbm_part* part, const double* rho_u);
mlbm_status mlbm_part_get_fields(mlbm_part* part, double* rho_u);
mlbm_status mlbm_part_set_populations(mlbm_part* part, const double* f);
mlbm_status mlbm_part_get_populations(mlbm_part* part, double* f);
mlbm_status mlbm_part_permeability(mlbm_part* part, double* k, double* u_superficial, double* u_intrinsic,
                                   double* tortuosity);

/* ------------------------------------------------ device-level reductions */
/*
 * Area-weighted FP64 sums over n nodes of device arrays (FP32): rho[n],
 * ux[n], uy[n], area[n], and mask[n] (uint8, nodes with mask 0 are skipped;
 * NULL: all).  out[6] (device, FP64) receives
 *   sum A, sum rho A, sum ux A, sum uy A, sum |u| A, sum |u|^2 A.
 * Two kernels: per-block partial sums into scratch (device, FP64, at least
 * mlbm_reduce_scratch_doubles(n) entries), then one block adds the partials
 * in a fixed order, so the result is bitwise reproducible.  Asynchronous on
 * `stream` (a cudaStream_t, NULL = default stream).
 * With n = 0 the sums are all zero and rho, ux, uy, area may be NULL.
 * Errors: MLBM_E_INVALID (null pointers, n < 0, scratch too small), MLBM_E_CUDA.
 */
int64_t mlbm_reduce_scratch_doubles(int64_t n);
mlbm_status mlbm_reduce_fields_device(const float* rho, const float* ux, const float* uy, const float* area,
                                      const uint8_t* mask, int64_t n, double* scratch, int64_t scratch_len,
                                      double* out, void* stream);

/*
 * mlbm_reduce_fields_device without a scratch argument, for callers that
 * cannot allocate device memory: code that must run inside a memory budget
 * fixed up front, code embedded in another runtime that owns the device pool,
 * or latency-critical loops that cannot afford an allocation's implicit
 * synchronisation.  The paper has no counterpart; this is a library service.
 * The partial sums live in a file-scope device array of 6 * 1024 doubles
 * (48 KiB) that every GPU loading the library keeps until exit; the
 * reduction never needs more, for any n.  n must be in
 * [0, mlbm_reduce_noalloc_max_nodes()] (2^31 - 1), else MLBM_E_INVALID.
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress) and caches it for the current CUDA
 * context; make that first call before any stream capture.  A call under a
 * different context of the device (after cudaDeviceReset, or a context the
 * caller made current) looks the address up again, so it is never taken from
 * a context that is gone.  All calls share the array: calls that overlap
 * on the GPU (different streams, no ordering between them) race and give
 * wrong sums.  Nothing in it has to start at zero (each call writes every
 * partial it reads).  Calls no allocating routine.  Inputs and out[6] as for
 * mlbm_reduce_fields_device.
 */
int64_t mlbm_reduce_noalloc_max_nodes(void);
mlbm_status mlbm_reduce_fields_device_noalloc(const float* rho, const float* ux, const float* uy, const float* area,
                                              const uint8_t* mask, int64_t n, double* out, void* stream);

/* ------------------------------------------------ lattice LBM (comparison) */
/*
 * The paper's comparison method: lattice Boltzmann on a regular nx x ny grid
 * (Sec. 2.1, Eq. (1)-(3): populations move one spacing per step), with the
 * same FP32 collision as the meshless step (BGK, or TRT with tau_minus).
 * cell[ny][nx] (row-major, host): 0 fluid, 1 solid (half-way bounce-back on
 * the links that come from it), 2 equilibrium (the state is
 * f^eq(rho_b, u_b) from eq_values[ny][nx][3] every step).  Links from
 * outside a non-periodic side bounce back too.  Starts at rest (rho = 1,
 * u = 0).  Populations in mlbm_lattice_set/get_populations are FP64
 * [ny * nx][9] (unshifted).  mlbm_lattice_force is the momentum exchange on
 * the bounce-back links, relative to the rest state (as mlbm_drag_lift):
 * F = sum 2 (f*_k'(x) - w_k') e_k'.  mlbm_lattice_step is asynchronous on
 * the lattice's own stream (mlbm_lattice_sync waits); the others are
 * synchronous.  Sizes: 1 <= ny <= 65535, nx ny < 2^31.
 * Errors: MLBM_E_INVALID, MLBM_E_CUDA, MLBM_E_OOM.
 */
typedef struct mlbm_lattice mlbm_lattice;
mlbm_status mlbm_lattice_init(mlbm_lattice** out, int nx, int ny, int periodic_x, int periodic_y,
                              const uint8_t* cell, const double* eq_values, const mlbm_params* p);
void mlbm_lattice_destroy(mlbm_lattice* L);
mlbm_status mlbm_lattice_step(mlbm_lattice* L, int64_t n_steps);
mlbm_status mlbm_lattice_sync(mlbm_lattice* L);
/* n_steps steps bracketed by CUDA events on the lattice's stream; *ms = their time */
mlbm_status mlbm_lattice_time_steps(mlbm_lattice* L, int64_t n_steps, double* ms);
mlbm_status mlbm_lattice_set_populations(mlbm_lattice* L, const double* f);
mlbm_status mlbm_lattice_get_populations(mlbm_lattice* L, double* f);
mlbm_status mlbm_lattice_force(mlbm_lattice* L, double* fx, double* fy);

/* ------------------------------------------------------ learned warm start */
/*
 * The paper starts every run from rest (Sec. 3.2: body-force driven flow
 * through porous samples until steady).  The library adds an optional
 * learned initial state: a per-node multilayer perceptron
 * 16 -> 64 -> 64 -> 64 -> n_out with ReLU between layers reads 16 local
 * geometry features (mlbm_features_device) and predicts the steady velocity
 * (n_out = 2) or the steady velocity and density deviation (n_out = 3) in
 * units of per-sample scales; the solver then starts from that state instead
 * of from rest and converges to the same steady state (the prediction only
 * changes where the iteration starts).  The cold start (rest) stays the
 * default and the fallback.
 *
 * Network: y = x W + b per layer, parameters packed in FP32 in the order
 * W1[16][64], b1[64], W2[64][64], b2, W3[64][64], b3, W4[64][n_out],
 * b4[n_out] (mlbm_mlp_param_count(n_out) floats: 9538 for n_out = 2).  The
 * kernels run the layers on BF16 tensor cores with FP32 accumulation:
 * features, weights, hidden activations (after bias and ReLU) and, in the
 * backward pass, the output error and the hidden errors are rounded to BF16
 * (round to nearest even) where they enter a product; biases, accumulators,
 * gradients and the Adam state are FP32.  Loss = mean over rows of
 * |y - t|^2.
 *
 * Device arrays: X[n][16], T[n][n_out] and Y[n][n_out], FP32 row-major;
 * all calls are asynchronous on `stream` (a cudaStream_t, NULL = default
 * stream) unless they return a host value.  An mlbm_mlp owns its device
 * memory (created on the current device) and must only be used by one stream
 * at a time.  Errors: MLBM_E_INVALID (NULL pointers, n or n_out out of
 * range), MLBM_E_CUDA, MLBM_E_OOM.
 */
typedef struct mlbm_mlp mlbm_mlp;

/* parameter count for n_out outputs (1..3), -1 otherwise */
int64_t mlbm_mlp_param_count(int n_out);
/* He-normal weights (counter-based generator seeded by `seed`), zero biases;
   n_out in 1..3. */
mlbm_status mlbm_mlp_create(mlbm_mlp** out, int n_out, uint64_t seed);
void mlbm_mlp_destroy(mlbm_mlp* m);
/* n_out of the network (-1 for NULL) */
int mlbm_mlp_outputs(const mlbm_mlp* m);
/* host FP32 params[mlbm_mlp_param_count(n_out)]; set also resets the Adam state */
mlbm_status mlbm_mlp_set_params(mlbm_mlp* m, const float* params);
mlbm_status mlbm_mlp_get_params(mlbm_mlp* m, float* params);
/* Y[n][n_out] = network(X[n][16]); n >= 0. */
mlbm_status mlbm_mlp_forward_device(mlbm_mlp* m, const float* X, int64_t n, float* Y, void* stream);
/* Full-batch gradient of the loss over all n rows into grads (device,
   param_count floats, packed order; NULL: kept internally) and the loss
   (host double, NULL: not returned; returning it synchronises `stream`).
   Reproducible: per-block partial sums are added in a fixed order. */
mlbm_status mlbm_mlp_gradients_device(mlbm_mlp* m, const float* X, const float* T, int64_t n, float* grads,
                                      double* loss, void* stream);
/* `steps` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected,
   learning rate lr) on minibatches of `batch` rows drawn with replacement
   from the n rows by a counter-based hash of (seed, step, row); batch = n
   with seed = 0 takes every row once per step (full batch).  loss (host,
   nullable) receives the mean loss of the last minibatch, evaluated with
   the parameters before its update. */
mlbm_status mlbm_mlp_train_device(mlbm_mlp* m, const float* X, const float* T, int64_t n, int64_t batch,
                                  int64_t steps, float lr, uint64_t seed, double* loss, void* stream);

/*
 * Geometry features of every node, X[n][16] (device, FP32, caller's node
 * order), for the node set and geometry of mlbm_build_stencils, with length
 * scale L > 0 (the library's studies use the mean disk radius) and
 * ell = min(8 L, half the smaller box extent):
 *   0   clamp(d1 / L, 0, 4)   d1 = distance to the nearest solid surface
 *                             (disk, or periodic image of a disk, or solid side)
 *   1,2 unit vector from that surface point to the node (0 if no solid)
 *   3   clamp(d2 / L, 0, 4)   d2 = distance to the second nearest solid object
 *   4..7 free paths along +x, -x, +y, -y (distance to the first solid along
 *        the ray, at most ell) over L; a ray meets a disk where it enters
 *        it, and an entry behind the start by more than 1e-4 r (a node on
 *        the surface looking out of the solid) does not count
 *   8   clamp(f(+y) f(-y) / L^2, 0, 16), 9  clamp((f(+y) + f(-y)) / L, 0, 8)
 *   10..13 local porosity 1 - (solid area within distance rho_j of the node)
 *         / (pi rho_j^2), rho_j = min(c_j L, half the smaller box extent),
 *         c_j = 1, 2, 4, 8: disks (with their periodic images) cut by the
 *         circle in closed form (circle-circle lens), solid sides as
 *         circular segments;
 *   14  porosity of the box, 1 - sum(pi r^2) / box area
 *   15  4 (y - y0) (y1 - y) / (y1 - y0)^2 (position across the box)
 * With no solid object d1 = d2 = 4 L.  Computed on the device with the
 * positions and displacements in FP64 and the geometry in FP32 (the features
 * feed a BF16 network): within about 1e-5 of an FP64 evaluation, except that
 * the nearest of two nearly equidistant objects, or a ray grazing a disk, may
 * be decided the other way.
 * Inputs are host arrays (copied to the device inside); synchronous.
 * Errors: MLBM_E_INVALID, MLBM_E_CUDA.
 */
mlbm_status mlbm_features_device(const mlbm_nodes* nodes, const mlbm_geometry* geo, double L, float* X);

/*
 * Warm start: sets the state of ctx from the network's prediction Y =
 * network(X) for every node but the equilibrium-overwrite ones (those take
 * their boundary values): u = scale_u[s] * (Y0, Y1) and, when the network
 * has 3 outputs, rho = 1 + scale_rho[s] * Y2 minus the area-weighted mean of
 * that deviation over the sample (the sample keeps the mass of the rest
 * state); with 2 outputs rho = 1.  BGK contexts start from the equilibrium
 * of that state, as mlbm_set_fields.  X[n][16] (device, caller's node order;
 * for a batch the samples' rows one after another); scale_u[] and
 * scale_rho[] host, one per sample (scale_rho may be NULL with 2 outputs).
 * A sample whose prediction holds a non-finite value, a speed above 0.3
 * (outside the low-Mach range of the scheme) or a density deviation above
 * 0.1 starts from rest instead (the cold-start fallback); n_cold (nullable)
 * receives the number of such samples.  Resets the step count; synchronous.
 * Errors: MLBM_E_INVALID, MLBM_E_CUDA.
 */
mlbm_status mlbm_warm_start(mlbm_ctx* ctx, mlbm_mlp* m, const float* X, const double* scale_u,
                            const double* scale_rho, int* n_cold);

/* Last error message of this thread ("" when none). */
const char* mlbm_last_error(void);

/* Library version string. */
const char* mlbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MLBM_H */
