/*
 * tt.h — C ABI of the GB300 adjoint-state traveltime tomography library (libttgb.so).
 *
 * The library computes, for a batch of seismic sources on one spherical grid, the hot path
 * of Eikonal-based adjoint-state traveltime tomography (TomoATT, arXiv 2412.00031):
 *   tt_forward  factored fast-sweeping solve of the anisotropic Eikonal equation (Eq. "4"
 *               of Sec. 2.1, with T = T0 * tau, Sec. 3.1), hyperplane-parallel (Sec. 3.4)
 *   tt_misfit   receiver traveltimes, misfits chi_t and chi_cs (Eqs. 2-3) and adjoint
 *               sources R = dchi/dT (Eqs. A1-A3)
 *   tt_adjoint  upwind fast-sweeping solve of the adjoint equation (Eq. 5)
 *   tt_kernel   FP64 accumulation of the sensitivity kernels K_s, K_xi, K_eta (Eqs. 6-8)
 *   tt_misfit_cr   common-receiver differential times (Eqs. 4, A4)
 *   tt_field_at_points, tt_misfit_table, tt_reloc_kernels, tt_reloc_update
 *                  earthquake location and origin-time kernels and update (Eq. 10, B1-B11)
 *   tt_tele2d, tt_tele_region_times, tt_forward_tele
 *                  teleseismic events: 2-D times in a 1-D model, the region's face data and
 *                  the region's solve with those faces held fixed
 *   tt_kernel_density, tt_kernel_normalize, tt_mgrid_project, tt_mgrid_expand,
 *   tt_model_update   regularisation and update of the inversion step (Eqs. 11-19)
 *
 * Conventions shared by every call:
 *  - Grid: n_r x n_t x n_p nodes, uniform in radius r (index i, i = 0 is the deepest
 *    layer), latitude theta (index j) and longitude phi (index k). A scalar field is stored
 *    [n_r][n_t][n_p] with k fastest. r = earth_radius_km - depth.
 *  - Batched fields (tau, T, P) hold one value per node and source, stored node-major with
 *    the source index fastest: element (node n, source b) is at n * n_src + b. Consecutive
 *    GPU lanes then read consecutive sources of one node.
 *  - dtype TT_F32 or TT_F64 selects float or double for every model and batched field of a
 *    call. Misfit quantities, adjoint sources and kernels are always double.
 *  - Pointers named d_* are device pointers; h_* are host pointers. The caller allocates
 *    and frees every buffer it passes; the library never frees caller memory. The context
 *    owns only its workspace (schedules, tables, per-source state, barrier words).
 *  - Calls are issued on the context's CUDA stream. A call returns after its kernels are
 *    enqueued, except where noted: tt_forward and tt_adjoint wait for their iteration
 *    counts (one small device-to-host copy) to report convergence.
 *  - Errors are returned as tt_status; tt_last_error gives a one-line message. No call
 *    throws, aborts or traps. After TT_ECUDA the context should be destroyed.
 *  - One context per host thread; a context is not thread-safe.
 */
#ifndef TT_H
#define TT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TT_API_VERSION 1
#define TT_MAX_BATCH 4096 /* sources per forward/adjoint call */
#define TT_MAX_DIM 1024   /* nodes per axis */

typedef enum {
    TT_OK = 0,
    TT_EINVAL = 1,         /* invalid argument: sizes, positions, model values (see each call) */
    TT_ENOTCONVERGED = 2,  /* some source reached max_iter; outputs hold the last iterate */
    TT_ECUDA = 3,          /* a CUDA runtime call failed */
    TT_ETIMEOUT = 4,       /* a device-side wait exceeded opts.spin_limit_ns; outputs undefined */
    TT_ENOMEM = 5          /* workspace allocation failed */
} tt_status;

typedef enum { TT_F32 = 0, TT_F64 = 1 } tt_dtype;
typedef enum { TT_GEOM_SPHERICAL = 0, TT_GEOM_FLAT = 1 } tt_geometry;
/* Values of tt_opts.init (the forward's starting tau). */
typedef enum { TT_INIT_ONE = 0, TT_INIT_GIVEN = 1, TT_INIT_NET = 2, TT_INIT_ABOVE = 3 } tt_init;

/* Study region (Sec. 2.1 problem statement; Sec. 4 for the spherical parameterisation).
 * TT_GEOM_FLAT is a Cartesian test geometry: theta and phi become lengths R_E*theta and
 * R_E*phi and the metric factors r and r cos(theta) are replaced by R_E. */
typedef struct {
    int n_r, n_t, n_p;            /* nodes per axis, 4 .. TT_MAX_DIM */
    double depth_min_km, depth_max_km;
    double lat_min_deg, lat_max_deg;
    double lon_min_deg, lon_max_deg;
    double earth_radius_km;       /* 6371 for the Earth */
    int geometry;                 /* tt_geometry */
} tt_grid;

/* Model: slowness s (s/km, > 0) and azimuthal anisotropy xi, eta (Eq. "4"; the matrix M is
 * positive definite only for xi^2 + eta^2 < 1/4). Device arrays [n_r][n_t][n_p]. */
typedef struct {
    const void *d_s, *d_xi, *d_eta;
    int dtype;                    /* tt_dtype of the three arrays */
} tt_model;

typedef struct {
    double depth_km, lat_deg, lon_deg;
} tt_point;

/* Observations of a batch of n_src sources at a global list of n_rec receivers
 * (Eqs. 2-3). Absolute times: for source b, records abs_off[b] .. abs_off[b+1]-1, each a
 * receiver index, an observed time and a weight w_{n|m}. Common-source differential times:
 * for source b, unordered pairs cs_off[b] .. cs_off[b+1]-1, each (m, i, dT_obs, w) meaning
 * T(x_m) - T(x_i) observed as dT_obs with weight w; an unordered pair stands for the two
 * ordered terms of Eq. 3 with weight w/2 each. alpha and beta weight chi_t and chi_cs
 * (Eq. 1). Receiver positions are host memory; every other array is device memory. */
typedef struct {
    int n_src, n_rec;
    const tt_point *h_rec;
    const int *d_abs_off, *d_abs_rec;
    const double *d_abs_tobs, *d_abs_w;
    const int *d_cs_off, *d_cs_m, *d_cs_i;
    const double *d_cs_dtobs, *d_cs_w;
    double alpha, beta;
} tt_data;

typedef struct {
    double tol_fwd;         /* stop when the largest |tau change| of one iteration < tol_fwd */
    double tol_adj;         /* stop when the largest |P change| <= tol_adj * max |P| */
    int max_iter_fwd, max_iter_adj;
    int init;               /* tt_forward: 0 = start from tau = 1, 1 = start from the tau passed
                               in, 2 = start from the warm-start network (tt_net_set_weights),
                               3 = start from above: every node outside the fixed set starts
                               at 2 hi / lo, hi = max s / sqrt(1 - 2 g), lo = min s /
                               sqrt(1 + 2 g), g = sqrt(xi^2 + eta^2) over the model's nodes
                               (twice a straight-ray bound of tau; computed on the device).
                               The fast sweeping method's own start: the Godunov update then
                               only lowers tau, and converges in fewer iterations than from
                               tau = 1. Every start reaches the same fixed point. */
    long long spin_limit_ns;/* bound on every device-side wait; 0 = 2 s */
    int launch_blocks;      /* persistent sweep launch: 0 = automatic, else at most this many
                               blocks (results do not depend on it) */
    int sweep_schedule;     /* forward sweep schedule: 0 = automatic; 1 = node hyperplanes;
                               2, 3, 4 = tile hyperplanes with 2x4x8, 4x4x4, 2x8x8 tiles
                               (r x theta x phi). Results do not depend on it. */
    int adj_chunk;          /* adjoint: sources per launch (the slices run one after another);
                               0 = all sources in one launch. A launch runs its sources as up
                               to 4 barrier groups side by side. Results do not depend on it. */
    int fwd_groups;         /* node-hyperplane forward sweep: barrier groups per launch
                               (1..8), 0 = automatic. Results do not depend on it. */
    int fwd_slots;          /* forward sweep: 0 = every source of the call resident at once;
                               S > 0 (rounded up to a multiple of 32, below n_src) = retire and
                               refill: one launch keeps S sources in flight and a source that
                               converges (or reaches max_iter_fwd) hands its slot to the next
                               one. Results and iteration counts do not depend on it. */
    int scheme;             /* forward local solver: 0 = Lax-Friedrichs (Sec. 3.1, the paper's;
                               any model); 1 = Godunov upwind for isotropic models (xi = eta
                               = 0: tt_forward returns TT_EINVAL otherwise, after the solve);
                               2 = Godunov upwind for anisotropic models (any model: upwind
                               sides along theta and phi from the characteristic direction
                               M grad T, the Schur-complement form of M on each axis subset).
                               The Godunov solvers run on the node-hyperplane schedule. */
    int adj_groups;         /* adjoint: barrier groups per launch (1..8; each gets at least 32
                               sources), 0 = automatic (one per 64 sources, at most 4).
                               Results do not depend on it. */
    int fwd_order;          /* 0 = sweep a batch of 64 sources or more in the order of its last
                               forward iteration counts, fewest first, so that a barrier group
                               holds sources that converge together: a plan from its second
                               run on (its adjoint likewise, by the adjoint counts), a
                               tt_forward call when the context has solved the same source
                               positions before (it remembers the last 64 source sets);
                               otherwise, and with retire-and-refill, the given order. 1 =
                               always the given order. Results do not depend on it. */
} tt_opts;

typedef struct tt_ctx tt_ctx;

/* Measurements of the last persistent sweep of one kind (forward or adjoint). */
typedef struct {
    double sweep_ms;          /* device time of the sweep launch, CUDA events on the context's
                                 stream around that launch only */
    long long node_updates;   /* (node, source) updates it performed, fixed sets excluded */
    long long node_sweeps;    /* node visits counted once per batch: nodes x 8 x max iterations */
    int iters_max;            /* largest per-source iteration count */
    int grid_blocks, block_threads;
    long long launches;       /* kernels this context has launched since it was created */
    double warm_ms;           /* forward: device time of the warm-start inference (opts.init = 2),
                                 0 otherwise */
} tt_stats;

#define TT_STATS_FORWARD 0
#define TT_STATS_ADJOINT 1
#define TT_STATS_KERNEL 2   /* the last kernel accumulation (tt_kernel or a plan's): sweep_ms its
                               device time, node_updates = nodes x sources, node_sweeps = nodes */

/* Fills opts with the defaults for dtype: tol_fwd 1e-6 (F32) / 1e-8 (F64), tol_adj the
 * same, 500 iterations, init 0, spin limit 2 s. */
void tt_default_opts(tt_opts *opts, int dtype);

/* Creates a context for one grid on one CUDA stream (cudaStream_t passed as void*, NULL for
 * the default stream) of the current device. Validates the grid (TT_EINVAL) and builds the
 * hyperplane schedules and coordinate tables (TT_ENOMEM / TT_ECUDA on failure). */
tt_status tt_ctx_create(tt_ctx **out, const tt_grid *grid, void *cuda_stream);
void tt_ctx_destroy(tt_ctx *ctx);
const char *tt_last_error(const tt_ctx *ctx);

/* Forward solve (Eq. "4", Sec. 3.1) for n_src sources at h_src (host, inside the grid).
 * d_tau: device [N][n_src] of the model's dtype, the factored traveltime tau; read as the
 * starting value when opts->init = 1, always written. d_T: device [N][n_src], written with
 * T = T0 * tau (may be NULL). h_iters: host [n_src], iterations taken per source (may be
 * NULL). Each source stops on its own criterion; sweeps of converged sources are skipped.
 * TT_EINVAL: bad sizes, a source outside the grid, s <= 0 or xi^2 + eta^2 >= 1/4 somewhere.
 * Synchronises the stream once at the end. */
tt_status tt_forward(tt_ctx *ctx, const tt_model *model, const tt_point *h_src, int n_src,
                     void *d_tau, void *d_T, const tt_opts *opts, int *h_iters);

/* Misfit (Eqs. 2-3) and adjoint sources (Eqs. A2-A3) of a batch. d_T: device [N][n_src]
 * traveltimes from tt_forward, dtype as given. Outputs (device, double): d_Tr [n_src][n_rec]
 * trilinearly interpolated receiver times, d_chi [n_src][2] (chi_t, chi_cs per source),
 * d_R [n_src][n_rec] = alpha dchi_t/dT + beta dchi_cs/dT. Any output may be NULL except
 * d_R. TT_EINVAL: receiver outside the grid, index out of range. */
tt_status tt_misfit(tt_ctx *ctx, const void *d_T, int dtype, const tt_data *data,
                    double *d_Tr, double *d_chi, double *d_R);

/* Adjoint solve (Eq. 5) for the same n_src sources. d_T: the forward traveltimes; d_R:
 * device double [n_src][n_rec] adjoint sources at the receivers h_rec (host, n_rec);
 * d_P: device [N][n_src] output adjoint field (P = 0 on the 3x3x3 source set). xi and eta
 * of the model enter the flux velocity -M grad T. h_iters as in tt_forward. */
tt_status tt_adjoint(tt_ctx *ctx, const tt_model *model, const tt_point *h_src, int n_src,
                     const void *d_T, int n_rec, const tt_point *h_rec, const double *d_R,
                     void *d_P, const tt_opts *opts, int *h_iters);

/* Kernel accumulation (Eqs. 6-8): for every node adds sum_b P s^2 to d_Ks,
 * sum_b P ((d_theta T / r)^2 - (d_phi T / (r cos theta))^2) to d_Kxi and
 * sum_b -2 P (d_theta T / r)(d_phi T / (r cos theta)) to d_Keta (device double [N], read
 * and written; zero them before the first batch). Each source's term is formed in the
 * fields' precision; every 32nd source is summed by one lane with a compensated (TwoSum)
 * accumulator in that precision, the warp merges the lanes' accumulators the same way, and
 * the batch's total is added to the FP64 kernels. The sums run in a fixed order, so the
 * result is bitwise reproducible. */
tt_status tt_kernel(tt_ctx *ctx, const tt_model *model, int n_src, const void *d_T,
                    const void *d_P, double *d_Ks, double *d_Kxi, double *d_Keta);

/* ---- Common-receiver differential times (Eq. 4) and their adjoint source (Eq. A4). ---- */

/* Pairs of sources of one batch observed at a common receiver. The entries of (source b,
 * receiver m) are d_off[b * n_rec + m] .. d_off[b * n_rec + m + 1] - 1 (d_off: n_src * n_rec
 * + 1 ints, non-decreasing, n_entries = d_off[last]); entry q names the other source
 * d_other[q] (0 <= j < n_src, j != b), dT_obs = T_b^obs(x_m) - T_j^obs(x_m) as d_dtobs[q], and
 * the pair's weight d_w[q]. An unordered pair {b, j} with weight w stands for the two ordered
 * terms of Eq. 4 with weight w / 2 each and is listed twice: under (b, m) with dT_obs and
 * under (j, m) with -dT_obs. gamma weights chi_cr (Eq. 1). Device arrays. */
typedef struct {
    int n_src, n_rec, n_entries;
    const int *d_off, *d_other;
    const double *d_dtobs, *d_w;
    double gamma;
} tt_cr_data;

/* chi_cr and its adjoint source from the batch's receiver-time table d_Tr (device double
 * [n_src][n_rec], as tt_misfit writes it): d_R[b][m] += gamma dchi_cr/dT_b(x_m) (Eq. A4;
 * device double [n_src][n_rec], read and written: call after tt_misfit, before tt_adjoint),
 * d_chi_cr[b] = source b's ordered terms of Eq. 4 (device double [n_src]; they sum to
 * chi_cr). Fixed-order sums. An entry naming a source out of range is skipped and the call
 * returns TT_EINVAL (after synchronising the context's stream). */
tt_status tt_misfit_cr(tt_ctx *ctx, const tt_cr_data *d, const double *d_Tr, double *d_chi_cr,
                       double *d_R);

/* The entry table of tt_cr_data from a list of unordered pairs (Eq. 4's pairs of sources at a
 * common receiver), on the host. h_pairs: n_pairs rows (b, j, m, dT_obs, w) of doubles, the
 * pair {b, j} observed at receiver m with T_b^obs(x_m) - T_j^obs(x_m) = dT_obs and weight w.
 * Writes host arrays the caller allocates: h_off (n_src * n_rec + 1 ints) and h_other,
 * h_dtobs, h_w (2 * n_pairs each). Each pair is entered twice, under (b, m) with (j, dT_obs,
 * w) and under (j, m) with (b, -dT_obs, w); within one (source, receiver) the entries keep
 * the order of the list, first-source listings before second-source ones, so the
 * fixed-order sums of tt_misfit_cr are reproducible. b, j and m must be integral, in range
 * and b != j, else TT_EINVAL with nothing written. ctx may be NULL (it only receives the
 * error message). Touches no device memory and needs no GPU. */
tt_status tt_cr_pack(tt_ctx *ctx, int n_src, int n_rec, int n_pairs, const double *h_pairs,
                     int *h_off, int *h_other, double *h_dtobs, double *h_w);

/* ---- The inversion step's regularisation and update (Sec. 3.3; step 4 of Sec. 2). ---- */

/* Kernel density (Eq. 19): adds sum over the n_src sources of d_P[node][b] to d_Kd (device
 * double [N], read and written; zero it before the first batch). d_P: device [N][n_src] of
 * dtype, the adjoint fields computed by tt_adjoint with every adjoint source R = 1 (Eq. 19
 * defines K_d from those fields). FP64 sums in a fixed order (bitwise reproducible). */
tt_status tt_kernel_density(tt_ctx *ctx, const void *d_P, int n_src, int dtype, double *d_Kd);

/* Kernel-density normalisation (Eq. 18), in place on the three device double [N] kernels:
 * K <- K / (d_Kd + eps)^zeta. eps > 0, zeta >= 0, else TT_EINVAL. */
tt_status tt_kernel_normalize(tt_ctx *ctx, double *d_Ks, double *d_Kxi, double *d_Keta,
                              const double *d_Kd, double eps, double zeta);

/* Eq. 18 with the damping taken relative to the density: eps = eps_rel * max_n d_Kd[n]
 * (1e-300 if that maximum is 0), the maximum an FP64 reduction on the device, so the step
 * needs no host round trip. eps_rel > 0, zeta >= 0, else TT_EINVAL. */
tt_status tt_kernel_normalize_rel(tt_ctx *ctx, double *d_Ks, double *d_Kxi, double *d_Keta,
                                  const double *d_Kd, double eps_rel, double zeta);

/* Step-size control (step 4 of Sec. 2): the total misfit of a batch (Eqs. 2-4),
 * alpha sum_b d_chi[b][0] + beta sum_b d_chi[b][1] + gamma sum_b d_chi_cr[b] over n_src sources
 * (d_chi as tt_misfit writes it; d_chi_cr as tt_misfit_cr writes it, or NULL), an FP64 sum in a
 * fixed order on the device. *h_total (host) receives it; the call waits for the stream. */
tt_status tt_misfit_total(tt_ctx *ctx, int n_src, const double *d_chi, double alpha,
                          double beta, const double *d_chi_cr, double gamma, double *h_total);

/* H offset inversion grids of the multiple-grid parameterisation (Eqs. 11-14): n_grids
 * grids of n_r x n_t x n_p nodes (3..4096 per axis; 1..64 grids). Along each axis grid h has
 * its nodes at x_min + (a - h / n_grids) dc, a = 0..n-1, dc = (x_max - x_min) / (n - 2):
 * every grid covers the forward domain, offset from the next by dc / n_grids. The basis
 * function of node (a, b, c) of grid h is the product of the axes' hat functions / n_grids
 * (Eq. 11). */
typedef struct {
    int n_r, n_t, n_p;
    int n_grids;
} tt_mgrid;

/* Projection of a kernel onto the basis (Eq. 17): d_G[h][a][b][c] = sum over the forward
 * nodes of d_K B^h_abc dV, with dV = r^2 cos(theta) dr dtheta dphi the node volume (the
 * integral of Eq. 17 read as this nodal sum). d_K: device double [N]; d_G: device double
 * [n_grids][n_r][n_t][n_p]. Fixed-order sums. */
tt_status tt_mgrid_project(tt_ctx *ctx, const tt_mgrid *mg, const double *d_K, double *d_G);

/* Expansion of coefficients onto the forward grid (Eq. 15): d_D[node] = sum over grids and
 * basis functions of d_G B^h_l(node). Applied to the projected kernels it gives the smoothed
 * descent direction. d_G as above, d_D device double [N]. */
tt_status tt_mgrid_expand(tt_ctx *ctx, const tt_mgrid *mg, const double *d_G, double *d_D);

/* Model update of one gradient-descent step (step 4 of Sec. 2), in place on the model's
 * device arrays (cast from const): s <- s (1 - step d_Ds / max|d_Ds|),
 * xi <- xi - step d_Dxi / max|d_Dxi|, eta <- eta - step d_Deta / max|d_Deta|. The kernels
 * are derivatives of chi with respect to ln s, xi and eta (Eq. 9); a zero direction leaves
 * its field unchanged. step in (0, 1), else TT_EINVAL. Step-size control (halving a step
 * that raises chi) is the caller's loop. */
tt_status tt_model_update(tt_ctx *ctx, const tt_model *model, const double *d_Ds,
                          const double *d_Dxi, const double *d_Deta, double step);

/* ---- Earthquake location and origin time (Eq. 10, Appendix B, Eqs. B1-B11). ----
 * By reciprocity the time from event n to receiver m equals Gamma_m(x_n), the traveltime of
 * a wavefront started at receiver m (run tt_forward with the receivers as the sources), and
 * the arrival is Gamma_m(x_n) + tau_n with origin time tau_n. The misfits of Eqs. 2-4 and
 * their adjoint sources R = dchi/dT (Eqs. A2-A4) evaluated on those arrivals give
 *   K_x,n = sum_m R[n][m] grad Gamma_m(x_n),  K_tau,n = sum_m R[n][m]   (Eqs. B5-B11). */

/* Values and gradients at points of M batched fields. d_G: device [N][M] of dtype (the
 * layout tt_forward writes, field index fastest). d_pts: device double [n_pts][3] (depth km,
 * latitude deg, longitude deg). Outputs (device double): d_val [n_pts][M], the trilinear
 * interpolant in index space (as for receiver times); d_grad [n_pts][M][3], its gradient
 * in physical components (d/dr, d/(r dtheta), d/(r cos(theta) dphi)) at the point. So
 * K_x is the exact derivative of the discrete misfit with respect to the position.
 * TT_EINVAL for a point outside the grid (after synchronising the stream; that row is
 * computed from the nearest cell and holds no meaning). */
tt_status tt_field_at_points(tt_ctx *ctx, const void *d_G, int dtype, int n_fields, int n_pts,
                             const double *d_pts, double *d_val, double *d_grad);

/* Misfit (Eqs. 2-3) and adjoint sources (Eqs. A2-A3) from given arrivals rather than
 * fields: Tr[n][m] = d_val[n][m] + d_otime[n] (d_otime device double [n_src] or NULL = 0).
 * data as for tt_misfit (its h_rec is not read and may be NULL); outputs as tt_misfit:
 * d_Tr (may be NULL), d_chi [n_src][2] (may be NULL), d_R [n_src][n_rec]. For the
 * common-receiver terms pass d_Tr on to tt_misfit_cr, which adds into d_R.
 * TT_EINVAL: a record naming a receiver out of range (after synchronising the stream). */
tt_status tt_misfit_table(tt_ctx *ctx, const double *d_val, const double *d_otime,
                          const tt_data *data, double *d_Tr, double *d_chi, double *d_R);

/* The location and origin-time kernels: d_Kx [n_src][3] = sum_m d_R[n][m] d_grad[n][m]
 * (physical components, as d_grad) and d_Ktau [n_src] = sum_m d_R[n][m]. Device doubles;
 * d_R and d_grad as written by tt_misfit_table (+ tt_misfit_cr) and tt_field_at_points with
 * the events as the points. Fixed-order sums (bitwise reproducible). */
tt_status tt_reloc_kernels(tt_ctx *ctx, int n_src, int n_rec, const double *d_R,
                           const double *d_grad, double *d_Kx, double *d_Ktau);

/* One gradient-descent step of the events, in place (the paper names gradient descent and
 * gives no step rule; this is the normalised step also used for the model): each event moves
 * by -step_km d_Kx[n] / max_n |d_Kx[n]| km in physical components and is then clamped to
 * the grid; d_otime[n] (may be NULL) moves by -step_s d_Ktau[n] / max_n |d_Ktau[n]|. A zero
 * maximum moves nothing. d_pts as for tt_field_at_points. step_km, step_s >= 0 and finite,
 * else TT_EINVAL. Step-size control is the caller's loop. */
tt_status tt_reloc_update(tt_ctx *ctx, int n_src, double *d_pts, double *d_otime,
                          const double *d_Kx, const double *d_Ktau, double step_km,
                          double step_s);

/* ---- Teleseismic events (the boundary condition of Eq. "4" for an event outside the
 * region): the times on the region's faces come from 2-D eikonal solves in a 1-D model. ---- */

/* 2-D traveltimes of n_ev events in a 1-D model, in (r, Delta) with Delta the epicentral
 * angle: r_min_km .. r_max_km on n_r nodes, 0 .. d_max_deg on n_d nodes (n_r, n_d >= 4).
 * d_s_r: device [n_r] slowness at the grid radii, of dtype; h_r_src_km: host [n_ev] the
 * events' radii (inside [r_min, r_max]); d_T: device [n_ev][n_r][n_d] output of dtype.
 * Factored (T0 = s(r_s) x chord) Godunov sweeps, the axis Delta = 0 a mirror, the other
 * faces extrapolated; each event stops when an iteration's largest change of tau is below
 * tol. h_iters: host [n_ev] iterations (may be NULL). Synchronises the stream;
 * TT_ENOTCONVERGED when an event reached max_iter. */
tt_status tt_tele2d(tt_ctx *ctx, int dtype, int n_r, int n_d, double r_min_km, double r_max_km,
                    double d_max_deg, const void *d_s_r, int n_ev, const double *h_r_src_km,
                    double tol, int max_iter, void *d_T, int *h_iters);

/* The 2-D times of tt_tele2d interpolated (bilinearly in r and Delta) at every node of the
 * context's grid, for events at h_events (host [n_ev]; only latitude and longitude are read):
 * d_T device [N][n_ev] of dtype, the layout of tt_forward. Its faces are the Dirichlet data
 * of the region's solve and its interior a starting value. The 2-D grid must cover the
 * region (radii and epicentral angles), else TT_EINVAL. */
tt_status tt_tele_region_times(tt_ctx *ctx, int dtype, int n_r, int n_d, double r_min_km,
                               double r_max_km, double d_max_deg, const void *d_T2, int n_ev,
                               const tt_point *h_events, void *d_T);

/* The region's solve for teleseismic events: Lax-Friedrichs sweeps (Sec. 3.1) of T itself
 * (no factor) in the 8 orderings, hyperplane by hyperplane, with the six faces held fixed.
 * d_T: device [N][n_ev] of the model's dtype; on entry its faces are the Dirichlet data and
 * its interior the start (tt_tele_region_times gives both); on return the solution. Each
 * event stops when an iteration's largest change is below opts->tol_fwd (at most
 * opts->max_iter_fwd iterations; TT_ENOTCONVERGED otherwise). The update is computed in the
 * fields' precision: in FP32, T of order 100 s is resolved to about 1e-5 s, so tol_fwd should
 * not be set below that. All events run in one persistent launch (the sweep kernel of
 * tt_forward) that tests convergence on the device. h_iters: host [n_ev] (may be NULL). Waits
 * for the stream before returning. */
tt_status tt_forward_tele(tt_ctx *ctx, const tt_model *model, int n_ev, void *d_T,
                          const tt_opts *opts, int *h_iters);

/* Largest receiver count tt_misfit_noalloc accepts: the size of its static scratch. */
#define TT_NOALLOC_MAX_REC 1024

/* tt_misfit_noalloc — the results of tt_misfit (same kernels, same outputs, same layouts)
 * without a context and without any device allocation. It is meant for callers that cannot
 * allocate device memory at the point of the call: for example a serving process that
 * handed all of its HBM to its own pool allocator at start-up, or a pipeline stage that must
 * not take cudaMalloc's implicit device-wide synchronisation. The paper has no counterpart;
 * it is a convenience of this library.
 * Scratch: one static device array of about 156 KB per GPU that loads the library (held
 * until the process exits), holding the receiver positions, cells and weights and two flags;
 * hence n_rec must be 1..TT_NOALLOC_MAX_REC, and larger counts return TT_EINVAL with a
 * message saying so. The flags are cleared by every call; the other contents are whatever
 * the last call left. Every call on a device shares that array, so calls whose GPU work
 * overlaps (other host threads, other streams) race; issue them one after another.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture. CUDA loads a
 * library's device code lazily by default, so that first call may also be what loads this
 * module onto the device and places the static array in device memory: make it before the
 * device's memory is handed to the caller's pool, or that placement can fail for lack of
 * memory (TT_ECUDA).
 * grid: the study region, validated by the same rules as tt_ctx_create (spherical grids
 * must stay inside latitudes (-89, 89)). cuda_stream: the cudaStream_t to
 * run on (NULL for the default stream). h_err/err_len: optional host buffer that receives a
 * one-line message (may be NULL). The call waits for its stream before returning. */
tt_status tt_misfit_noalloc(const tt_grid *grid, const void *d_T, int dtype,
                            const tt_data *data, double *d_Tr, double *d_chi, double *d_R,
                            void *cuda_stream, char *h_err, int err_len);

/* Autotuner: times the candidate launch configurations of the forward sweep on this
 * workload and writes the fastest into opts (sweep_schedule, fwd_groups). Candidates, in
 * this order: node hyperplanes with 1, 2, 4 and 8 barrier groups, then tile hyperplanes
 * 2x4x8, 4x4x4, 2x8x8 (tiles need n_src >= 32 and rows of 16-byte multiples; skipped
 * ones time 0). With Lax-Friedrichs (opts->scheme = 0) each runs max_iter_fwd = 2
 * iterations; with a Godunov solver each runs the whole solve on the node-hyperplane
 * schedule (tile candidates time 0), since there the sources' unequal iteration counts decide
 * how barrier groups share the GPU. The runs use a scratch tau owned by the context; every
 * candidate gives the same results, so only time decides. h_ms (host [7], may be NULL)
 * receives each candidate's device time per iteration. The choice is cached per
 * (n_src, dtype, scheme): a later call with the same triple only writes it into opts. */
tt_status tt_autotune(tt_ctx *ctx, const tt_model *model, const tt_point *h_src, int n_src,
                      tt_opts *opts, double *h_ms);

/* Autotuner of the adjoint sweep (Eq. 5): times whole adjoint solves of this batch (d_T, n_rec,
 * h_rec and d_R as for tt_adjoint; the adjoint field goes to a workspace buffer) in six launch
 * configurations and writes the fastest into opts (adj_chunk, adj_groups). Candidates, in
 * this order (adj_chunk, adj_groups): (all, 1), (all, 2), (all, 4), (all, 8), (128, auto),
 * (64, 1); h_ms (host [6], may be NULL) receives each one's device time (0 = skipped: fewer
 * than 32 sources per group, or a chunk no smaller than the batch). Results do not depend on
 * the choice. Cached per (n_src, dtype) like tt_autotune. */
tt_status tt_autotune_adjoint(tt_ctx *ctx, const tt_model *model, const tt_point *h_src,
                              int n_src, const void *d_T, int n_rec, const tt_point *h_rec,
                              const double *d_R, tt_opts *opts, double *h_ms);

/* ---- Warm-start network. A small 3D convolutional network predicts the factored correction
 * tau of Sec. 3.1 (T = T0 tau) from local quantities, so that the forward sweep of Sec. 3.1
 * starts closer to its fixed point (opts.init = 2); the sweep still runs to tol_fwd, so the
 * result meets the same tolerance whatever the network predicts.
 *
 * Input: six channels per node, s / s0 - 1 (s0 = slowness at the source), xi, eta, and the
 * offset D to the source in the source's (up, north, east) frame in units of 100 km (the
 * offset that defines T0). Network: four 3x3x3 convolutions 6 -> 32 -> 32 -> 32 -> 1, zero
 * padding outside the grid, ReLU after the first three; output y; warm start
 * tau = 1 + clamp(y, -0.5, 1), and tau = 1 where y is not a number (the fixed set keeps
 * tau = 1). Any start in [0.5, 2] converges to the same fixed point, so a poor or broken
 * network costs sweeps but not accuracy.
 * Parameters: one FP32 vector of tt_net_param_count() values: for each layer l, weights
 * W[27][C_in][C_out] (tap (dz * 3 + dy) * 3 + dx reads the node at offset (dz-1, dy-1, dx-1)
 * along (r, theta, phi)), then biases b[C_out].
 * Fields are channels-last FP32 on the network's grid: features [n][Nn][6], outputs
 * [n][Nn], where Nn = tt_net_nodes(ctx). The network's grid is the context's grid (stride 1,
 * the default) or, after tt_net_set_stride(ctx, 2), every other node along each axis with the
 * last node of an axis always included (n -> ceil((n - 1) / 2) + 1 nodes): the warm start
 * then evaluates the network there, about 8x fewer nodes, and interpolates its clamped
 * prediction trilinearly to every node. A network is trained for one stride (its 3x3x3
 * taps span that spacing), so the stride goes with the weights.
 * All calls below wait for the context's stream before returning. */
int tt_net_param_count(void);
/* Sets the stride of the network's grid (1 or 2; TT_EINVAL otherwise). Affects every call
 * below and opts.init = 2 of later forward calls and plans (a plan keeps the stride it was
 * created with). */
tt_status tt_net_set_stride(tt_ctx *ctx, int stride);
/* Nn: the node count of the network's grid (0 for a NULL context). */
int tt_net_nodes(const tt_ctx *ctx);
/* d_x (device [n_src][Nn][6] float) = the network input for each source at the nodes of the
 * network's grid (the values of the solver-grid node each one sits on). */
tt_status tt_net_features(tt_ctx *ctx, const tt_model *model, const tt_point *h_src, int n_src,
                          float *d_x);
/* d_y (device [n_grids][Nn] float) = network output y for n_grids inputs d_x, FP32 weights. */
tt_status tt_net_forward(tt_ctx *ctx, const float *d_theta, const float *d_x, int n_grids,
                         float *d_y);
/* Masked mean squared error loss = sum m (y - (tau - 1))^2 / sum m over n_grids grids
 * (d_target = the converged tau and d_mask, device [n_grids][Nn] float) and its gradient
 * with respect to the parameters
 * (d_grad, device [tt_net_param_count()], overwritten). The loss goes to *h_loss (may be
 * NULL). Deterministic: fixed-order reductions. */
tt_status tt_net_loss_grad(tt_ctx *ctx, const float *d_theta, const float *d_x,
                           const float *d_target, const float *d_mask, int n_grids,
                           float *d_grad, double *h_loss);
/* tt_net_loss_grad with the convolutions on the tensor cores: the forward pass, the
 * gradients through the layers' inputs (transposed convolutions, gated by the ReLU of the
 * layer below) and the weight and bias gradients (input rows times output-gradient rows,
 * summed over the rows) run on tcgen05 with BF16 operands (weights, activations and
 * gradients rounded to BF16) and FP32 accumulation in tensor memory; the per-SM sums are
 * added in FP64 in a fixed order. Same arguments and outputs as tt_net_loss_grad; the
 * result is that gradient to BF16 accuracy (bar stated in the tests). Deterministic.
 * TT_ETIMEOUT if a device-side wait exceeds 2 s. */
tt_status tt_net_loss_grad_tc(tt_ctx *ctx, const float *d_theta, const float *d_x,
                              const float *d_target, const float *d_mask, int n_grids,
                              float *d_grad, double *h_loss);
/* One Adam step (Kingma & Ba) on d_theta with first and second moments d_m, d_v (device,
 * zero before step 1); step counts from 1. */
tt_status tt_net_adam(tt_ctx *ctx, float *d_theta, const float *d_grad, float *d_m, float *d_v,
                      int step, float lr, float beta1, float beta2, float eps);
/* Stores the weights the warm start uses (device FP32 vector, rounded to BF16 and kept by
 * the context; inference accumulates in FP32). Needed before opts.init = 2. */
tt_status tt_net_set_weights(tt_ctx *ctx, const float *d_theta);
/* The warm start's inference with the stored weights: d_y (device [n_grids][Nn] float) =
 * network output for d_x (device [n_grids][Nn][6] float, as tt_net_features writes it). All
 * four layers run on the tensor cores (tcgen05, BF16 operands: the features are rounded
 * to BF16; FP32 accumulation); activations between layers are BF16. Agrees with
 * tt_net_forward to BF16 accuracy. TT_ETIMEOUT if a device-side wait exceeds 2 s. */
tt_status tt_net_infer(tt_ctx *ctx, const float *d_x, int n_grids, float *d_y);
/* The start of opts.init = 2 without the sweep: d_tau (device [N][n_src], the model's dtype)
 * = 1 + the clamped network prediction (interpolated from the network's grid when its stride
 * is 2), and 1 on each source's fixed set. Needs tt_net_set_weights. TT_ETIMEOUT if a
 * device-side wait exceeds 2 s. */
tt_status tt_net_start(tt_ctx *ctx, const tt_model *model, const tt_point *h_src, int n_src,
                       void *d_tau);

/* A plan: one whole step over one batch (forward, misfit and adjoint sources, adjoint,
 * kernels) captured once into a CUDA graph and replayed by tt_plan_run, so that a step costs
 * one graph launch and one small read-back. The plan binds the model arrays, the data and the
 * output buffers given here (their contents may change between runs: an inversion updates
 * s, xi, eta in place) and owns its own workspace; the source and receiver positions are
 * fixed at creation. Each run overwrites tau, T, P, chi, R and the kernels Ks, Kxi, Keta
 * (which then hold this batch's sums only). Shapes as in the individual calls: tau, T, P
 * [N][n_src] of the model's dtype, d_chi [n_src][2] (may be NULL), d_R [n_src][n_rec].
 * Creation synchronises the stream; the graph uses the context's stream. */
typedef struct tt_plan tt_plan;
tt_status tt_plan_create(tt_plan **out, tt_ctx *ctx, const tt_model *model,
                         const tt_point *h_src, int n_src, const tt_data *data,
                         const tt_opts *opts, void *d_tau, void *d_T, void *d_P, double *d_chi,
                         double *d_R, double *d_Ks, double *d_Kxi, double *d_Keta);
/* tt_plan_create with the common-receiver differential times of the batch in the step
 * (Eq. 4 and its adjoint source, Eq. A4; tt_cr_data as for tt_misfit_cr, its n_src and
 * n_rec those of the batch): after the misfit the graph writes the receiver-time table to
 * d_Tr (device double [n_src][n_rec]), adds gamma dchi_cr/dT into d_R and writes each
 * source's share of chi_cr to d_chi_cr (device double [n_src]), then runs the adjoint. Every
 * entry's other source is checked once at creation (TT_EINVAL if outside the batch);
 * entries must not change between runs. Pairs across batches need the joined tables and stay
 * with tt_misfit_cr. */
tt_status tt_plan_create_cr(tt_plan **out, tt_ctx *ctx, const tt_model *model,
                            const tt_point *h_src, int n_src, const tt_data *data,
                            const tt_cr_data *cr, const tt_opts *opts, void *d_tau, void *d_T,
                            void *d_P, double *d_chi, double *d_Tr, double *d_chi_cr,
                            double *d_R, double *d_Ks, double *d_Kxi, double *d_Keta);
/* Replays the step and waits for it; h_iters_fwd / h_iters_adj (host [n_src], may be NULL)
 * receive the iteration counts. Statuses as tt_forward and tt_adjoint. */
tt_status tt_plan_run(tt_plan *plan, int *h_iters_fwd, int *h_iters_adj);
void tt_plan_destroy(tt_plan *plan);

/* Copies the measurements of the last forward (which = TT_STATS_FORWARD) or adjoint
 * (TT_STATS_ADJOINT) sweep, or of the last kernel accumulation (TT_STATS_KERNEL, which first
 * waits for that accumulation to finish). Host only; call after the solve returned. */
tt_status tt_get_stats(const tt_ctx *ctx, int which, tt_stats *out);

#ifdef __cplusplus
}
#endif
#endif
