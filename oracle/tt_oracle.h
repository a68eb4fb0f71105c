/*
 * FP64 CPU oracle for adjoint-state traveltime tomography (TomoATT, arXiv 2412.00031).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, single-threaded restatement of the
 * method, used by the test suite, by the smoke check and by the CPU-baseline leg of the
 * benchmark. The product library never links, loads or calls it, and it shares no code,
 * header, table or helper with the CUDA path.
 *
 * Every array is a plain C array in FP64. Fields are stored [n_r][n_t][n_p] with the
 * longitude index fastest. One call handles one source.
 *
 * What each function follows:
 *   or_T0            multiplicative factor T0 of Sec. 3.1 (Luo & Qian factorisation)
 *   or_forward       anisotropic Eikonal equation (Eq. "4", spherical form) solved by
 *                    factored Lax-Friedrichs fast sweeping (Sec. 3.1, Sec. 3.4)
 *   or_receiver_times, or_misfit   objective terms Eqs. 2-3, adjoint sources Eqs. A2-A3
 *   or_adjoint       adjoint equation Eq. 5 solved by upwind fast sweeping
 *   or_kernel_add    kernels Eqs. 6-8 accumulated over sources
 * Readings where the paper is silent are listed in the .c file beside the code.
 */
#ifndef TT_ORACLE_H
#define TT_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n_r, n_t, n_p;
    double depth_min_km, depth_max_km;
    double lat_min_deg, lat_max_deg;
    double lon_min_deg, lon_max_deg;
    double earth_radius_km;
    int flat; /* 0: spherical (r, latitude, longitude); 1: flat Cartesian test geometry */
} or_grid;

typedef struct {
    double depth_km, lat_deg, lon_deg;
} or_point;

/* T0 and its physical gradient components (p_r, p_theta, p_phi) at every node. */
void or_T0(const or_grid *g, const double *s, const double *xi, const double *eta,
           or_point src, double *T0, double *p0 /* [N][3], may be NULL */);

/* Forward solve for one source. tau_init may be NULL (tau = 1). Writes tau and T = T0*tau.
 * Returns the number of iterations taken; *conv is set to 1 when the L-infinity update
 * fell below tol, *last_err to the final L-infinity update. */
int or_forward(const or_grid *g, const double *s, const double *xi, const double *eta,
               or_point src, double tol, int max_iter, const double *tau_init,
               double *tau, double *T, int *conv, double *last_err);
/* or_forward with the Godunov local solver (R14) for isotropic models (xi = eta = 0). */
int or_forward_godunov(const or_grid *g, const double *s, const double *xi, const double *eta,
                       or_point src, double tol, int max_iter, const double *tau_init,
                       double *tau, double *T, int *conv, double *last_err);
/* or_forward with the anisotropic Godunov local solver (R16), any model. */
int or_forward_godunov_aniso(const or_grid *g, const double *s, const double *xi,
                             const double *eta, or_point src, double tol, int max_iter,
                             const double *tau_init, double *tau, double *T, int *conv,
                             double *last_err);

/* Trilinear interpolation of nodal T at n_rec points. */
void or_receiver_times(const or_grid *g, const double *T, int n_rec, const or_point *rec,
                       double *Tr);

/* Misfit and adjoint sources of one source from receiver times Tr[n_rec].
 * Absolute data: n_abs records (rec index, T_obs, weight).
 * Common-source differential data: n_cs unordered pairs (m, i, dT_obs, weight).
 * Writes chi[0] = chi_t, chi[1] = chi_cs and R[n_rec] = alpha*dchi_t/dT + beta*dchi_cs/dT. */
void or_misfit(int n_rec, const double *Tr,
               int n_abs, const int *abs_rec, const double *abs_tobs, const double *abs_w,
               int n_cs, const int *cs_m, const int *cs_i, const double *cs_dtobs,
               const double *cs_w, double alpha, double beta, double *chi, double *R);

/* Adjoint solve for one source. R[n_rec] are the adjoint sources at the receivers.
 * Returns iterations; *conv as in or_forward (criterion relative to max |P|). */
int or_adjoint(const or_grid *g, const double *T, const double *xi, const double *eta,
               or_point src, int n_rec, const or_point *rec, const double *R,
               double tol, int max_iter, double *P, int *conv, double *last_err);

/* Adds one source's contribution to the kernels: Ks += s^2 P, Kxi += P(g_t^2 - g_p^2),
 * Keta += -2 P g_t g_p. */
void or_kernel_add(const or_grid *g, const double *s, const double *T, const double *P,
                   double *Ks, double *Kxi, double *Keta);

/* Net adjoint flux from the non-fixed nodes into the fixed source set (test of Eq. 5's
 * conservation form: at convergence it equals the sum of the adjoint sources). */
double or_fixed_set_inflow(const or_grid *g, const double *T, const double *xi,
                           const double *eta, or_point src, const double *P);

/* Control volume of every node (used to turn kernels into integrals, Eq. 9). */
void or_node_volumes(const or_grid *g, double *dV);

/* Hyperplane-ordered variant of the forward sweep, used only to test that the sweep
 * result does not depend on the order in which a hyperplane's nodes are visited. */
int or_forward_hyperplane(const or_grid *g, const double *s, const double *xi,
                          const double *eta, or_point src, double tol, int max_iter,
                          const double *tau_init, double *tau, double *T, int *conv,
                          double *last_err);

/* Timing units of the CPU baseline: n_sweeps forward sweeps from tau = 1, or n_sweeps
 * adjoint sweeps from P = 0 (orderings 0, 1, ... as in a solve). */
void or_forward_sweeps(const or_grid *g, const double *s, const double *xi, const double *eta,
                       or_point src, int n_sweeps, double *tau);
void or_adjoint_sweeps(const or_grid *g, const double *T, const double *xi, const double *eta,
                       or_point src, int n_rec, const or_point *rec, const double *R,
                       int n_sweeps, double *P);

#ifdef __cplusplus
}
#endif
/* Teleseismic events (R17): 2-D traveltimes in a 1-D model, and the 3-D solve with the
 * faces of the region held fixed. */
int or_tele2d(int n_r, int n_d, double r_min, double r_max, double d_max, const double *s_r,
              double r_s, double tol, int max_iter, double *T, int *conv);
int or_forward_tele(const or_grid *g, const double *s, const double *xi, const double *eta,
                    double tol, int max_iter, double *T, int *conv, double *last_err);

#endif
