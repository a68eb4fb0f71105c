/*
 * FP64 CPU oracle for adjoint-state traveltime tomography (TomoATT, arXiv 2412.00031).
 * TEST INFRASTRUCTURE ONLY: see tt_oracle.h. Plain loops, no blocking, no fusion.
 *
 * Readings of the paper used here (it names the methods but not their discretisation):
 *  R1  Grid: r_i = R_E - depth_max + i*dr (radius ascending), theta = latitude (Eq. "4" uses
 *      1/(r cos theta)), phi = longitude, uniform spacing per axis, R_E = 6371 km by default.
 *  R2  Factor (Sec. 3.1, multiplicative factorisation): T = T0 * tau with
 *      T0 = s0 * sqrt(D^T M0^-1 D), D = the Cartesian offset to the source expressed in the
 *      source's local (up, north, east) frame, (s0, xi0, eta0) interpolated at the source.
 *  R3  Fixed set: tau = 1 on the 3x3x3 nodes around the node nearest the source.
 *  R4  Local solver: Lax-Friedrichs update of tau with Cauchy-Schwarz viscosity bounds.
 *  R5  Sweep orderings: o = 0..7, r direction from bit 2, theta from bit 1, phi from bit 0
 *      (bit set = descending); lexicographic visiting order with phi innermost.
 *  R6  Boundary: tau on each face = max(2 tau_1 - tau_2, tau_2) after every sweep, faces in
 *      the order r, theta, phi (low face, then high face), fixed nodes exempt.
 *  R7  Convergence: largest |change| over the interior updates of one iteration < tol.
 *  R8  Receiver time: trilinear interpolation of nodal T in index space.
 *  R9  Adjoint: conservative first-order upwind finite-volume form of Eq. 5, zero flux
 *      through the outer faces, P = 0 on the fixed set, Gauss-Seidel sweeps in the same
 *      8 orderings over every node; the point source of Eq. 5 is spread to the 8 corners
 *      of the receiver's cell with the trilinear weights of R8, divided by the node volume.
 *  R10 Kernel gradients: central differences of nodal T, one-sided on the faces.
 *  R14 Godunov local solver (isotropic models, xi = eta = 0; an alternative to R4): one-sided
 *      differences of tau toward the upwind neighbour of each axis, the neighbour with the
 *      smaller first-order estimate of T = T0 tau (T0 at the neighbour taken as
 *      T0_c (1 +- u_d / e_d), u = grad T0 / T0, e_d = 1 / (delta_d h_d)); tau_c is the
 *      smallest root, over the 7 non-empty subsets of axes, of
 *      sum_d (a_d tau - b_d)^2 = (s / T0)^2 (the larger root of each quadratic) whose
 *      one-sided differences all have the upwind sign; with no such root tau_c is kept.
 *  R17 Teleseismic sources (the boundary condition of Eq. "4" for an event outside the region):
 *      the times on the region's faces come from a 2-D eikonal solve in a 1-D global model
 *      s(r), in (r, Delta) with Delta the epicentral angle from the event. The 2-D solve is
 *      factored as R2 (T0 = s(r_s) x chord) with R14's Godunov update in two dimensions,
 *      mirror symmetry on the axis Delta = 0, R6's extrapolation on the other faces, and R3's
 *      fixed set (3 x 2 nodes next to the event, on the axis). The faces of the 3-D region
 *      take the bilinear interpolation of the 2-D times at their (r, Delta). The 3-D solve
 *      is R4's Lax-Friedrichs update on T itself (T0 = 1, no factor), with the faces held
 *      fixed (Dirichlet data, no extrapolation) and the interior swept from a given start.
 *  R16 Godunov local solver for anisotropic models (M of Eq. "4" with xi, eta; an alternative
 *      to R4): as R14, with two changes. (a) Along theta and phi the upwind neighbour is the
 *      side the characteristic comes from: the sign of (M g)_d, g the central-difference
 *      gradient of T / T0 at the node (the quantity LF evaluates); along r, where M has no
 *      cross term, the neighbour with the smaller estimate of T as in R14. (b) For a subset S
 *      of axes the gradient components off S take the values that minimise H, so the
 *      quadratic form on S is the Schur complement W = ((M^-1)_SS)^-1, and the causality
 *      test is sg_d (W g_S)_d >= 0 for d in S (the characteristic M g enters from the
 *      upwind side; it is zero along the axes off S).
 */
#include "tt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define DEG (3.14159265358979323846 / 180.0)

/* ---------------------------------------------------------------- geometry (R1) */

typedef struct {
    int nr, nt, np;
    double r0, dr, t0, dt, p0, dp, re;
    int flat;
} geo;

static geo make_geo(const or_grid *g)
{
    geo G;
    G.nr = g->n_r; G.nt = g->n_t; G.np = g->n_p;
    G.re = g->earth_radius_km;
    G.r0 = g->earth_radius_km - g->depth_max_km;
    G.dr = (g->depth_max_km - g->depth_min_km) / (g->n_r - 1);
    G.t0 = g->lat_min_deg * DEG;
    G.dt = (g->lat_max_deg - g->lat_min_deg) * DEG / (g->n_t - 1);
    G.p0 = g->lon_min_deg * DEG;
    G.dp = (g->lon_max_deg - g->lon_min_deg) * DEG / (g->n_p - 1);
    G.flat = g->flat;
    return G;
}

static long idx(const geo *G, int i, int j, int k) { return ((long)i * G->nt + j) * G->np + k; }
static double rad_of(const geo *G, int i) { return G->r0 + i * G->dr; }
static double lat_of(const geo *G, int j) { return G->t0 + j * G->dt; }
static double lon_of(const geo *G, int k) { return G->p0 + k * G->dp; }

/* Scale factors of the physical gradient components: p = (dT/dr / h1, dT/dtheta / h2,
 * dT/dphi / h3). Spherical: h1 = 1, h2 = r, h3 = r cos(theta) (Eq. "4"). Flat test
 * geometry: h2 = h3 = R_E, so theta and phi become lengths R_E*theta and R_E*phi. */
static double h2_at(const geo *G, double r) { return G->flat ? G->re : r; }
static double h3_at(const geo *G, double r, double th) { return G->flat ? G->re : r * cos(th); }

/* Position in Cartesian km and the local unit vectors (e_r, e_theta, e_phi). */
static void position(const geo *G, double r, double th, double ph, double X[3])
{
    if (G->flat) { X[0] = r; X[1] = G->re * th; X[2] = G->re * ph; return; }
    X[0] = r * cos(th) * cos(ph);
    X[1] = r * cos(th) * sin(ph);
    X[2] = r * sin(th);
}

static void frame(const geo *G, double th, double ph, double E[3][3])
{
    /* E[a] is the a-th local unit vector (a = r, theta, phi) in Cartesian components. */
    if (G->flat) {
        memset(E, 0, 9 * sizeof(double));
        E[0][0] = E[1][1] = E[2][2] = 1.0;
        return;
    }
    E[0][0] = cos(th) * cos(ph); E[0][1] = cos(th) * sin(ph); E[0][2] = sin(th);
    E[1][0] = -sin(th) * cos(ph); E[1][1] = -sin(th) * sin(ph); E[1][2] = cos(th);
    E[2][0] = -sin(ph); E[2][1] = cos(ph); E[2][2] = 0.0;
}

/* Fractional grid index of a point. */
static void frac_index(const geo *G, or_point p, double f[3])
{
    double r = G->re - p.depth_km;
    f[0] = (r - G->r0) / G->dr;
    f[1] = (p.lat_deg * DEG - G->t0) / G->dt;
    f[2] = (p.lon_deg * DEG - G->p0) / G->dp;
}

/* Trilinear cell and weights (R8): base corner b[3], weights w[8] for corners
 * (di, dj, dk) enumerated as c = di*4 + dj*2 + dk. */
static void trilinear(const geo *G, or_point p, int b[3], double w[8])
{
    double f[3];
    int n[3] = {G->nr, G->nt, G->np};
    double u[3];
    frac_index(G, p, f);
    for (int a = 0; a < 3; a++) {
        int i0 = (int)floor(f[a]);
        if (i0 < 0) i0 = 0;
        if (i0 > n[a] - 2) i0 = n[a] - 2;
        b[a] = i0;
        u[a] = f[a] - i0;
    }
    for (int c = 0; c < 8; c++) {
        double wr = (c & 4) ? u[0] : 1.0 - u[0];
        double wt = (c & 2) ? u[1] : 1.0 - u[1];
        double wp = (c & 1) ? u[2] : 1.0 - u[2];
        w[c] = wr * wt * wp;
    }
}

static double interp(const geo *G, const double *F, or_point p)
{
    int b[3];
    double w[8], acc = 0.0;
    trilinear(G, p, b, w);
    for (int c = 0; c < 8; c++)
        acc += w[c] * F[idx(G, b[0] + ((c >> 2) & 1), b[1] + ((c >> 1) & 1), b[2] + (c & 1))];
    return acc;
}

/* ---------------------------------------------------------------- factor T0 (R2) */

typedef struct {
    double Xs[3];      /* source position */
    double Es[3][3];   /* source frame */
    double Minv[3][3]; /* inverse of M(xi0, eta0) */
    double s0;
    int ci, cj, ck;    /* node nearest the source (R3) */
} source_factor;

/* The anisotropy matrix of Eq. "4" in (r, theta, phi) components. */
static void aniso_M(double xi, double eta, double M[3][3])
{
    M[0][0] = 1.0; M[0][1] = 0.0;            M[0][2] = 0.0;
    M[1][0] = 0.0; M[1][1] = 1.0 - 2.0 * xi; M[1][2] = 2.0 * eta;
    M[2][0] = 0.0; M[2][1] = 2.0 * eta;      M[2][2] = 1.0 + 2.0 * xi;
}

static void inverse3(double A[3][3], double B[3][3])
{
    double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
               - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
               + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    B[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
    B[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
    B[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
    B[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
    B[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
    B[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
    B[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
    B[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
    B[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
}

static source_factor make_source(const geo *G, const double *s, const double *xi,
                                 const double *eta, or_point src)
{
    source_factor S;
    double M[3][3], f[3];
    double r = G->re - src.depth_km, th = src.lat_deg * DEG, ph = src.lon_deg * DEG;
    int n[3] = {G->nr, G->nt, G->np};
    int c[3];
    position(G, r, th, ph, S.Xs);
    frame(G, th, ph, S.Es);
    S.s0 = interp(G, s, src);
    aniso_M(interp(G, xi, src), interp(G, eta, src), M);
    inverse3(M, S.Minv);
    frac_index(G, src, f);
    for (int a = 0; a < 3; a++) {
        c[a] = (int)floor(f[a] + 0.5);
        if (c[a] < 0) c[a] = 0;
        if (c[a] > n[a] - 1) c[a] = n[a] - 1;
    }
    S.ci = c[0]; S.cj = c[1]; S.ck = c[2];
    return S;
}

static int is_fixed(const source_factor *S, int i, int j, int k)
{
    return abs(i - S->ci) <= 1 && abs(j - S->cj) <= 1 && abs(k - S->ck) <= 1;
}

/* T0 at a node and the physical components of grad T0 there. */
static double factor_at(const geo *G, const source_factor *S, int i, int j, int k, double p0[3])
{
    double r = rad_of(G, i), th = lat_of(G, j), ph = lon_of(G, k);
    double X[3], d[3], D[3], MD[3], grad[3], E[3][3];
    position(G, r, th, ph, X);
    for (int a = 0; a < 3; a++) d[a] = X[a] - S->Xs[a];
    for (int a = 0; a < 3; a++) D[a] = S->Es[a][0] * d[0] + S->Es[a][1] * d[1] + S->Es[a][2] * d[2];
    for (int a = 0; a < 3; a++)
        MD[a] = S->Minv[a][0] * D[0] + S->Minv[a][1] * D[1] + S->Minv[a][2] * D[2];
    double q = D[0] * MD[0] + D[1] * MD[1] + D[2] * MD[2];
    double T0 = S->s0 * sqrt(q);
    if (p0) {
        if (q <= 0.0) {
            p0[0] = p0[1] = p0[2] = 0.0;
        } else {
            /* grad_X T0 = s0^2 Es^T Minv D / T0, then projected on the node's frame. */
            for (int a = 0; a < 3; a++)
                grad[a] = (S->Es[0][a] * MD[0] + S->Es[1][a] * MD[1] + S->Es[2][a] * MD[2])
                          * S->s0 * S->s0 / T0;
            frame(G, th, ph, E);
            for (int a = 0; a < 3; a++)
                p0[a] = E[a][0] * grad[0] + E[a][1] * grad[1] + E[a][2] * grad[2];
        }
    }
    return T0;
}

void or_T0(const or_grid *g, const double *s, const double *xi, const double *eta,
           or_point src, double *T0, double *p0)
{
    geo G = make_geo(g);
    source_factor S = make_source(&G, s, xi, eta, src);
    for (int i = 0; i < G.nr; i++)
        for (int j = 0; j < G.nt; j++)
            for (int k = 0; k < G.np; k++) {
                long n = idx(&G, i, j, k);
                double p[3];
                T0[n] = factor_at(&G, &S, i, j, k, p);
                if (p0) { p0[3 * n] = p[0]; p0[3 * n + 1] = p[1]; p0[3 * n + 2] = p[2]; }
            }
}

/* ---------------------------------------------------------------- forward (R3-R7) */

/* Lax-Friedrichs update of tau at interior node (i,j,k) (R4). With T = T0 tau,
 *   p = tau_c p0 + T0 (D_r tau / h1, D_t tau / h2, D_p tau / h3)   (central differences)
 *   H(p) = sqrt(p^T M p)                                           (Eq. "4": H = s)
 *   sigma_1 = T0, sigma_2 = T0 sqrt(1 - 2 xi) / h2, sigma_3 = T0 sqrt(1 + 2 xi) / h3
 *   tau_c <- [s - H(p) + sum_d sigma_d (tau_d+ + tau_d-) / (2 delta_d)] / sum_d sigma_d / delta_d
 * sigma_d bounds |dH/d(d_d tau)|, which keeps the scheme monotone. */
static double lf_update(const geo *G, const source_factor *S, const double *s,
                        const double *xi, const double *eta, const double *tau,
                        int i, int j, int k)
{
    long c = idx(G, i, j, k);
    double p0[3];
    double T0 = factor_at(G, S, i, j, k, p0);
    double r = rad_of(G, i), th = lat_of(G, j);
    double h[3] = {1.0, h2_at(G, r), h3_at(G, r, th)};
    double del[3] = {G->dr, G->dt, G->dp};
    double tp[3], tm[3];
    tp[0] = tau[idx(G, i + 1, j, k)]; tm[0] = tau[idx(G, i - 1, j, k)];
    tp[1] = tau[idx(G, i, j + 1, k)]; tm[1] = tau[idx(G, i, j - 1, k)];
    tp[2] = tau[idx(G, i, j, k + 1)]; tm[2] = tau[idx(G, i, j, k - 1)];

    double p[3];
    for (int d = 0; d < 3; d++)
        p[d] = tau[c] * p0[d] + T0 * (tp[d] - tm[d]) / (2.0 * del[d]) / h[d];
    double M[3][3];
    aniso_M(xi[c], eta[c], M);
    double q = 0.0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) q += p[a] * M[a][b] * p[b];
    double H = sqrt(q);

    double sigma[3] = {T0, T0 * sqrt(1.0 - 2.0 * xi[c]) / h[1], T0 * sqrt(1.0 + 2.0 * xi[c]) / h[2]};
    double num = s[c] - H, den = 0.0;
    for (int d = 0; d < 3; d++) {
        num += sigma[d] * (tp[d] + tm[d]) / (2.0 * del[d]);
        den += sigma[d] / del[d];
    }
    return num / den;
}

/* Godunov update of tau at interior node (i,j,k) (R14; xi = eta = 0). With sigma_d = +1 for a
 * backward (lower-neighbour) difference and -1 for a forward one, the physical gradient over
 * T0 along axis d is a_d tau_c - b_d, a_d = u_d + sigma_d e_d, b_d = sigma_d e_d tau_nb. */
static double godunov_update(const geo *G, const source_factor *S, const double *s,
                             const double *tau, int i, int j, int k)
{
    long c = idx(G, i, j, k);
    double p0[3];
    double T0 = factor_at(G, S, i, j, k, p0);
    double r = rad_of(G, i), th = lat_of(G, j);
    double h[3] = {1.0, h2_at(G, r), h3_at(G, r, th)};
    double del[3] = {G->dr, G->dt, G->dp};
    double tp[3], tm[3];
    tp[0] = tau[idx(G, i + 1, j, k)]; tm[0] = tau[idx(G, i - 1, j, k)];
    tp[1] = tau[idx(G, i, j + 1, k)]; tm[1] = tau[idx(G, i, j - 1, k)];
    tp[2] = tau[idx(G, i, j, k + 1)]; tm[2] = tau[idx(G, i, j, k - 1)];
    double a[3], b[3], sg[3];
    for (int d = 0; d < 3; d++) {
        double u = p0[d] / T0, e = 1.0 / (del[d] * h[d]);
        /* T at the neighbours over T0_c, to first order */
        double tlo = tm[d] * (1.0 - u / e), thi = tp[d] * (1.0 + u / e);
        sg[d] = tlo <= thi ? 1.0 : -1.0;
        double nb = tlo <= thi ? tm[d] : tp[d];
        a[d] = u + sg[d] * e;
        b[d] = sg[d] * e * nb;
    }
    double rhs = s[c] / T0;
    double best = -1.0;
    for (int mask = 1; mask < 8; mask++) {
        double A = 0.0, B = 0.0, C = -rhs * rhs;
        for (int d = 0; d < 3; d++)
            if (mask >> d & 1) { A += a[d] * a[d]; B += a[d] * b[d]; C += b[d] * b[d]; }
        double disc = B * B - A * C;
        if (!(A > 0.0) || disc < 0.0) continue;
        double t = (B + sqrt(disc)) / A;
        int ok = 1;
        for (int d = 0; d < 3; d++)
            if ((mask >> d & 1) && sg[d] * (a[d] * t - b[d]) < 0.0) ok = 0;
        if (ok && (best < 0.0 || t < best)) best = t;
    }
    return best < 0.0 ? tau[c] : best;
}

/* Face extrapolation after every sweep (R6). */
static void extrapolate_faces(const geo *G, const source_factor *S, double *tau)
{
    int nr = G->nr, nt = G->nt, np = G->np;
    for (int j = 0; j < nt; j++)
        for (int k = 0; k < np; k++) {
            if (!is_fixed(S, 0, j, k)) {
                double a = tau[idx(G, 1, j, k)], b = tau[idx(G, 2, j, k)];
                tau[idx(G, 0, j, k)] = fmax(2.0 * a - b, b);
            }
            if (!is_fixed(S, nr - 1, j, k)) {
                double a = tau[idx(G, nr - 2, j, k)], b = tau[idx(G, nr - 3, j, k)];
                tau[idx(G, nr - 1, j, k)] = fmax(2.0 * a - b, b);
            }
        }
    for (int i = 0; i < nr; i++)
        for (int k = 0; k < np; k++) {
            if (!is_fixed(S, i, 0, k)) {
                double a = tau[idx(G, i, 1, k)], b = tau[idx(G, i, 2, k)];
                tau[idx(G, i, 0, k)] = fmax(2.0 * a - b, b);
            }
            if (!is_fixed(S, i, nt - 1, k)) {
                double a = tau[idx(G, i, nt - 2, k)], b = tau[idx(G, i, nt - 3, k)];
                tau[idx(G, i, nt - 1, k)] = fmax(2.0 * a - b, b);
            }
        }
    for (int i = 0; i < nr; i++)
        for (int j = 0; j < nt; j++) {
            if (!is_fixed(S, i, j, 0)) {
                double a = tau[idx(G, i, j, 1)], b = tau[idx(G, i, j, 2)];
                tau[idx(G, i, j, 0)] = fmax(2.0 * a - b, b);
            }
            if (!is_fixed(S, i, j, np - 1)) {
                double a = tau[idx(G, i, j, np - 2)], b = tau[idx(G, i, j, np - 3)];
                tau[idx(G, i, j, np - 1)] = fmax(2.0 * a - b, b);
            }
        }
}

/* Map a loop counter to a grid index for sweep direction dir (+1 ascending, -1 descending)
 * over [lo, hi]. */
static int swept(int q, int dir, int lo, int hi) { return dir > 0 ? lo + q : hi - q; }

/* Godunov update for anisotropic models (R16). */
static double godunov_aniso_update(const geo *G, const source_factor *S, const double *s,
                                   const double *xi, const double *eta, const double *tau,
                                   int i, int j, int k)
{
    long c = idx(G, i, j, k);
    double p0[3];
    double T0 = factor_at(G, S, i, j, k, p0);
    double r = rad_of(G, i), th = lat_of(G, j);
    double h[3] = {1.0, h2_at(G, r), h3_at(G, r, th)};
    double del[3] = {G->dr, G->dt, G->dp};
    double tp[3], tm[3];
    tp[0] = tau[idx(G, i + 1, j, k)]; tm[0] = tau[idx(G, i - 1, j, k)];
    tp[1] = tau[idx(G, i, j + 1, k)]; tm[1] = tau[idx(G, i, j - 1, k)];
    tp[2] = tau[idx(G, i, j, k + 1)]; tm[2] = tau[idx(G, i, j, k - 1)];
    double M[3][3], Mi[3][3];
    aniso_M(xi[c], eta[c], M);
    inverse3(M, Mi);
    double u[3], e[3], gc[3];
    for (int d = 0; d < 3; d++) {
        u[d] = p0[d] / T0;
        e[d] = 1.0 / (del[d] * h[d]);
        gc[d] = u[d] * tau[c] + 0.5 * e[d] * (tp[d] - tm[d]);
    }
    double a[3], b[3], sg[3];
    for (int d = 0; d < 3; d++) {
        int lower;
        if (d == 0) {
            lower = tm[d] * (1.0 - u[d] / e[d]) <= tp[d] * (1.0 + u[d] / e[d]);
        } else {
            double f = M[d][0] * gc[0] + M[d][1] * gc[1] + M[d][2] * gc[2];
            lower = f >= 0.0;
        }
        sg[d] = lower ? 1.0 : -1.0;
        a[d] = u[d] + sg[d] * e[d];
        b[d] = sg[d] * e[d] * (lower ? tm[d] : tp[d]);
    }
    double rhs = s[c] / T0;
    double best = -1.0;
    for (int mask = 1; mask < 8; mask++) {
        int ax[3], n = 0;
        for (int d = 0; d < 3; d++)
            if (mask >> d & 1) ax[n++] = d;
        /* W = ((M^-1)_SS)^-1, the form on S after minimising H over the other components */
        double W[3][3];
        if (n == 1) {
            W[0][0] = 1.0 / Mi[ax[0]][ax[0]];
        } else if (n == 2) {
            double p = Mi[ax[0]][ax[0]], q = Mi[ax[0]][ax[1]], w = Mi[ax[1]][ax[1]];
            double det = p * w - q * q;
            W[0][0] = w / det; W[0][1] = W[1][0] = -q / det; W[1][1] = p / det;
        } else {
            for (int x = 0; x < 3; x++)
                for (int y = 0; y < 3; y++) W[x][y] = M[x][y];
        }
        double A = 0.0, B = 0.0, C = -rhs * rhs;
        for (int x = 0; x < n; x++)
            for (int y = 0; y < n; y++) {
                A += W[x][y] * a[ax[x]] * a[ax[y]];
                B += W[x][y] * a[ax[x]] * b[ax[y]];
                C += W[x][y] * b[ax[x]] * b[ax[y]];
            }
        double disc = B * B - A * C;
        if (!(A > 0.0) || disc < 0.0) continue;
        double t = (B + sqrt(disc)) / A;
        int ok = 1;
        for (int x = 0; x < n; x++) {
            double f = 0.0;
            for (int y = 0; y < n; y++) f += W[x][y] * (a[ax[y]] * t - b[ax[y]]);
            if (sg[ax[x]] * f < 0.0) ok = 0;
        }
        if (ok && (best < 0.0 || t < best)) best = t;
    }
    return best < 0.0 ? tau[c] : best;
}

/* One sweep of the interior in lexicographic order (R5); returns the largest |change|. */
/* The local solver of the chosen scheme: 0 = Lax-Friedrichs (R4), 1 = Godunov for isotropic
 * models (R14), 2 = Godunov for anisotropic models (R16). */
static double local_update(const geo *G, const source_factor *S, const double *s,
                           const double *xi, const double *eta, const double *tau, int i, int j,
                           int k, int scheme)
{
    if (scheme == 2) return godunov_aniso_update(G, S, s, xi, eta, tau, i, j, k);
    return scheme == 1 ? godunov_update(G, S, s, tau, i, j, k)
                       : lf_update(G, S, s, xi, eta, tau, i, j, k);
}

static double sweep_lex(const geo *G, const source_factor *S, const double *s,
                        const double *xi, const double *eta, double *tau, int o, int scheme)
{
    int dr = (o & 4) ? -1 : 1, dt = (o & 2) ? -1 : 1, dp = (o & 1) ? -1 : 1;
    double err = 0.0;
    for (int a = 0; a < G->nr - 2; a++)
        for (int b = 0; b < G->nt - 2; b++)
            for (int c = 0; c < G->np - 2; c++) {
                int i = swept(a, dr, 1, G->nr - 2);
                int j = swept(b, dt, 1, G->nt - 2);
                int k = swept(c, dp, 1, G->np - 2);
                if (is_fixed(S, i, j, k)) continue;
                long n = idx(G, i, j, k);
                double v = local_update(G, S, s, xi, eta, tau, i, j, k, scheme);
                err = fmax(err, fabs(v - tau[n]));
                tau[n] = v;
            }
    return err;
}

/* The same sweep visiting the nodes hyperplane by hyperplane (a + b + c = L, Sec. 3.4);
 * within a plane the nodes are visited in reverse lexicographic order on purpose. */
static double sweep_planes(const geo *G, const source_factor *S, const double *s,
                           const double *xi, const double *eta, double *tau, int o, int scheme)
{
    int dr = (o & 4) ? -1 : 1, dt = (o & 2) ? -1 : 1, dp = (o & 1) ? -1 : 1;
    int na = G->nr - 2, nb = G->nt - 2, nc = G->np - 2;
    double err = 0.0;
    for (int L = 0; L <= na + nb + nc - 3; L++)
        for (int a = na - 1; a >= 0; a--)
            for (int b = nb - 1; b >= 0; b--) {
                int c = L - a - b;
                if (c < 0 || c >= nc) continue;
                int i = swept(a, dr, 1, G->nr - 2);
                int j = swept(b, dt, 1, G->nt - 2);
                int k = swept(c, dp, 1, G->np - 2);
                if (is_fixed(S, i, j, k)) continue;
                long n = idx(G, i, j, k);
                double v = local_update(G, S, s, xi, eta, tau, i, j, k, scheme);
                err = fmax(err, fabs(v - tau[n]));
                tau[n] = v;
            }
    return err;
}

static int forward_impl(const or_grid *g, const double *s, const double *xi, const double *eta,
                        or_point src, double tol, int max_iter, const double *tau_init,
                        double *tau, double *T, int *conv, double *last_err, int planes,
                        int scheme)
{
    geo G = make_geo(g);
    source_factor S = make_source(&G, s, xi, eta, src);
    long N = (long)G.nr * G.nt * G.np;
    for (long n = 0; n < N; n++) tau[n] = tau_init ? tau_init[n] : 1.0;
    for (int i = 0; i < G.nr; i++)
        for (int j = 0; j < G.nt; j++)
            for (int k = 0; k < G.np; k++)
                if (is_fixed(&S, i, j, k)) tau[idx(&G, i, j, k)] = 1.0;

    int it = 0;
    double err = 0.0;
    *conv = 0;
    while (it < max_iter) {
        err = 0.0;
        for (int o = 0; o < 8; o++) {
            double e = planes ? sweep_planes(&G, &S, s, xi, eta, tau, o, scheme)
                              : sweep_lex(&G, &S, s, xi, eta, tau, o, scheme);
            err = fmax(err, e);
            extrapolate_faces(&G, &S, tau);
        }
        it++;
        if (err < tol) { *conv = 1; break; }
    }
    if (last_err) *last_err = err;
    if (T)
        for (int i = 0; i < G.nr; i++)
            for (int j = 0; j < G.nt; j++)
                for (int k = 0; k < G.np; k++) {
                    long n = idx(&G, i, j, k);
                    T[n] = factor_at(&G, &S, i, j, k, NULL) * tau[n];
                }
    return it;
}

int or_forward(const or_grid *g, const double *s, const double *xi, const double *eta,
               or_point src, double tol, int max_iter, const double *tau_init,
               double *tau, double *T, int *conv, double *last_err)
{
    return forward_impl(g, s, xi, eta, src, tol, max_iter, tau_init, tau, T, conv, last_err, 0, 0);
}

/* The forward solve with the Godunov local solver (R14): xi and eta must be zero (isotropic);
 * they enter only the factor's source values, as in or_forward. */
int or_forward_godunov(const or_grid *g, const double *s, const double *xi, const double *eta,
                       or_point src, double tol, int max_iter, const double *tau_init,
                       double *tau, double *T, int *conv, double *last_err)
{
    return forward_impl(g, s, xi, eta, src, tol, max_iter, tau_init, tau, T, conv, last_err, 0, 1);
}

/* The forward solve with the anisotropic Godunov local solver (R16): any model. */
int or_forward_godunov_aniso(const or_grid *g, const double *s, const double *xi,
                             const double *eta, or_point src, double tol, int max_iter,
                             const double *tau_init, double *tau, double *T, int *conv,
                             double *last_err)
{
    return forward_impl(g, s, xi, eta, src, tol, max_iter, tau_init, tau, T, conv, last_err, 0, 2);
}

int or_forward_hyperplane(const or_grid *g, const double *s, const double *xi,
                          const double *eta, or_point src, double tol, int max_iter,
                          const double *tau_init, double *tau, double *T, int *conv,
                          double *last_err)
{
    return forward_impl(g, s, xi, eta, src, tol, max_iter, tau_init, tau, T, conv, last_err, 1, 0);
}

/* ---------------------------------------------------------------- misfit (Eqs. 2-3, A2-A3) */

void or_receiver_times(const or_grid *g, const double *T, int n_rec, const or_point *rec,
                       double *Tr)
{
    geo G = make_geo(g);
    for (int m = 0; m < n_rec; m++) Tr[m] = interp(&G, T, rec[m]);
}

/* chi_t = sum w/2 (T_m - T_obs)^2 (Eq. 2), dchi_t/dT_m = w (T_m - T_obs) (Eq. A2).
 * The common-source pairs are an unordered list: a pair (m, i) with weight w stands for the
 * two ordered terms (m, i) and (i, m) of Eq. 3 with weight w/2 each, so
 * chi_cs = sum w/2 e^2 with e = (T_m - T_i) - dT_obs, and Eq. A3 gives +w e to R_m and
 * -w e to R_i. */
void or_misfit(int n_rec, const double *Tr,
               int n_abs, const int *abs_rec, const double *abs_tobs, const double *abs_w,
               int n_cs, const int *cs_m, const int *cs_i, const double *cs_dtobs,
               const double *cs_w, double alpha, double beta, double *chi, double *R)
{
    double chi_t = 0.0, chi_cs = 0.0;
    for (int m = 0; m < n_rec; m++) R[m] = 0.0;
    for (int a = 0; a < n_abs; a++) {
        int m = abs_rec[a];
        double e = Tr[m] - abs_tobs[a];
        chi_t += 0.5 * abs_w[a] * e * e;
        R[m] += alpha * abs_w[a] * e;
    }
    for (int q = 0; q < n_cs; q++) {
        int m = cs_m[q], i = cs_i[q];
        double e = (Tr[m] - Tr[i]) - cs_dtobs[q];
        chi_cs += 0.5 * cs_w[q] * e * e;
        R[m] += beta * cs_w[q] * e;
        R[i] -= beta * cs_w[q] * e;
    }
    chi[0] = chi_t;
    chi[1] = chi_cs;
}

/* ---------------------------------------------------------------- adjoint (Eq. 5, R9) */

/* Derivative of T along theta / phi at a node, in index units divided by the spacing:
 * central inside, one-sided on the faces (R10). */
static double d_theta(const geo *G, const double *T, int i, int j, int k)
{
    if (j == 0) return (T[idx(G, i, 1, k)] - T[idx(G, i, 0, k)]) / G->dt;
    if (j == G->nt - 1) return (T[idx(G, i, j, k)] - T[idx(G, i, j - 1, k)]) / G->dt;
    return (T[idx(G, i, j + 1, k)] - T[idx(G, i, j - 1, k)]) / (2.0 * G->dt);
}

static double d_phi(const geo *G, const double *T, int i, int j, int k)
{
    if (k == 0) return (T[idx(G, i, j, 1)] - T[idx(G, i, j, 0)]) / G->dp;
    if (k == G->np - 1) return (T[idx(G, i, j, k)] - T[idx(G, i, j, k - 1)]) / G->dp;
    return (T[idx(G, i, j, k + 1)] - T[idx(G, i, j, k - 1)]) / (2.0 * G->dp);
}

/* Velocity a = -(M grad T) (physical component normal to the face) on the face between
 * node (i,j,k) and its + neighbour along axis d, and the face's area factor A = J / h_d
 * (J = h1 h2 h3). M and the cross-derivative are averaged over the two nodes. */
static double face_velocity(const geo *G, const double *T, const double *xi, const double *eta,
                            int d, int i, int j, int k, double *area)
{
    double r = rad_of(G, i), th = lat_of(G, j);
    if (d == 0) {
        double rf = r + 0.5 * G->dr;
        *area = G->flat ? G->re * G->re : rf * rf * cos(th);
        return -(T[idx(G, i + 1, j, k)] - T[idx(G, i, j, k)]) / G->dr;
    }
    if (d == 1) {
        double thf = th + 0.5 * G->dt;
        double h2 = h2_at(G, r), h3 = h3_at(G, r, thf);
        long c = idx(G, i, j, k), n = idx(G, i, j + 1, k);
        double xh = 0.5 * (xi[c] + xi[n]), eh = 0.5 * (eta[c] + eta[n]);
        double pt = (T[n] - T[c]) / G->dt / h2;
        double pp = 0.5 * (d_phi(G, T, i, j, k) + d_phi(G, T, i, j + 1, k)) / h3;
        *area = h3; /* J / h2 = h1 h3 */
        return -((1.0 - 2.0 * xh) * pt + 2.0 * eh * pp);
    }
    {
        double h2 = h2_at(G, r), h3 = h3_at(G, r, th);
        long c = idx(G, i, j, k), n = idx(G, i, j, k + 1);
        double xh = 0.5 * (xi[c] + xi[n]), eh = 0.5 * (eta[c] + eta[n]);
        double pp = (T[n] - T[c]) / G->dp / h3;
        double pt = 0.5 * (d_theta(G, T, i, j, k) + d_theta(G, T, i, j, k + 1)) / h2;
        *area = h2; /* J / h3 = h1 h2 */
        return -(2.0 * eh * pt + (1.0 + 2.0 * xh) * pp);
    }
}

/* Upwind Gauss-Seidel update of P at node (i,j,k): the discrete Eq. 5 times J_c,
 *   sum_d [A+ (a+^+ P_c + a+^- P_d+) - A- (a-^+ P_d- + a-^- P_c)] / delta_d = J_c S_c,
 * solved for P_c (x^+ = max(x,0), x^- = min(x,0); faces on the outer boundary carry no
 * flux). src is J_c S_c. */
static double adj_update(const geo *G, const source_factor *S, const double *T,
                         const double *xi, const double *eta, const double *P,
                         double src, int i, int j, int k)
{
    int n[3] = {G->nr, G->nt, G->np};
    int c[3] = {i, j, k};
    double del[3] = {G->dr, G->dt, G->dp};
    double out = 0.0, in = 0.0;
    for (int d = 0; d < 3; d++) {
        double A;
        if (c[d] < n[d] - 1) { /* + face */
            double a = face_velocity(G, T, xi, eta, d, i, j, k, &A);
            int q[3] = {i, j, k};
            q[d]++;
            out += A * fmax(a, 0.0) / del[d];
            in -= A * fmin(a, 0.0) * P[idx(G, q[0], q[1], q[2])] / del[d];
        }
        if (c[d] > 0) { /* - face, i.e. the + face of the - neighbour */
            int q[3] = {i, j, k};
            q[d]--;
            double a = face_velocity(G, T, xi, eta, d, q[0], q[1], q[2], &A);
            out -= A * fmin(a, 0.0) / del[d];
            in += A * fmax(a, 0.0) * P[idx(G, q[0], q[1], q[2])] / del[d];
        }
    }
    (void)S;
    if (out <= 1e-30) return 0.0;
    return (src + in) / out;
}

/* One adjoint sweep in ordering o over every node (R9); returns the largest |change|. */
static double adj_sweep(const geo *G, const source_factor *S, const double *T, const double *xi,
                        const double *eta, double *P, const double *JS, int o)
{
    int dr = (o & 4) ? -1 : 1, dt = (o & 2) ? -1 : 1, dp = (o & 1) ? -1 : 1;
    double err = 0.0;
    for (int a = 0; a < G->nr; a++)
        for (int bb = 0; bb < G->nt; bb++)
            for (int cc = 0; cc < G->np; cc++) {
                int i = swept(a, dr, 0, G->nr - 1);
                int j = swept(bb, dt, 0, G->nt - 1);
                int k = swept(cc, dp, 0, G->np - 1);
                if (is_fixed(S, i, j, k)) continue;
                long n = idx(G, i, j, k);
                double v = adj_update(G, S, T, xi, eta, P, JS[n], i, j, k);
                err = fmax(err, fabs(v - P[n]));
                P[n] = v;
            }
    return err;
}

/* J_c S_c at every node: R_m spread with trilinear weights over the node volume
 * J_c dr dt dp; the J_c cancels (R9). */
static double *point_sources(const geo *G, int n_rec, const or_point *rec, const double *R)
{
    long N = (long)G->nr * G->nt * G->np;
    double *JS = (double *)calloc((size_t)N, sizeof(double));
    for (int m = 0; m < n_rec; m++) {
        int b[3];
        double w[8];
        trilinear(G, rec[m], b, w);
        for (int c = 0; c < 8; c++)
            JS[idx(G, b[0] + ((c >> 2) & 1), b[1] + ((c >> 1) & 1), b[2] + (c & 1))] +=
                R[m] * w[c] / (G->dr * G->dt * G->dp);
    }
    return JS;
}

/* The fixed set only needs the source position; the adjoint does not use T0, so the factor
 * is built with unit slowness and isotropy. */
static source_factor adjoint_source(const geo *G, or_point src)
{
    long N = (long)G->nr * G->nt * G->np;
    double *ones = (double *)calloc((size_t)N, sizeof(double));
    double *zeros = (double *)calloc((size_t)N, sizeof(double));
    for (long q = 0; q < N; q++) ones[q] = 1.0;
    source_factor S = make_source(G, ones, zeros, zeros, src);
    free(ones);
    free(zeros);
    return S;
}

int or_adjoint(const or_grid *g, const double *T, const double *xi, const double *eta,
               or_point src, int n_rec, const or_point *rec, const double *R,
               double tol, int max_iter, double *P, int *conv, double *last_err)
{
    geo G = make_geo(g);
    long N = (long)G.nr * G.nt * G.np;
    source_factor S = adjoint_source(&G, src);
    double *JS = point_sources(&G, n_rec, rec, R);

    for (long q = 0; q < N; q++) P[q] = 0.0;
    int it = 0;
    double err = 0.0;
    *conv = 0;
    while (it < max_iter) {
        err = 0.0;
        for (int o = 0; o < 8; o++) err = fmax(err, adj_sweep(&G, &S, T, xi, eta, P, JS, o));
        it++;
        double pmax = 0.0;
        for (long q = 0; q < N; q++) pmax = fmax(pmax, fabs(P[q]));
        if (err <= tol * pmax) { *conv = 1; break; }
    }
    if (last_err) *last_err = err;
    free(JS);
    return it;
}

double or_fixed_set_inflow(const or_grid *g, const double *T, const double *xi,
                           const double *eta, or_point src, const double *P)
{
    geo G = make_geo(g);
    source_factor S = adjoint_source(&G, src);
    int n[3] = {G.nr, G.nt, G.np};
    double del[3] = {G.dr, G.dt, G.dp};
    double vol = G.dr * G.dt * G.dp, flux = 0.0;
    for (int i = 0; i < G.nr; i++)
        for (int j = 0; j < G.nt; j++)
            for (int k = 0; k < G.np; k++) {
                if (is_fixed(&S, i, j, k)) continue;
                int c[3] = {i, j, k};
                double Pc = P[idx(&G, i, j, k)];
                for (int d = 0; d < 3; d++) {
                    double A;
                    if (c[d] < n[d] - 1) {
                        int q[3] = {i, j, k};
                        q[d]++;
                        if (is_fixed(&S, q[0], q[1], q[2])) {
                            double a = face_velocity(&G, T, xi, eta, d, i, j, k, &A);
                            flux += A * fmax(a, 0.0) * Pc * vol / del[d];
                        }
                    }
                    if (c[d] > 0) {
                        int q[3] = {i, j, k};
                        q[d]--;
                        if (is_fixed(&S, q[0], q[1], q[2])) {
                            double a = face_velocity(&G, T, xi, eta, d, q[0], q[1], q[2], &A);
                            flux -= A * fmin(a, 0.0) * Pc * vol / del[d];
                        }
                    }
                }
            }
    return flux;
}

/* ---------------------------------------------------------------- kernels (Eqs. 6-8) */

void or_kernel_add(const or_grid *g, const double *s, const double *T, const double *P,
                   double *Ks, double *Kxi, double *Keta)
{
    geo G = make_geo(g);
    for (int i = 0; i < G.nr; i++)
        for (int j = 0; j < G.nt; j++)
            for (int k = 0; k < G.np; k++) {
                long n = idx(&G, i, j, k);
                double r = rad_of(&G, i), th = lat_of(&G, j);
                double gt = d_theta(&G, T, i, j, k) / h2_at(&G, r);
                double gp = d_phi(&G, T, i, j, k) / h3_at(&G, r, th);
                Ks[n] += P[n] * s[n] * s[n];
                Kxi[n] += P[n] * (gt * gt - gp * gp);
                Keta[n] += -2.0 * P[n] * gt * gp;
            }
}

void or_node_volumes(const or_grid *g, double *dV)
{
    geo G = make_geo(g);
    for (int i = 0; i < G.nr; i++)
        for (int j = 0; j < G.nt; j++)
            for (int k = 0; k < G.np; k++) {
                double r = rad_of(&G, i), th = lat_of(&G, j);
                double J = h2_at(&G, r) * h3_at(&G, r, th);
                dV[idx(&G, i, j, k)] = J * G.dr * G.dt * G.dp;
            }
}

/* ---------------------------------------------------------------- timing samples */

/* n_sweeps forward sweeps (orderings 0, 1, ...) with face extrapolation, from tau = 1: the
 * unit of work the CPU baseline times. */
void or_forward_sweeps(const or_grid *g, const double *s, const double *xi, const double *eta,
                       or_point src, int n_sweeps, double *tau)
{
    geo G = make_geo(g);
    source_factor S = make_source(&G, s, xi, eta, src);
    long N = (long)G.nr * G.nt * G.np;
    for (long n = 0; n < N; n++) tau[n] = 1.0;
    for (int q = 0; q < n_sweeps; q++) {
        sweep_lex(&G, &S, s, xi, eta, tau, q % 8, 0);
        extrapolate_faces(&G, &S, tau);
    }
}

/* n_sweeps adjoint sweeps from P = 0 (same unit of work for the adjoint). */
void or_adjoint_sweeps(const or_grid *g, const double *T, const double *xi, const double *eta,
                       or_point src, int n_rec, const or_point *rec, const double *R,
                       int n_sweeps, double *P)
{
    geo G = make_geo(g);
    long N = (long)G.nr * G.nt * G.np;
    source_factor S = adjoint_source(&G, src);
    double *JS = point_sources(&G, n_rec, rec, R);
    for (long q = 0; q < N; q++) P[q] = 0.0;
    for (int q = 0; q < n_sweeps; q++) adj_sweep(&G, &S, T, xi, eta, P, JS, q % 8);
    free(JS);
}

/* ---------------------------------------------------------------- teleseismic (R17) */

/* Slowness of the 1-D model at radius r: linear between the n_r samples s_r on
 * [r_min, r_max]. */
static double s_of_r(int n_r, double r_min, double dr, const double *s_r, double r)
{
    double f = (r - r_min) / dr;
    int i = (int)floor(f);
    if (i < 0) i = 0;
    if (i > n_r - 2) i = n_r - 2;
    double w = f - i;
    return (1.0 - w) * s_r[i] + w * s_r[i + 1];
}

/* The 2-D factored Godunov update at (i, j) of the (r, Delta) grid: R14 in two dimensions.
 * Physical gradient components (d/dr, d/(r dDelta)); the factor T0 = s_s L with L the chord
 * from the event at (r_s, 0) to (r, Delta), u = grad T0 / T0 = (r - r_s cos D, r_s sin D) / L^2. */
static double god2d_update(int n_r, int n_d, double r_min, double dr, double dd, double r_s,
                           double s_s, const double *s_r, const double *tau, int i, int j)
{
    double r = r_min + i * dr, D = j * dd;
    double L2 = r * r + r_s * r_s - 2.0 * r * r_s * cos(D);
    double L = sqrt(L2), T0 = s_s * L;
    double u[2] = {(r - r_s * cos(D)) / L2, r_s * sin(D) / L2};
    double e[2] = {1.0 / dr, 1.0 / (r * dd)};
    double lo[2] = {tau[(i - 1) * n_d + j], tau[i * n_d + (j > 0 ? j - 1 : 1)]};
    double hi[2] = {tau[(i + 1) * n_d + j], tau[i * n_d + j + 1]};
    double a[2], b[2], sg[2];
    for (int d = 0; d < 2; d++) {
        double tlo = lo[d] * (1.0 - u[d] / e[d]), thi = hi[d] * (1.0 + u[d] / e[d]);
        sg[d] = tlo <= thi ? 1.0 : -1.0;
        double nb = tlo <= thi ? lo[d] : hi[d];
        a[d] = u[d] + sg[d] * e[d];
        b[d] = sg[d] * e[d] * nb;
    }
    double rhs = s_of_r(n_r, r_min, dr, s_r, r) / T0;
    double best = -1.0;
    for (int mask = 1; mask < 4; mask++) {
        double A = 0.0, B = 0.0, C = -rhs * rhs;
        for (int d = 0; d < 2; d++)
            if (mask >> d & 1) { A += a[d] * a[d]; B += a[d] * b[d]; C += b[d] * b[d]; }
        double disc = B * B - A * C;
        if (!(A > 0.0) || disc < 0.0) continue;
        double t = (B + sqrt(disc)) / A;
        int ok = 1;
        for (int d = 0; d < 2; d++)
            if ((mask >> d & 1) && sg[d] * (a[d] * t - b[d]) < 0.0) ok = 0;
        if (ok && (best < 0.0 || t < best)) best = t;
    }
    return best < 0.0 ? tau[i * n_d + j] : best;
}

/* 2-D traveltimes from an event at radius r_s (R17): T [n_r][n_d] on r in [r_min, r_max],
 * Delta in [0, d_max] (radians), 1-D slowness s_r [n_r]. Returns iterations; *conv = 1 when
 * the largest change of an iteration fell below tol. */
int or_tele2d(int n_r, int n_d, double r_min, double r_max, double d_max, const double *s_r,
              double r_s, double tol, int max_iter, double *T, int *conv)
{
    double dr = (r_max - r_min) / (n_r - 1), dd = d_max / (n_d - 1);
    double s_s = s_of_r(n_r, r_min, dr, s_r, r_s);
    int is = (int)floor((r_s - r_min) / dr + 0.5);
    if (is < 0) is = 0;
    if (is > n_r - 1) is = n_r - 1;
    double *tau = (double *)malloc(sizeof(double) * (size_t)n_r * n_d);
    if (!tau) return -1;
    for (long q = 0; q < (long)n_r * n_d; q++) tau[q] = 1.0;
    int it = 0;
    *conv = 0;
    while (it < max_iter) {
        double err = 0.0;
        for (int o = 0; o < 4; o++) {
            int di = (o & 2) ? -1 : 1, dj = (o & 1) ? -1 : 1;
            for (int a = 0; a < n_r - 2; a++)
                for (int b = 0; b < n_d - 1; b++) {
                    int i = di > 0 ? 1 + a : n_r - 2 - a;
                    int j = dj > 0 ? b : n_d - 2 - b;
                    if (abs(i - is) <= 1 && j <= 1) continue;       /* fixed set */
                    double v = god2d_update(n_r, n_d, r_min, dr, dd, r_s, s_s, s_r, tau, i, j);
                    err = fmax(err, fabs(v - tau[i * n_d + j]));
                    tau[i * n_d + j] = v;
                }
            /* faces r (low, high), then Delta = d_max (R6); the axis Delta = 0 is a mirror */
            for (int j = 0; j < n_d; j++) {
                if (!(abs(0 - is) <= 1 && j <= 1))
                    tau[j] = fmax(2.0 * tau[n_d + j] - tau[2 * n_d + j], tau[2 * n_d + j]);
                if (!(abs(n_r - 1 - is) <= 1 && j <= 1))
                    tau[(n_r - 1) * n_d + j] = fmax(2.0 * tau[(n_r - 2) * n_d + j] - tau[(n_r - 3) * n_d + j],
                                                    tau[(n_r - 3) * n_d + j]);
            }
            for (int i = 0; i < n_r; i++)
                tau[i * n_d + n_d - 1] = fmax(2.0 * tau[i * n_d + n_d - 2] - tau[i * n_d + n_d - 3],
                                              tau[i * n_d + n_d - 3]);
        }
        it++;
        if (err < tol) { *conv = 1; break; }
    }
    for (int i = 0; i < n_r; i++)
        for (int j = 0; j < n_d; j++) {
            double r = r_min + i * dr, D = j * dd;
            double L = sqrt(fmax(r * r + r_s * r_s - 2.0 * r * r_s * cos(D), 0.0));
            T[i * n_d + j] = s_s * L * tau[i * n_d + j];
        }
    free(tau);
    return it;
}

/* R4's Lax-Friedrichs update of T itself (T0 = 1, no factor) at an interior node. */
static double lf_plain_update(const geo *G, const double *s, const double *xi, const double *eta,
                              const double *T, int i, int j, int k)
{
    long c = idx(G, i, j, k);
    double r = rad_of(G, i), th = lat_of(G, j);
    double h[3] = {1.0, h2_at(G, r), h3_at(G, r, th)};
    double del[3] = {G->dr, G->dt, G->dp};
    double tp[3], tm[3];
    tp[0] = T[idx(G, i + 1, j, k)]; tm[0] = T[idx(G, i - 1, j, k)];
    tp[1] = T[idx(G, i, j + 1, k)]; tm[1] = T[idx(G, i, j - 1, k)];
    tp[2] = T[idx(G, i, j, k + 1)]; tm[2] = T[idx(G, i, j, k - 1)];
    double p[3];
    for (int d = 0; d < 3; d++) p[d] = (tp[d] - tm[d]) / (2.0 * del[d]) / h[d];
    double M[3][3];
    aniso_M(xi[c], eta[c], M);
    double q = 0.0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) q += p[a] * M[a][b] * p[b];
    double sigma[3] = {1.0, sqrt(1.0 - 2.0 * xi[c]) / h[1], sqrt(1.0 + 2.0 * xi[c]) / h[2]};
    double num = s[c] - sqrt(q), den = 0.0;
    for (int d = 0; d < 3; d++) {
        num += sigma[d] * (tp[d] + tm[d]) / (2.0 * del[d]);
        den += sigma[d] / del[d];
    }
    return num / den;
}

/* The 3-D solve of a teleseismic event (R17): T [N] holds the start on entry, its boundary
 * nodes (the six faces) being the Dirichlet data, which are kept; interior nodes are swept
 * in the 8 orderings of R5 until the largest change of an iteration is below tol. */
int or_forward_tele(const or_grid *g, const double *s, const double *xi, const double *eta,
                    double tol, int max_iter, double *T, int *conv, double *last_err)
{
    geo G = make_geo(g);
    int it = 0;
    double err = 0.0;
    *conv = 0;
    while (it < max_iter) {
        err = 0.0;
        for (int o = 0; o < 8; o++) {
            int dr = (o & 4) ? -1 : 1, dt = (o & 2) ? -1 : 1, dp = (o & 1) ? -1 : 1;
            for (int a = 0; a < G.nr - 2; a++)
                for (int b = 0; b < G.nt - 2; b++)
                    for (int c = 0; c < G.np - 2; c++) {
                        int i = swept(a, dr, 1, G.nr - 2);
                        int j = swept(b, dt, 1, G.nt - 2);
                        int k = swept(c, dp, 1, G.np - 2);
                        long n = idx(&G, i, j, k);
                        double v = lf_plain_update(&G, s, xi, eta, T, i, j, k);
                        err = fmax(err, fabs(v - T[n]));
                        T[n] = v;
                    }
        }
        it++;
        if (err < tol) { *conv = 1; break; }
    }
    if (last_err) *last_err = err;
    return it;
}
