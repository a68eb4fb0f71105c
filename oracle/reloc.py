"""FP64 oracle of the earthquake-location and origin-time kernels (test infrastructure only).

Eq. 10 and Appendix B (Eqs. B1-B11). By reciprocity the time from source n to receiver m is
the time Gamma_m(x_{s,n}) of a wavefront started at receiver m, so with origin time tau_n the
synthetic arrival is Gamma_m(x_{s,n}) + tau_n. Every misfit of Eqs. 2-4 then depends on
x_{s,n} and tau_n only through these arrivals, and with R_{n,m} = dchi / dT_n(x_{r,m}) (the
adjoint sources of Eqs. A2-A4):
  K_x,n   = sum_m R_{n,m} grad Gamma_m(x_{s,n})     (Eqs. B4-B7)
  K_tau,n = sum_m R_{n,m}                           (Eqs. B8-B11; the common-source terms
                                                     cancel in the sum, Eq. B10)
Reading R15 (the paper does not say how Gamma and its gradient are evaluated at a point):
  Gamma_m(x) is the trilinear interpolant of the nodal field in index space (R8), and
  grad Gamma_m(x) is the gradient of that same interpolant in physical components
  (d/dr, d/(r dtheta), d/(r cos(theta) dphi)) at the point's own r and theta. K_x is then the
  exact derivative of the discrete misfit with respect to the source position.
Fields are numpy float64 arrays; points are (depth_km, lat_deg, lon_deg).
"""
import numpy as np

from . import misfit as _misfit
from .cr import misfit_cr

DEG = np.pi / 180.0


def _geometry(g):
    get = (lambda k: g[k]) if isinstance(g, dict) else (lambda k: getattr(g, k))
    n = (get("n_r"), get("n_t"), get("n_p"))
    re = get("earth_radius_km")
    r0 = re - get("depth_max_km")
    dr = (get("depth_max_km") - get("depth_min_km")) / (n[0] - 1)
    t0 = get("lat_min_deg") * DEG
    dt = (get("lat_max_deg") - get("lat_min_deg")) * DEG / (n[1] - 1)
    p0 = get("lon_min_deg") * DEG
    dp = (get("lon_max_deg") - get("lon_min_deg")) * DEG / (n[2] - 1)
    return n, re, (r0, t0, p0), (dr, dt, dp), bool(get("flat"))


def field_at(g, F, p):
    """Value and physical gradient at point p of the trilinear interpolant of the nodal field
    F [n_r][n_t][n_p] (R8, R15). The cell is the one whose lower corner is floor of the
    fractional index, clamped to the grid; u in [0, 1] is the position within it."""
    n, re, org, d, flat = _geometry(g)
    depth, lat, lon = p
    r = re - depth
    th = lat * DEG
    f = ((r - org[0]) / d[0], (th - org[1]) / d[1], (lon * DEG - org[2]) / d[2])
    base, u = [], []
    for a in range(3):
        i0 = min(max(int(np.floor(f[a])), 0), n[a] - 2)
        base.append(i0)
        u.append(f[a] - i0)
    c = F[base[0]:base[0] + 2, base[1]:base[1] + 2, base[2]:base[2] + 2]
    wr = np.array([1.0 - u[0], u[0]])
    wt = np.array([1.0 - u[1], u[1]])
    wp = np.array([1.0 - u[2], u[2]])
    dw = np.array([-1.0, 1.0])          # d/du of (1 - u, u)
    val = np.einsum("i,j,k,ijk->", wr, wt, wp, c)
    d_i = np.einsum("i,j,k,ijk->", dw, wt, wp, c)     # d/d(fractional index), per axis
    d_j = np.einsum("i,j,k,ijk->", wr, dw, wp, c)
    d_k = np.einsum("i,j,k,ijk->", wr, wt, dw, c)
    h2 = re if flat else r
    h3 = re if flat else r * np.cos(th)
    grad = np.array([d_i / d[0], d_j / (d[1] * h2), d_k / (d[2] * h3)])
    return val, grad


def table(g, fields, pts):
    """fields: list of M nodal fields (Gamma_m, one per receiver); pts: [n_pts] points.
    Returns val [n_pts][M] and grad [n_pts][M][3]."""
    val = np.zeros((len(pts), len(fields)))
    grad = np.zeros((len(pts), len(fields), 3))
    for q, p in enumerate(pts):
        for m, F in enumerate(fields):
            val[q, m], grad[q, m] = field_at(g, F, p)
    return val, grad


def misfit_table(Tr, abs_recs, cs_recs, alpha=1.0, beta=1.0, cr=None):
    """Misfit and adjoint sources from a table of arrivals Tr [n_src][n_rec] (Eqs. 2-4,
    A2-A4). abs_recs[n] = (rec, tobs, w) arrays of source n's absolute records; cs_recs[n] =
    (m, i, dtobs, w) of its common-source pairs; cr = (Tobs, W, gamma) as in oracle.cr.
    Returns (chi_t, chi_cs, chi_cr, R)."""
    ns, nr = Tr.shape
    R = np.zeros((ns, nr))
    chi_t = chi_cs = chi_cr = 0.0
    for n in range(ns):
        ar, at, aw = abs_recs[n]
        cm, ci, cd, cw = cs_recs[n]
        ct, cc, Rn = _misfit(Tr[n], ar, at, aw, cm, ci, cd, cw, alpha, beta)
        chi_t += ct
        chi_cs += cc
        R[n] += Rn
    if cr is not None:
        Tobs, W, gamma = cr
        c, _, Rc = misfit_cr(Tr, Tobs, W, gamma)
        chi_cr = c
        R += Rc
    return chi_t, chi_cs, chi_cr, R


def kernels(R, grad):
    """K_x [n_src][3] = sum_m R[n, m] grad[n, m] (Eqs. B5-B7) and K_tau [n_src] =
    sum_m R[n, m] (Eqs. B9-B11), each sum over m in increasing order."""
    ns, nr = R.shape
    Kx = np.zeros((ns, 3))
    Kt = np.zeros(ns)
    for n in range(ns):
        for m in range(nr):
            Kx[n] += R[n, m] * grad[n, m]
            Kt[n] += R[n, m]
    return Kx, Kt


def update(g, pts, tau, Kx, Kt, step_km, step_s):
    """One gradient-descent step of the event locations and origin times (reading R15b: the
    paper names gradient descent and gives no step rule). Each event moves by
    -step_km K_x,n / max_n |K_x,n| km in physical components (up, north, east): depth by
    +step_km K_r / max, latitude by -step_km K_theta / (max h2) radians, longitude by
    -step_km K_phi / (max h3) radians, with h2 = r, h3 = r cos(theta) at the event (R_E for
    both in flat geometry); then it is clamped to the grid. Origin times move by
    -step_s K_tau,n / max_n |K_tau,n|. A zero maximum moves nothing. Returns new copies."""
    n, re, org, d, flat = _geometry(g)
    get = (lambda k: g[k]) if isinstance(g, dict) else (lambda k: getattr(g, k))
    pts = np.array(pts, dtype=np.float64)
    tau = np.array(tau, dtype=np.float64)
    mx = max(float(np.sqrt((K ** 2).sum())) for K in Kx)
    mt = float(np.abs(Kt).max())
    for q in range(len(pts)):
        if mx > 0:
            dx = -step_km * Kx[q] / mx
            r = re - pts[q, 0]
            th = pts[q, 1] * DEG
            h2 = re if flat else r
            h3 = re if flat else r * np.cos(th)
            pts[q, 0] -= dx[0]
            pts[q, 1] += dx[1] / h2 / DEG
            pts[q, 2] += dx[2] / h3 / DEG
            pts[q, 0] = min(max(pts[q, 0], get("depth_min_km")), get("depth_max_km"))
            pts[q, 1] = min(max(pts[q, 1], get("lat_min_deg")), get("lat_max_deg"))
            pts[q, 2] = min(max(pts[q, 2], get("lon_min_deg")), get("lon_max_deg"))
        if mt > 0:
            tau[q] -= step_s * Kt[q] / mt
    return pts, tau
