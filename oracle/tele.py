"""FP64 oracle of teleseismic boundary times (reading R17 of tt_oracle.c; test
infrastructure only: the test suite, the smoke check and the benchmark's CPU-baseline leg).

An event outside the region (Eq. "4"'s boundary condition for teleseismic events): a 2-D
eikonal solve in a 1-D global model s(r) from the event gives T(r, Delta), Delta the
epicentral angle; the region's faces take its bilinear interpolation at their (r, Delta);
the 3-D solve then runs on T itself with those faces held fixed.
"""
import ctypes as C

import numpy as np

from . import _f, lib, make_grid

DEG = np.pi / 180.0


def _lib():
    L = lib()
    L.or_tele2d.restype = C.c_int
    L.or_forward_tele.restype = C.c_int
    return L


def tele2d(r_min, r_max, n_r, d_max_deg, n_d, s_r, r_s, tol=1e-10, max_iter=500):
    """T [n_r][n_d] on r in [r_min, r_max] (km) and Delta in [0, d_max_deg] from an event at
    radius r_s on the axis Delta = 0; s_r [n_r] the slowness at the grid radii. Returns
    (T, iterations, converged)."""
    s_r, ps = _f(s_r)
    T = np.zeros((n_r, n_d))
    conv = C.c_int(0)
    it = _lib().or_tele2d(C.c_int(n_r), C.c_int(n_d), C.c_double(r_min), C.c_double(r_max),
                          C.c_double(d_max_deg * DEG), ps, C.c_double(r_s), C.c_double(tol),
                          C.c_int(max_iter), T.ctypes.data_as(C.POINTER(C.c_double)),
                          C.byref(conv))
    return T, it, bool(conv.value)


def epicentral_angle(lat, lon, lat_s, lon_s):
    """Great-circle angle (radians) between points given in degrees (arrays broadcast)."""
    a, b, la, lb = lat * DEG, lat_s * DEG, lon * DEG, lon_s * DEG
    c = np.sin(a) * np.sin(b) + np.cos(a) * np.cos(b) * np.cos(la - lb)
    return np.arccos(np.clip(c, -1.0, 1.0))


def interp2d(T2, r_min, r_max, d_max_deg, r, D):
    """Bilinear interpolation of T2 [n_r][n_d] at radii r (km) and angles D (radians)."""
    n_r, n_d = T2.shape
    fr = (r - r_min) / (r_max - r_min) * (n_r - 1)
    fd = D / (d_max_deg * DEG) * (n_d - 1)
    i = np.clip(np.floor(fr).astype(int), 0, n_r - 2)
    j = np.clip(np.floor(fd).astype(int), 0, n_d - 2)
    u, v = fr - i, fd - j
    return ((1 - u) * (1 - v) * T2[i, j] + u * (1 - v) * T2[i + 1, j] +
            (1 - u) * v * T2[i, j + 1] + u * v * T2[i + 1, j + 1])


def region_times(g, T2, r_min, r_max, d_max_deg, lat_s, lon_s):
    """The 2-D times at every node of the region (spherical grid g): the faces' Dirichlet
    data, and the interior's starting values."""
    get = (lambda k: g[k]) if isinstance(g, dict) else (lambda k: getattr(g, k))
    n = (get("n_r"), get("n_t"), get("n_p"))
    depth = np.linspace(get("depth_max_km"), get("depth_min_km"), n[0])
    r = get("earth_radius_km") - depth
    lat = np.linspace(get("lat_min_deg"), get("lat_max_deg"), n[1])
    lon = np.linspace(get("lon_min_deg"), get("lon_max_deg"), n[2])
    R, LA, LO = np.meshgrid(r, lat, lon, indexing="ij")
    return interp2d(T2, r_min, r_max, d_max_deg, R, epicentral_angle(LA, LO, lat_s, lon_s))


def forward_tele(g, s, xi, eta, T_start, tol=1e-8, max_iter=500):
    """The 3-D solve with the faces of T_start held fixed. Returns (T, iterations, converged)."""
    G = make_grid(g)
    s, ps = _f(s); xi, px = _f(xi); eta, pe = _f(eta)
    T = np.ascontiguousarray(T_start, dtype=np.float64).copy()
    conv = C.c_int(0); err = C.c_double(0)
    it = _lib().or_forward_tele(C.byref(G), ps, px, pe, C.c_double(tol), C.c_int(max_iter),
                                T.ctypes.data_as(C.POINTER(C.c_double)), C.byref(conv),
                                C.byref(err))
    return T, it, bool(conv.value)
