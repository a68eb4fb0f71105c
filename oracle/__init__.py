"""Python access to the FP64 CPU oracle (test infrastructure only).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg use this module.
The product package never imports it. Fields are numpy float64 arrays of shape
(n_r, n_t, n_p); one call handles one source. See tt_oracle.c for the equations each
function follows.
"""
import ctypes as C

import numpy as np

from . import build as _build


class Grid(C.Structure):
    _fields_ = [("n_r", C.c_int), ("n_t", C.c_int), ("n_p", C.c_int),
                ("depth_min_km", C.c_double), ("depth_max_km", C.c_double),
                ("lat_min_deg", C.c_double), ("lat_max_deg", C.c_double),
                ("lon_min_deg", C.c_double), ("lon_max_deg", C.c_double),
                ("earth_radius_km", C.c_double), ("flat", C.c_int)]


class Point(C.Structure):
    _fields_ = [("depth_km", C.c_double), ("lat_deg", C.c_double), ("lon_deg", C.c_double)]


_lib = None
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        L.or_forward.restype = C.c_int
        L.or_forward_hyperplane.restype = C.c_int
        L.or_forward_godunov.restype = C.c_int
        L.or_forward_godunov_aniso.restype = C.c_int
        L.or_adjoint.restype = C.c_int
        L.or_fixed_set_inflow.restype = C.c_double
        _lib = L
    return _lib


def make_grid(g):
    """g: dict or object with the grid description keys (see tt_inputs.GridSpec)."""
    get = (lambda k: g[k]) if isinstance(g, dict) else (lambda k: getattr(g, k))
    return Grid(get("n_r"), get("n_t"), get("n_p"), get("depth_min_km"), get("depth_max_km"),
                get("lat_min_deg"), get("lat_max_deg"), get("lon_min_deg"), get("lon_max_deg"),
                get("earth_radius_km"), int(get("flat")))


def _f(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


def _points(pts):
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    arr = (Point * max(len(pts), 1))()
    for q, p in enumerate(pts):
        arr[q] = Point(*p)
    return arr, len(pts)


def T0(g, s, xi, eta, src):
    G = make_grid(g)
    shape = (G.n_r, G.n_t, G.n_p)
    s, ps = _f(s); xi, px = _f(xi); eta, pe = _f(eta)
    T0 = np.zeros(shape); p0 = np.zeros(shape + (3,))
    lib().or_T0(C.byref(G), ps, px, pe, Point(*src), T0.ctypes.data_as(_dp), p0.ctypes.data_as(_dp))
    return T0, p0


def forward(g, s, xi, eta, src, tol=1e-8, max_iter=500, tau_init=None, hyperplane=False,
            scheme="lf"):
    """Returns (tau, T, iterations, converged, last_err). scheme: "lf" (Lax-Friedrichs, R4),
    "godunov" (R14; isotropic models only: xi = eta = 0) or "godunov_aniso" (R16; any
    model)."""
    G = make_grid(g)
    shape = (G.n_r, G.n_t, G.n_p)
    s, ps = _f(s); xi, px = _f(xi); eta, pe = _f(eta)
    tau = np.zeros(shape); T = np.zeros(shape)
    conv = C.c_int(0); err = C.c_double(0)
    init = None
    if tau_init is not None:
        init, pinit = _f(tau_init)
    if scheme == "godunov":
        assert not hyperplane and not xi.any() and not eta.any(), "Godunov: isotropic models"
        fn = lib().or_forward_godunov
    elif scheme == "godunov_aniso":
        assert not hyperplane
        fn = lib().or_forward_godunov_aniso
    else:
        fn = lib().or_forward_hyperplane if hyperplane else lib().or_forward
    it = fn(C.byref(G), ps, px, pe, Point(*src), C.c_double(tol), C.c_int(max_iter),
            pinit if init is not None else None, tau.ctypes.data_as(_dp), T.ctypes.data_as(_dp),
            C.byref(conv), C.byref(err))
    return tau, T, it, bool(conv.value), err.value


def receiver_times(g, T, rec):
    G = make_grid(g)
    T, pT = _f(T)
    arr, n = _points(rec)
    Tr = np.zeros(n)
    lib().or_receiver_times(C.byref(G), pT, C.c_int(n), arr, Tr.ctypes.data_as(_dp))
    return Tr


def misfit(Tr, abs_rec, abs_tobs, abs_w, cs_m, cs_i, cs_dtobs, cs_w, alpha=1.0, beta=1.0):
    """Returns (chi_t, chi_cs, R)."""
    Tr, pTr = _f(Tr)
    ar, par = _i(abs_rec); at, pat = _f(abs_tobs); aw, paw = _f(abs_w)
    cm, pcm = _i(cs_m); ci, pci = _i(cs_i); cd, pcd = _f(cs_dtobs); cw, pcw = _f(cs_w)
    chi = np.zeros(2); R = np.zeros(len(Tr))
    lib().or_misfit(C.c_int(len(Tr)), pTr, C.c_int(len(ar)), par, pat, paw, C.c_int(len(cm)),
                    pcm, pci, pcd, pcw, C.c_double(alpha), C.c_double(beta),
                    chi.ctypes.data_as(_dp), R.ctypes.data_as(_dp))
    return chi[0], chi[1], R


def adjoint(g, T, xi, eta, src, rec, R, tol=1e-8, max_iter=500):
    """Returns (P, iterations, converged, last_err)."""
    G = make_grid(g)
    shape = (G.n_r, G.n_t, G.n_p)
    T, pT = _f(T); xi, px = _f(xi); eta, pe = _f(eta)
    arr, n = _points(rec)
    R, pR = _f(R)
    P = np.zeros(shape)
    conv = C.c_int(0); err = C.c_double(0)
    it = lib().or_adjoint(C.byref(G), pT, px, pe, Point(*src), C.c_int(n), arr, pR,
                          C.c_double(tol), C.c_int(max_iter), P.ctypes.data_as(_dp),
                          C.byref(conv), C.byref(err))
    return P, it, bool(conv.value), err.value


def kernel_add(g, s, T, P, Ks, Kxi, Keta):
    """Adds one source's Eqs. 6-8 contribution into the float64 arrays Ks, Kxi, Keta."""
    G = make_grid(g)
    s, ps = _f(s); T, pT = _f(T); P, pP = _f(P)
    for a in (Ks, Kxi, Keta):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().or_kernel_add(C.byref(G), ps, pT, pP, Ks.ctypes.data_as(_dp),
                        Kxi.ctypes.data_as(_dp), Keta.ctypes.data_as(_dp))


def fixed_set_inflow(g, T, xi, eta, src, P):
    G = make_grid(g)
    T, pT = _f(T); xi, px = _f(xi); eta, pe = _f(eta); P, pP = _f(P)
    return lib().or_fixed_set_inflow(C.byref(G), pT, px, pe, Point(*src), pP)


def node_volumes(g):
    G = make_grid(g)
    dV = np.zeros((G.n_r, G.n_t, G.n_p))
    lib().or_node_volumes(C.byref(G), dV.ctypes.data_as(_dp))
    return dV


def solve_source(g, s, xi, eta, src, rec, data, alpha=1.0, beta=1.0, tol_fwd=1e-8,
                 tol_adj=1e-8, max_iter=500):
    """One whole source solve: forward, misfit, adjoint. data: dict with abs_rec, abs_tobs,
    abs_w, cs_m, cs_i, cs_dtobs, cs_w (receiver indices into rec). Returns a dict."""
    tau, T, itf, cf, _ = forward(g, s, xi, eta, src, tol_fwd, max_iter)
    Tr = receiver_times(g, T, rec)
    chi_t, chi_cs, R = misfit(Tr, data["abs_rec"], data["abs_tobs"], data["abs_w"],
                              data["cs_m"], data["cs_i"], data["cs_dtobs"], data["cs_w"],
                              alpha, beta)
    P, ita, ca, _ = adjoint(g, T, xi, eta, src, rec, R, tol_adj, max_iter)
    return dict(tau=tau, T=T, Tr=Tr, chi_t=chi_t, chi_cs=chi_cs, R=R, P=P, iters_fwd=itf,
                iters_adj=ita, conv_fwd=cf, conv_adj=ca)


def forward_sweeps(g, s, xi, eta, src, n_sweeps):
    """n_sweeps forward sweeps from tau = 1 (CPU-baseline timing unit). Returns tau."""
    G = make_grid(g)
    s, ps = _f(s); xi, px = _f(xi); eta, pe = _f(eta)
    tau = np.zeros((G.n_r, G.n_t, G.n_p))
    lib().or_forward_sweeps(C.byref(G), ps, px, pe, Point(*src), C.c_int(n_sweeps),
                            tau.ctypes.data_as(_dp))
    return tau


def adjoint_sweeps(g, T, xi, eta, src, rec, R, n_sweeps):
    """n_sweeps adjoint sweeps from P = 0 (CPU-baseline timing unit). Returns P."""
    G = make_grid(g)
    T, pT = _f(T); xi, px = _f(xi); eta, pe = _f(eta)
    arr, n = _points(rec)
    R, pR = _f(R)
    P = np.zeros((G.n_r, G.n_t, G.n_p))
    lib().or_adjoint_sweeps(C.byref(G), pT, px, pe, Point(*src), C.c_int(n), arr, pR,
                            C.c_int(n_sweeps), P.ctypes.data_as(_dp))
    return P
