"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed-form traveltimes,
the paper's stated order of accuracy, exact discrete invariants (hyperplane independence,
conservation), brute-force evaluation of Eqs. 2-3, and analytic derivatives of the misfit.
"""
import json
import os

import numpy as np
import pytest

import tt_inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def _cart(grid, pts):
    """Cartesian position (km) of (depth, lat, lon) rows, written out independently."""
    pts = np.atleast_2d(pts)
    r = grid.earth_radius_km - pts[..., 0]
    if grid.flat:
        return np.stack([r, grid.earth_radius_km * np.deg2rad(pts[..., 1]),
                         grid.earth_radius_km * np.deg2rad(pts[..., 2])], -1)
    th, ph = np.deg2rad(pts[..., 1]), np.deg2rad(pts[..., 2])
    return np.stack([r * np.cos(th) * np.cos(ph), r * np.cos(th) * np.sin(ph), r * np.sin(th)], -1)


def _node_points(grid):
    depth, lat, lon = grid.axes()
    D, LA, LO = np.meshgrid(depth, lat, lon, indexing="ij")
    return np.stack([D, LA, LO], -1)


# ----------------------------------------------------------------------------- forward

def test_homogeneous_isotropic_is_slowness_times_chord(oracle):
    """Homogeneous isotropic medium: T = s * |x - x_s| exactly (Eq. "4" with M = I), on the
    41^3 spherical grid with the source at the surface centre."""
    w = I.homogeneous_41()
    g = w.grid
    tau, T, it, conv, err = oracle.forward(g.as_dict(), w.s, w.xi, w.eta, w.src[0], tol=1e-7)
    X = _cart(g, _node_points(g))
    Xs = _cart(g, w.src[0])[0]
    exact = np.linalg.norm(X - Xs, axis=-1) / 6.0
    assert conv and it == 1
    assert np.max(np.abs(T - exact)) <= 1e-12 * np.max(exact)


@pytest.mark.parametrize("xi0,eta0", [(0.03, -0.02), (-0.04, 0.01), (0.0, 0.045)])
def test_homogeneous_anisotropic_flat_is_elliptical(oracle, xi0, eta0):
    """Homogeneous anisotropic medium in the flat test geometry: the solution of
    grad T^T M grad T = s^2 is T = s sqrt(D^T M^-1 D) (elliptical traveltime)."""
    g = I.GridSpec(17, 19, 15, 0.0, 16.0, 0.0, 0.15, 0.0, 0.13, flat=1)
    s0 = 1 / 5.5
    s = np.full(g.shape, s0)
    xi, eta = np.full(g.shape, xi0), np.full(g.shape, eta0)
    src = np.array([9.0, 0.07, 0.05])
    tau, T, it, conv, _ = oracle.forward(g.as_dict(), s, xi, eta, src, tol=1e-10)
    M = np.array([[1, 0, 0], [0, 1 - 2 * xi0, 2 * eta0], [0, 2 * eta0, 1 + 2 * xi0]])
    D = _cart(g, _node_points(g)) - _cart(g, src)[0]
    exact = s0 * np.sqrt(np.einsum("...a,ab,...b->...", D, np.linalg.inv(M), D))
    assert conv
    assert np.max(np.abs(T - exact)) <= 1e-12 * np.max(exact)


def test_spherical_anisotropic_stays_near_factor(oracle):
    """In spherical coordinates a homogeneous anisotropic medium is not exactly elliptical
    (the local frame rotates across the grid); the correction tau must stay small."""
    g = I.GridSpec(21, 21, 21, 0.0, 20.0, 0.0, 0.2, 0.0, 0.2)
    s = np.full(g.shape, 1 / 6.0)
    tau, T, it, conv, _ = oracle.forward(g.as_dict(), s, np.full(g.shape, 0.03),
                                         np.full(g.shape, 0.02), [10.0, 0.1, 0.1], tol=1e-10)
    assert conv and np.max(np.abs(tau - 1)) < 1e-3


def _linear_gradient_errors(oracle, n):
    """Velocity linear in a Cartesian direction, v = v0 + G.(x - x_s): the exact traveltime
    is arccosh(1 + |G|^2 |x - x_s|^2 / (2 v(x) v(x_s))) / |G| in any coordinates."""
    g = I.GridSpec(n, n, n, 0.0, 40.0, 0.0, 0.4, 0.0, 0.4)
    X = _cart(g, _node_points(g))
    src = np.array([20.0, 0.2, 0.2])
    Xs = _cart(g, src)[0]
    Gv = -0.05 * Xs / np.linalg.norm(Xs)
    v = 6.0 + (X - Xs) @ Gv
    z = np.zeros(g.shape)
    _, T, _, conv, _ = oracle.forward(g.as_dict(), 1.0 / v, z, z, src, tol=1e-10, max_iter=1000)
    Gn = np.linalg.norm(Gv)
    exact = np.arccosh(1 + Gn ** 2 * np.sum((X - Xs) ** 2, -1) / (2 * v * 6.0)) / Gn
    assert conv
    e = np.abs(T - exact)
    return e.mean(), e.max()


def test_linear_gradient_first_order(oracle):
    """The factored sweep is first-order accurate (Sec. 3.1, Fig. 2): halving the spacing
    at least roughly halves the error. The paper's own figures (golden fixture) imply an
    observed order of log(0.0517/0.0096)/log(8) = 0.81; the oracle must not do worse."""
    gold = json.load(open(os.path.join(HERE, "golden", "fig2_first_order.json")))
    paper_order = (np.log(gold["l1_error_s"][0] / gold["l1_error_s"][1])
                   / np.log(gold["h_km"][0] / gold["h_km"][1]))
    errs = [_linear_gradient_errors(oracle, n) for n in (11, 21, 41)]
    for (m0, x0), (m1, x1) in zip(errs[:-1], errs[1:]):
        assert np.log2(m0 / m1) >= paper_order - 0.05
        assert np.log2(x0 / x1) >= 0.8
    # same order of magnitude as the paper's L1 errors at comparable spacings (1-4 km)
    assert errs[-1][0] < 0.01


def test_hyperplane_order_is_bitwise_identical(oracle):
    """Nodes on one hyperplane a+b+c = L never neighbour each other (Sec. 3.4), so visiting
    the sweep plane by plane gives exactly the lexicographic Gauss-Seidel result."""
    w = I.small_case(5, shape=(9, 11, 13), n_src=1)
    args = (w.grid.as_dict(), w.s, w.xi, w.eta, w.src[0], 1e-10, 200)
    a = oracle.forward(*args)
    b = oracle.forward(*args, hyperplane=True)
    assert a[2] == b[2]
    assert np.array_equal(a[0], b[0])


def test_any_initial_tau_reaches_same_fixed_point(oracle):
    """Fast sweeping converges from any bounded start (Sec. 3.1)."""
    w = I.small_case(7, shape=(13, 13, 13), n_src=1)
    g = w.grid.as_dict()
    rng = np.random.default_rng(7)
    a = oracle.forward(g, w.s, w.xi, w.eta, w.src[0], tol=1e-12, max_iter=2000)
    init = 1.0 + 0.3 * rng.random(w.grid.shape)
    b = oracle.forward(g, w.s, w.xi, w.eta, w.src[0], tol=1e-12, max_iter=2000, tau_init=init)
    assert a[3] and b[3]
    assert np.max(np.abs(a[0] - b[0])) < 1e-9


# ----------------------------------------------------------------------------- misfit

def test_misfit_matches_ordered_double_sum():
    """Eq. 2 and Eq. 3 written as the paper's ordered sums (symmetric weights w/2 for each
    unordered pair), R from a central difference of chi (exact for a quadratic)."""
    import oracle as O
    rng = np.random.default_rng(11)
    n = 7
    Tr = rng.uniform(2, 9, n)
    abs_rec = np.array([0, 2, 3, 5, 6]); abs_tobs = Tr[abs_rec] + rng.normal(0, 0.1, 5)
    abs_w = rng.uniform(0.5, 2, 5)
    pairs = [(0, 2), (3, 5), (6, 0), (2, 5)]
    cs_m = np.array([p[0] for p in pairs]); cs_i = np.array([p[1] for p in pairs])
    cs_dt = rng.normal(0, 1, len(pairs)); cs_w = rng.uniform(0.5, 2, len(pairs))
    alpha, beta = 0.7, 1.3

    def chi_paper(T):
        ct = sum(abs_w[a] / 2 * (T[abs_rec[a]] - abs_tobs[a]) ** 2 for a in range(5))
        W = np.zeros((n, n)); DT = np.zeros((n, n))
        for q, (m, i) in enumerate(pairs):
            W[m, i] = W[i, m] = cs_w[q] / 2
            DT[m, i], DT[i, m] = cs_dt[q], -cs_dt[q]
        cc = sum(W[m, i] / 2 * ((T[m] - T[i]) - DT[m, i]) ** 2 for m in range(n) for i in range(n))
        return ct, cc

    ct, cc, R = O.misfit(Tr, abs_rec, abs_tobs, abs_w, cs_m, cs_i, cs_dt, cs_w, alpha, beta)
    pt, pc = chi_paper(Tr)
    assert ct == pytest.approx(pt, rel=1e-13) and cc == pytest.approx(pc, rel=1e-13)
    h = 1e-3
    for m in range(n):
        e = np.zeros(n); e[m] = h
        fp, fm = chi_paper(Tr + e), chi_paper(Tr - e)
        fd = (alpha * (fp[0] - fm[0]) + beta * (fp[1] - fm[1])) / (2 * h)
        assert R[m] == pytest.approx(fd, rel=1e-8, abs=1e-10)


def test_receiver_interpolation_is_exact_for_trilinear_fields(oracle):
    g = I.GridSpec(6, 7, 8, 0.0, 5.0, 0.0, 0.06, 0.0, 0.07)
    depth, lat, lon = g.axes()
    D, LA, LO = np.meshgrid(depth, lat, lon, indexing="ij")
    f = lambda d, a, o: 1.0 + 0.3 * d + 20 * a - 7 * o + 2.0 * d * a * o
    pts = np.array([[0.0, 0.031, 0.012], [3.3, 0.0, 0.07], [4.99, 0.05, 0.035]])
    Tr = oracle.receiver_times(g.as_dict(), f(D, LA, LO), pts)
    assert np.allclose(Tr, f(pts[:, 0], pts[:, 1], pts[:, 2]), rtol=1e-12)


# ----------------------------------------------------------------------------- adjoint

@pytest.fixture(scope="module")
def adjoint_case():
    import oracle as O
    w = I.small_case(1, shape=(15, 17, 19), n_src=1, n_rec=6)
    g = w.grid.as_dict()
    _, T, _, _, _ = O.forward(g, w.s, w.xi, w.eta, w.src[0], tol=1e-12, max_iter=1000)
    return w, g, T


def test_adjoint_positive_and_conservative(oracle, adjoint_case):
    """Eq. 5 in conservation form: with R >= 0 the adjoint field is >= 0, and the net flux
    into the fixed source set equals the total adjoint source sum_m R_m."""
    w, g, T = adjoint_case
    R = np.linspace(0.2, 1.4, len(w.rec))
    P, it, conv, _ = oracle.adjoint(g, T, w.xi, w.eta, w.src[0], w.rec, R, tol=1e-13, max_iter=500)
    assert conv and P.min() >= 0.0 and P.max() > 0
    inflow = oracle.fixed_set_inflow(g, T, w.xi, w.eta, w.src[0], P)
    assert inflow == pytest.approx(R.sum(), rel=1e-9)


def test_adjoint_is_linear_in_sources(oracle, adjoint_case):
    w, g, T = adjoint_case
    rng = np.random.default_rng(3)
    R1, R2 = rng.normal(size=len(w.rec)), rng.normal(size=len(w.rec))
    solve = lambda R: oracle.adjoint(g, T, w.xi, w.eta, w.src[0], w.rec, R, tol=1e-14,
                                     max_iter=500)[0]
    P1, P2, P12 = solve(R1), solve(R2), solve(2.0 * R1 - 0.5 * R2)
    assert np.max(np.abs(P12 - (2.0 * P1 - 0.5 * P2))) <= 1e-10 * np.max(np.abs(P12))


# ----------------------------------------------------------------------------- kernels

def _flat_uniform_case(oracle, n):
    g = I.GridSpec(n, n, n, 0.0, 20.0, 0.0, 0.18, 0.0, 0.18, flat=1)
    s0, x0, e0 = 1 / 6.0, 0.03, -0.02
    src = np.array([16.0, 0.05, 0.06])
    rec = np.array([[0.0, 0.14, 0.12], [0.0, 0.12, 0.15], [0.0, 0.15, 0.05]])
    data = dict(abs_rec=np.arange(3), abs_tobs=np.array([3.0, 3.1, 2.9]), abs_w=np.ones(3),
                cs_m=np.array([0]), cs_i=np.array([1]), cs_dtobs=np.array([0.05]),
                cs_w=np.ones(1))
    gd = g.as_dict()
    s, xi, eta = (np.full(g.shape, v) for v in (s0, x0, e0))
    r = oracle.solve_source(gd, s, xi, eta, src, rec, data, tol_fwd=1e-13, tol_adj=1e-13,
                            max_iter=3000)
    K = [np.zeros(g.shape) for _ in range(3)]
    oracle.kernel_add(gd, s, r["T"], r["P"], *K)
    dV = oracle.node_volumes(gd)
    return g, (s0, x0, e0), src, rec, r, K, dV


def test_kernels_match_analytic_uniform_perturbations(oracle):
    """Eq. 9 with a uniform perturbation of s, xi or eta in a homogeneous flat medium, where
    the traveltime is the closed form T = s sqrt(D^T M^-1 D): sum_x K dV must equal
    sum_m R_m dT_m with dT from differentiating the closed form. Pins the kernel formulas
    of Eqs. 6-8, including the signs and the factor -2 of Eq. 8."""
    g, (s0, x0, e0), src, rec, r, (Ks, Kx, Ke), dV = _flat_uniform_case(oracle, 25)
    D = _cart(g, rec) - _cart(g, src)[0]

    def T_closed(s, xi, eta):
        M = np.array([[1, 0, 0], [0, 1 - 2 * xi, 2 * eta], [0, 2 * eta, 1 + 2 * xi]])
        return s * np.sqrt(np.einsum("ma,ab,mb->m", D, np.linalg.inv(M), D))

    h = 1e-6
    dT_s = (T_closed(s0 * (1 + h), x0, e0) - T_closed(s0 * (1 - h), x0, e0)) / (2 * h)
    dT_x = (T_closed(s0, x0 + h, e0) - T_closed(s0, x0 - h, e0)) / (2 * h)
    dT_e = (T_closed(s0, x0, e0 + h) - T_closed(s0, x0, e0 - h)) / (2 * h)
    R = r["R"]
    for K, dT in ((Ks, dT_s), (Kx, dT_x), (Ke, dT_e)):
        pred, exact = np.sum(K * dV), np.sum(R * dT)
        assert pred / exact == pytest.approx(1.0, abs=0.08)


def test_kernel_discrepancy_shrinks_with_spacing(oracle):
    """A local Gaussian perturbation: the adjoint kernel and a finite difference of the
    discrete misfit agree to first order in the spacing (the continuous adjoint is not the
    exact discrete gradient). Checked for s and eta; xi keeps the right sign (its FD also
    moves the Lax-Friedrichs viscosity, an O(h) term the kernel does not see)."""
    out = {}
    for n in (13, 25):
        g = I.GridSpec(n, n, n, 0.0, 20.0, 0.0, 0.18, 0.0, 0.18)
        v = I.background_velocity(g) * (1 + 0.03 * I.checker(g, 1, 1, 1))
        s = 1 / v
        xi = 0.03 * I.checker(g, 1, 1, 1)
        eta = 0.03 * I.checker(g, 1, 1, 1, phase_cos_phi=True)
        src = np.array([16.0, 0.05, 0.06])
        rec = np.array([[0.0, 0.14, 0.12], [0.0, 0.12, 0.15], [0.0, 0.15, 0.05]])
        data = dict(abs_rec=np.arange(3), abs_tobs=np.array([3.0, 3.1, 2.9]), abs_w=np.ones(3),
                    cs_m=np.array([0]), cs_i=np.array([1]), cs_dtobs=np.array([0.05]),
                    cs_w=np.ones(1))
        gd = g.as_dict()

        def chi(s_, xi_, eta_):
            _, T, _, _, _ = oracle.forward(gd, s_, xi_, eta_, src, 1e-12, 3000)
            ct, cc, _ = oracle.misfit(oracle.receiver_times(gd, T, rec), **data)
            return ct + cc

        r = oracle.solve_source(gd, s, xi, eta, src, rec, data, tol_fwd=1e-12, tol_adj=1e-12,
                                max_iter=3000)
        Ks, Kx, Ke = (np.zeros(g.shape) for _ in range(3))
        oracle.kernel_add(gd, s, r["T"], r["P"], Ks, Kx, Ke)
        dV = oracle.node_volumes(gd)
        P = _node_points(g)
        bump = np.exp(-(((P[..., 0] - 8.0) / 3.0) ** 2 + ((P[..., 1] - 0.1) / 0.03) ** 2
                        + ((P[..., 2] - 0.1) / 0.03) ** 2) / 2)
        e = 1e-3
        ds, dx = 0.02 * s * bump, 0.01 * bump
        fs = (chi(s + e * ds, xi, eta) - chi(s - e * ds, xi, eta)) / (2 * e)
        fx = (chi(s, xi + e * dx, eta) - chi(s, xi - e * dx, eta)) / (2 * e)
        fe = (chi(s, xi, eta + e * dx) - chi(s, xi, eta - e * dx)) / (2 * e)
        out[n] = (np.sum(Ks * dV * ds / s) / fs, np.sum(Kx * dV * dx) / fx,
                  np.sum(Ke * dV * dx) / fe)
    for q in (0, 2):
        assert abs(out[25][q] - 1) < 0.3
        assert abs(out[25][q] - 1) < 0.7 * abs(out[13][q] - 1)
    assert out[13][1] > 0.3 and out[25][1] > 0.3


def test_spherical_uniform_slowness_kernel(oracle):
    """Spherical grid at 60 deg latitude (cos(theta) far from 1, so metric and area factors
    matter): in a homogeneous medium T = s * chord exactly, so a uniform relative change of s
    changes chi by sum_m R_m T_m; Eq. 9 with Eq. 6 must reproduce it."""
    g = I.GridSpec(25, 25, 25, 0.0, 30.0, 60.0, 60.25, 10.0, 10.5)
    gd = g.as_dict()
    s, z = np.full(g.shape, 1 / 6.0), np.zeros(g.shape)
    src = np.array([24.0, 60.05, 10.1])
    rec = np.array([[0.0, 60.2, 10.4], [0.0, 60.18, 10.15], [0.0, 60.08, 10.42]])
    data = dict(abs_rec=np.arange(3), abs_tobs=np.array([3.0, 3.1, 2.9]), abs_w=np.ones(3),
                cs_m=np.array([0]), cs_i=np.array([2]), cs_dtobs=np.array([0.05]),
                cs_w=np.ones(1))
    r = oracle.solve_source(gd, s, z, z, src, rec, data, tol_fwd=1e-12, tol_adj=1e-12)
    K = [np.zeros(g.shape) for _ in range(3)]
    oracle.kernel_add(gd, s, r["T"], r["P"], *K)
    chord = np.linalg.norm(_cart(g, rec) - _cart(g, src)[0], axis=-1)
    pred = np.sum(K[0] * oracle.node_volumes(gd))
    assert pred / np.sum(r["R"] * chord / 6.0) == pytest.approx(1.0, abs=0.06)


@pytest.mark.parametrize("xi0,eta0", [(0.0, 0.1), (0.0, -0.08), (0.12, 0.0), (-0.1, 0.06)])
def test_adjoint_follows_straight_anisotropic_ray(oracle, xi0, eta0):
    """Eq. 5 transports the adjoint source along -M grad T. In a homogeneous anisotropic
    flat medium M grad T is parallel to x - x_s, so the adjoint field of one receiver is
    centred on the straight segment from the receiver to the source at every depth. With
    xi != 0 this pins the (1 -+ 2 xi) factors of the adjoint's face velocities, with
    eta != 0 its cross terms."""
    g = I.GridSpec(31, 41, 41, 0.0, 15.0, 0.0, 0.2, 0.0, 0.2, flat=1)
    gd = g.as_dict()
    s, xi, eta = (np.full(g.shape, v) for v in (1 / 6.0, xi0, eta0))
    src, rec = np.array([14.0, 0.05, 0.06]), np.array([[0.0, 0.15, 0.14]])
    _, T, _, _, _ = oracle.forward(gd, s, xi, eta, src, 1e-12, 1000)
    P, _, conv, _ = oracle.adjoint(gd, T, xi, eta, src, rec, np.array([1.0]), 1e-12, 1000)
    assert conv
    depth, lat, lon = g.axes()
    cell = lat[1] - lat[0]
    for i in (8, 15, 22):
        w = P[i].sum()
        ct, cp = (P[i].sum(1) * lat).sum() / w, (P[i].sum(0) * lon).sum() / w
        f = (depth[i] - rec[0, 0]) / (src[0] - rec[0, 0])
        assert abs(ct - (rec[0, 1] + f * (src[1] - rec[0, 1]))) < 0.75 * cell
        assert abs(cp - (rec[0, 2] + f * (src[2] - rec[0, 2]))) < 0.75 * cell


def test_anisotropic_linear_gradient_first_order(oracle):
    """Constant M with velocity linear in x: the substitution y = M^-1/2 x makes the
    equation isotropic with velocity still linear, so T = arccosh(1 + |A G|^2 q /
    (2 v v_s)) / |A G| with q = D^T M^-1 D and A = M^1/2. First-order convergence."""
    xi0, eta0 = 0.04, -0.03
    M = np.array([[1, 0, 0], [0, 1 - 2 * xi0, 2 * eta0], [0, 2 * eta0, 1 + 2 * xi0]])
    w_, V = np.linalg.eigh(M)
    A = V @ np.diag(np.sqrt(w_)) @ V.T
    errs = []
    for n in (11, 21, 41):
        g = I.GridSpec(n, n, n, 0.0, 30.0, 0.0, 0.27, 0.0, 0.27, flat=1)
        X = _cart(g, _node_points(g))
        src = np.array([15.0, 0.135, 0.135])
        D = X - _cart(g, src)[0]
        Gv = np.array([-0.05, 0.01, 0.02])
        v = 6.0 + D @ Gv
        _, T, _, conv, _ = oracle.forward(g.as_dict(), 1.0 / v, np.full(g.shape, xi0),
                                          np.full(g.shape, eta0), src, 1e-10, 1000)
        AG = np.linalg.norm(A @ Gv)
        q = np.einsum("...a,ab,...b->...", D, np.linalg.inv(M), D)
        exact = np.arccosh(1 + AG ** 2 * q / (2 * v * 6.0)) / AG
        assert conv
        errs.append(np.abs(T - exact).max())
    assert np.log2(errs[0] / errs[1]) >= 0.8 and np.log2(errs[1] / errs[2]) >= 0.8
