"""Pins of the relocation-kernel oracle (oracle/reloc.py; Eq. 10, Eqs. B1-B11, reading R15)
against facts outside its own code:
- a field linear in the grid indices has the closed-form physical gradient, with the
  spherical metric at the point (pins the axis order, the spacings and the factors r and
  r cos(theta));
- K_x is the derivative of the total misfit (absolute, common-source and common-receiver
  terms) with respect to depth, latitude and longitude, by central differences;
- K_tau is the derivative with respect to the origin time; with common-source pairs only
  it vanishes (Eq. B10);
- reciprocity (Appendix B): Gamma_m(x_s) from a solve started at the receiver equals the
  time at the receiver from a solve started at the source, to first order in h.
"""
import numpy as np
import pytest

import tt_inputs as I


def _grid():
    return I.GridSpec(9, 11, 10, 0.0, 40.0, 10.0, 11.0, 20.0, 21.5)


def _points(g, n, rng):
    lo = np.array([g.depth_min_km, g.lat_min_deg, g.lon_min_deg])
    hi = np.array([g.depth_max_km, g.lat_max_deg, g.lon_max_deg])
    return lo + (hi - lo) * rng.uniform(0.02, 0.98, (n, 3))


def test_linear_index_field_has_the_closed_form_gradient():
    import oracle.reloc as L
    g = _grid()
    i, j, k = np.meshgrid(*[np.arange(n) for n in g.shape], indexing="ij")
    c = (0.7, -1.3, 0.4, 2.1)
    F = c[0] + c[1] * i + c[2] * j + c[3] * k
    rng = np.random.default_rng(1)
    deg = np.pi / 180
    dr = (g.depth_max_km - g.depth_min_km) / (g.n_r - 1)
    dt = (g.lat_max_deg - g.lat_min_deg) * deg / (g.n_t - 1)
    dp = (g.lon_max_deg - g.lon_min_deg) * deg / (g.n_p - 1)
    for p in _points(g, 20, rng):
        r = g.earth_radius_km - p[0]
        fi = (r - (g.earth_radius_km - g.depth_max_km)) / dr
        fj = (p[1] - g.lat_min_deg) * deg / dt
        fk = (p[2] - g.lon_min_deg) * deg / dp
        val, grad = L.field_at(g.as_dict(), F, p)
        assert abs(val - (c[0] + c[1] * fi + c[2] * fj + c[3] * fk)) <= 1e-12
        ref = [c[1] / dr, c[2] / (r * dt), c[3] / (r * np.cos(p[1] * deg) * dp)]
        np.testing.assert_allclose(grad, ref, rtol=1e-12)


def _case(seed, ns=4, nr=6, cs=True, absolute=True, cr=True):
    rng = np.random.default_rng(seed)
    g = _grid()
    fields = [rng.uniform(5.0, 15.0) + rng.standard_normal(g.shape) for _ in range(nr)]
    pts = _points(g, ns, rng)
    tau = rng.normal(0.0, 0.3, ns)
    Tobs = rng.uniform(5.0, 15.0, (ns, nr))
    abs_recs, cs_recs = [], []
    for n in range(ns):
        m = np.arange(nr) if absolute else np.zeros(0, int)
        abs_recs.append((m, Tobs[n, m] + rng.normal(0, 0.2, len(m)), rng.uniform(0.5, 2.0, len(m))))
        pairs = [(a, b) for a in range(nr) for b in range(a + 1, nr) if cs and rng.uniform() < 0.5]
        cm = np.array([a for a, _ in pairs], int)
        ci = np.array([b for _, b in pairs], int)
        cs_recs.append((cm, ci, Tobs[n, cm] - Tobs[n, ci] + rng.normal(0, 0.1, len(pairs)),
                        rng.uniform(0.5, 2.0, len(pairs))))
    W = np.zeros((ns, ns, nr))
    if cr:
        for m in range(nr):
            for a in range(ns):
                for b in range(a + 1, ns):
                    if rng.uniform() < 0.6:
                        W[a, b, m] = W[b, a, m] = rng.uniform(0.2, 1.0)
    return g.as_dict(), fields, pts, tau, Tobs, abs_recs, cs_recs, W


def _chi(g, fields, pts, tau, Tobs, abs_recs, cs_recs, W, alpha=1.0, beta=0.7, gamma=1.3):
    import oracle.reloc as L
    val, _ = L.table(g, fields, pts)
    Tr = val + tau[:, None]
    ct, cc, ccr, R = L.misfit_table(Tr, abs_recs, cs_recs, alpha, beta, (Tobs, W, gamma))
    return alpha * ct + beta * cc + gamma * ccr, R


def test_location_kernel_is_the_derivative_of_the_misfit():
    import oracle.reloc as L
    g, fields, pts, tau, Tobs, abs_recs, cs_recs, W = _case(2)
    _, R = _chi(g, fields, pts, tau, Tobs, abs_recs, cs_recs, W)
    _, grad = L.table(g, fields, pts)
    Kx, _ = L.kernels(R, grad)
    deg = np.pi / 180
    for n in range(len(pts)):
        r = g["earth_radius_km"] - pts[n, 0]
        fd = []
        for a, h in ((0, 1e-5), (1, 1e-7), (2, 1e-7)):
            q1, q2 = pts.copy(), pts.copy()
            q1[n, a] += h
            q2[n, a] -= h
            c1, _ = _chi(g, fields, q1, tau, Tobs, abs_recs, cs_recs, W)
            c2, _ = _chi(g, fields, q2, tau, Tobs, abs_recs, cs_recs, W)
            fd.append((c1 - c2) / (2 * h))
        # d/d depth = -d/dr; d/d lat (deg) = r deg K_theta; d/d lon (deg) = r cos(theta) deg K_phi
        ref = np.array([-fd[0], fd[1] / (r * deg), fd[2] / (r * np.cos(pts[n, 1] * deg) * deg)])
        np.testing.assert_allclose(Kx[n], ref, rtol=2e-6, atol=1e-8 * np.abs(ref).max())


def test_origin_time_kernel_is_the_derivative_of_the_misfit():
    import oracle.reloc as L
    g, fields, pts, tau, Tobs, abs_recs, cs_recs, W = _case(3)
    _, R = _chi(g, fields, pts, tau, Tobs, abs_recs, cs_recs, W)
    _, grad = L.table(g, fields, pts)
    _, Kt = L.kernels(R, grad)
    for n in range(len(pts)):
        t1, t2 = tau.copy(), tau.copy()
        t1[n] += 1e-5
        t2[n] -= 1e-5
        c1, _ = _chi(g, fields, pts, t1, Tobs, abs_recs, cs_recs, W)
        c2, _ = _chi(g, fields, pts, t2, Tobs, abs_recs, cs_recs, W)
        assert abs(Kt[n] - (c1 - c2) / 2e-5) <= 1e-7 * max(1.0, abs(Kt[n]))


def test_common_source_pairs_do_not_move_the_origin_time():
    """Eq. B10: a common-source difference does not contain tau_n."""
    import oracle.reloc as L
    g, fields, pts, tau, Tobs, abs_recs, cs_recs, W = _case(4, absolute=False, cr=False)
    _, R = _chi(g, fields, pts, tau, Tobs, abs_recs, cs_recs, W)
    _, grad = L.table(g, fields, pts)
    Kx, Kt = L.kernels(R, grad)
    assert np.abs(Kx).max() > 1e-3
    assert np.abs(Kt).max() <= 1e-12 * np.abs(R).max()


@pytest.mark.slow
def test_reciprocity_of_receiver_and_source_solves():
    """Appendix B: T_n(x_r) (solve from the source) = Gamma_m(x_s) (solve from the
    receiver). Both are first-order approximations of the same time: on a heterogeneous
    grid they agree to 0.025 % at 13^3 and 0.015 % at 25^3 (bound 0.1 %, and the gap must
    shrink with h). The gradient obeys the eikonal equation at the source, |grad Gamma| = s,
    to first order: -0.69 % at 13^3, -0.16 % at 25^3 (bound 0.5 %)."""
    import oracle as O
    import oracle.reloc as L
    gaps = []
    for n in (13, 25):
        g = I.GridSpec(n, n, n, 0.0, 30.0, 0.0, 0.3, 0.0, 0.3)
        gd = g.as_dict()
        i, j, k = np.meshgrid(*[np.linspace(0, 1, n)] * 3, indexing="ij")
        s = (1 / 6.0) * (1 + 0.05 * np.sin(3 * i) * np.cos(2 * j + k))
        z = np.zeros(g.shape)
        src = (22.0, 0.12, 0.17)
        rec = (0.0, 0.21, 0.08)
        _, Ts, _, ok1, _ = O.forward(gd, s, z, z, src, tol=1e-11, max_iter=1000)
        _, Gm, _, ok2, _ = O.forward(gd, s, z, z, rec, tol=1e-11, max_iter=1000)
        assert ok1 and ok2
        t_sr = O.receiver_times(gd, Ts, [rec])[0]
        g_rs, grad = L.field_at(gd, Gm, src)
        gaps.append(abs(t_sr - g_rs) / t_sr)
        f = np.array([(30.0 - src[0]) / 30.0, src[1] / 0.3, src[2] / 0.3])
        s_src = (1 / 6.0) * (1 + 0.05 * np.sin(3 * f[0]) * np.cos(2 * f[1] + f[2]))
        eik = abs(np.linalg.norm(grad) / s_src - 1.0)
    assert gaps[1] <= 1e-3
    assert gaps[1] <= 0.7 * gaps[0]
    assert eik <= 5e-3


def test_update_hand_values():
    """Reading R15b by hand: the event with the largest |K_x| moves step_km against it (a
    pure +r gradient deepens the event by step_km; a pure theta gradient moves it south by
    step_km / r radians); the others move in proportion; clamping stops at the grid."""
    import oracle.reloc as L
    g = _grid().as_dict()
    pts = np.array([[20.0, 10.5, 20.7], [10.0, 10.2, 21.0], [39.9, 10.9, 20.1]])
    Kx = np.array([[2.0, 0.0, 0.0], [0.0, 1.0, 0.0], [-0.5, 0.0, 0.0]])
    Kt = np.array([0.5, -2.0, 0.0])
    p, t = L.update(g, pts, np.zeros(3), Kx, Kt, 3.0, 0.1)
    r1 = g["earth_radius_km"] - 10.0
    np.testing.assert_allclose(p[0], [23.0, 10.5, 20.7], rtol=0, atol=1e-12)
    np.testing.assert_allclose(p[1], [10.0, 10.2 - 1.5 / r1 * 180 / np.pi, 21.0], rtol=0, atol=1e-12)
    assert abs(p[2, 0] - (39.9 - 0.75)) <= 1e-12                       # moves up 0.75 km
    np.testing.assert_allclose(t, [-0.025, 0.1, 0.0], rtol=0, atol=1e-15)
    p, _ = L.update(g, pts, np.zeros(3), -Kx, Kt, 3.0, 0.1)
    assert p[2, 0] == 40.0                                             # clamped at depth_max
