"""Pins of the oracle's anisotropic Godunov local solver (reading R16 of oracle/tt_oracle.c)
against facts outside its own code: the elliptical closed form of a homogeneous anisotropic
medium (exact), first order against the closed form of an anisotropic linear-velocity
medium, a fixed point that does not depend on the start, agreement with the isotropic
Godunov solver (R14) when xi = eta = 0, and a few iterations where Lax-Friedrichs needs
many."""
import numpy as np
import pytest

import tt_inputs as I
from test_oracle import _cart, _node_points


@pytest.fixture(scope="module")
def oracle():
    import oracle as O
    return O


def _M(xi0, eta0):
    return np.array([[1, 0, 0], [0, 1 - 2 * xi0, 2 * eta0], [0, 2 * eta0, 1 + 2 * xi0]])


@pytest.mark.parametrize("xi0,eta0", [(0.03, -0.02), (-0.04, 0.01), (0.0, 0.045)])
def test_homogeneous_anisotropic_flat_is_exact(oracle, xi0, eta0):
    """T = s sqrt(D^T M^-1 D) is the exact factor, so tau = 1 must be the fixed point."""
    g = I.GridSpec(17, 19, 15, 0.0, 16.0, 0.0, 0.15, 0.0, 0.13, flat=1)
    s0 = 1 / 5.5
    s = np.full(g.shape, s0)
    xi, eta = np.full(g.shape, xi0), np.full(g.shape, eta0)
    src = np.array([9.0, 0.07, 0.05])
    tau, T, it, conv, _ = oracle.forward(g.as_dict(), s, xi, eta, src, tol=1e-12,
                                         scheme="godunov_aniso")
    D = _cart(g, _node_points(g)) - _cart(g, src)[0]
    exact = s0 * np.sqrt(np.einsum("...a,ab,...b->...", D, np.linalg.inv(_M(xi0, eta0)), D))
    assert conv and np.abs(tau - 1).max() <= 1e-12
    assert np.max(np.abs(T - exact)) <= 1e-12 * np.max(exact)


def test_anisotropic_linear_gradient_first_order(oracle):
    """Constant M, velocity linear in x: y = M^-1/2 x makes the problem isotropic with a
    linear velocity, so T = arccosh(1 + |A G|^2 q / (2 v v_s)) / |A G|, q = D^T M^-1 D,
    A = M^1/2. Observed order >= 0.8 in the largest and the mean error."""
    xi0, eta0 = 0.04, -0.03
    M = _M(xi0, eta0)
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
        _, T, it, conv, _ = oracle.forward(g.as_dict(), 1.0 / v, np.full(g.shape, xi0),
                                           np.full(g.shape, eta0), src, 1e-10, 1000,
                                           scheme="godunov_aniso")
        AG = np.linalg.norm(A @ Gv)
        q = np.einsum("...a,ab,...b->...", D, np.linalg.inv(M), D)
        exact = np.arccosh(1 + AG ** 2 * q / (2 * v * 6.0)) / AG
        assert conv and it <= 10
        e = np.abs(T - exact)
        errs.append((e.max(), e.mean()))
    for (x0, m0), (x1, m1) in zip(errs[:-1], errs[1:]):
        assert np.log2(x0 / x1) >= 0.8 and np.log2(m0 / m1) >= 0.8


def test_fixed_point_does_not_depend_on_the_start(oracle):
    w = I.small_case(95, shape=(13, 14, 15), n_src=1)
    g = w.grid.as_dict()
    rng = np.random.default_rng(95)
    _, T1, _, c1, _ = oracle.forward(g, w.s, w.xi, w.eta, w.src[0], tol=1e-12,
                                     scheme="godunov_aniso")
    init = 1.0 + 0.3 * rng.uniform(size=w.grid.shape)
    _, T2, _, c2, _ = oracle.forward(g, w.s, w.xi, w.eta, w.src[0], tol=1e-12,
                                     tau_init=init, scheme="godunov_aniso")
    assert c1 and c2
    assert np.abs(T1 - T2).max() <= 1e-10 * np.abs(T1).max()


def test_isotropic_model_agrees_with_the_isotropic_solver(oracle):
    """With xi = eta = 0 the two readings differ only in how the theta and phi sides are
    picked; both are consistent upwind schemes and agree to far below their O(h) error."""
    w = I.small_case(96, shape=(15, 16, 17), n_src=2)
    z = np.zeros(w.grid.shape)
    g = w.grid.as_dict()
    for b in range(2):
        _, Ta, _, ca, _ = oracle.forward(g, w.s, z, z, w.src[b], tol=1e-12, scheme="godunov")
        _, Tb, _, cb, _ = oracle.forward(g, w.s, z, z, w.src[b], tol=1e-12,
                                         scheme="godunov_aniso")
        assert ca and cb
        assert np.abs(Ta - Tb).max() <= 1e-6 * np.abs(Ta).max()


def test_few_iterations_where_lax_friedrichs_needs_many(oracle):
    w = I.anisotropic_batch(n_src=2, shape=(33, 41, 41))
    g = w.grid.as_dict()
    for b in range(2):
        _, Tl, il, cl, _ = oracle.forward(g, w.s, w.xi, w.eta, w.src[b], tol=1e-6)
        _, Tg, ig, cg, _ = oracle.forward(g, w.s, w.xi, w.eta, w.src[b], tol=1e-6,
                                          scheme="godunov_aniso")
        assert cl and cg
        assert ig <= 8 and il >= 2 * ig
        assert np.abs(Tg - Tl).max() <= 0.05 * np.abs(Tl).max()     # same equation, O(h) apart
