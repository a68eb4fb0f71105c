"""Pins of the oracle's Godunov local solver (reading R14 of oracle/tt_oracle.c; isotropic
models): the homogeneous closed form (T = s x chord, tau = 1 exactly), first-order accuracy
against the arccosh traveltime of a linear velocity, a fixed point that does not depend on
the start, and the iteration counts that motivate the scheme (a few iterations where the
Lax-Friedrichs sweep needs a count growing with the grid)."""
import numpy as np
import pytest

import tt_inputs as I
from test_oracle import _cart, _node_points


@pytest.fixture(scope="module")
def oracle():
    import oracle as O
    return O


def test_homogeneous_sphere_is_exact(oracle):
    g = I.GridSpec(21, 21, 21, 0.0, 40.0, 0.0, 1.0, 0.0, 1.0)
    s = np.full(g.shape, 1 / 6.0)
    z = np.zeros(g.shape)
    src = np.array([0.0, 0.5, 0.5])
    tau, T, it, conv, _ = oracle.forward(g.as_dict(), s, z, z, src, tol=1e-12, scheme="godunov")
    X = _cart(g, _node_points(g))
    exact = np.linalg.norm(X - _cart(g, src)[0], axis=-1) / 6.0
    assert conv and np.abs(tau - 1).max() < 1e-12
    assert np.abs(T - exact).max() < 1e-10


def _linear_errors(oracle, n):
    g = I.GridSpec(n, n, n, 0.0, 40.0, 0.0, 0.4, 0.0, 0.4)
    X = _cart(g, _node_points(g))
    src = np.array([20.0, 0.2, 0.2])
    Xs = _cart(g, src)[0]
    Gv = -0.05 * Xs / np.linalg.norm(Xs)
    v = 6.0 + (X - Xs) @ Gv
    z = np.zeros(g.shape)
    _, T, _, conv, _ = oracle.forward(g.as_dict(), 1.0 / v, z, z, src, tol=1e-10,
                                      max_iter=200, scheme="godunov")
    Gn = np.linalg.norm(Gv)
    exact = np.arccosh(1 + Gn ** 2 * np.sum((X - Xs) ** 2, -1) / (2 * v * 6.0)) / Gn
    assert conv
    e = np.abs(T - exact)
    return e.mean(), e.max()


def test_linear_gradient_first_order(oracle):
    errs = [_linear_errors(oracle, n) for n in (11, 21, 41)]
    for (m0, x0), (m1, x1) in zip(errs[:-1], errs[1:]):
        assert np.log2(m0 / m1) >= 0.8
        assert np.log2(x0 / x1) >= 0.7
    assert errs[-1][0] < 0.01


def test_fixed_point_does_not_depend_on_the_start(oracle):
    w = I.small_case(92, shape=(13, 14, 15), n_src=1)
    z = np.zeros(w.grid.shape)
    g = w.grid.as_dict()
    a = oracle.forward(g, w.s, z, z, w.src[0], tol=1e-13, max_iter=200, scheme="godunov")
    rng = np.random.default_rng(92)
    b = oracle.forward(g, w.s, z, z, w.src[0], tol=1e-13, max_iter=200, scheme="godunov",
                       tau_init=1.0 + 0.3 * rng.uniform(size=w.grid.shape))
    assert a[3] and b[3]
    assert np.abs(a[1] - b[1]).max() <= 1e-10 * np.abs(a[1]).max()


def test_few_iterations_where_lax_friedrichs_needs_many(oracle):
    n = 41
    w = I.small_case(91, shape=(n, n, n), n_src=1)
    z = np.zeros(w.grid.shape)
    i, j, k = np.meshgrid(*[np.arange(m) for m in w.grid.shape], indexing="ij")
    s = (1 / 6.0) * (1 + 0.05 * np.sin(np.pi * i / 10) * np.sin(np.pi * j / 10) *
                     np.sin(np.pi * k / 10))
    g = w.grid.as_dict()
    god = oracle.forward(g, s, z, z, w.src[0], tol=1e-8, max_iter=500, scheme="godunov")
    lf = oracle.forward(g, s, z, z, w.src[0], tol=1e-8, max_iter=500)
    assert god[3] and lf[3]
    assert god[2] <= 6 and lf[2] >= 2 * god[2]
    # the two first-order schemes agree to their discretisation error
    assert np.abs(god[1] - lf[1]).max() <= 0.02 * np.abs(lf[1]).max()
