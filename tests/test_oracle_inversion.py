"""Pins of the inversion-step oracle (oracle/inversion.py) against facts that do not come
from its own code: the partition of unity of the offset hat bases, the closed form of a
hat function, the exact adjointness of projection (Eq. 17) and expansion (Eq. 15) under the
dV-weighted inner product, hand values of Eq. 18 and of the update, and the superposition
that makes K_d (Eq. 19) the sum of unit-source adjoint fields."""
import numpy as np

import oracle.inversion as V


def test_axis_bases_are_partitions_of_unity():
    for n, c, H in ((41, 11, 5), (17, 6, 3), (9, 11, 5), (201, 11, 5)):
        U = V.axis_basis(n, c, H)
        assert U.min() >= 0.0
        np.testing.assert_allclose(U.sum(axis=1), 1.0, rtol=0, atol=1e-14)
        # at most two hats overlap any point of one axis
        assert ((U > 0).sum(axis=1) <= 2).all()


def test_hat_functions_match_the_closed_form():
    n, c, H = 33, 7, 4
    U = V.axis_basis(n, c, H)
    x = np.arange(n) / (n - 1)
    dc = 1.0 / (c - 2)
    for h in range(H):
        for a in range(c):
            xa = (a - h / H) * dc
            ref = np.maximum(0.0, 1.0 - np.abs(x - xa) / dc)
            np.testing.assert_allclose(U[h, a], ref, rtol=0, atol=1e-14)


def test_coarse_nodes_on_forward_nodes_take_value_one():
    c = 11
    n = 4 * (c - 2) + 1        # grid 0's nodes fall on every 4th forward node
    U = V.axis_basis(n, c, 5)
    for a in range(c - 1):
        assert abs(U[0, a, 4 * a] - 1.0) <= 1e-14
        assert abs(U[0, :, 4 * a].sum() - 1.0) <= 1e-14


def test_expansion_of_ones_is_one():
    shape, coarse, H = (9, 13, 11), (5, 6, 5), 3
    B = V.bases(shape, coarse, H)
    D = V.expand(np.ones((H,) + coarse), B, H)
    np.testing.assert_allclose(D, 1.0, rtol=0, atol=1e-13)


def test_projection_is_the_adjoint_of_the_expansion():
    rng = np.random.default_rng(5)
    shape, coarse, H = (9, 13, 11), (5, 6, 5), 3
    B = V.bases(shape, coarse, H)
    K = rng.standard_normal(shape)
    dV = rng.uniform(0.5, 2.0, shape)
    G = rng.standard_normal((H,) + coarse)
    lhs = np.sum(V.project(K, dV, B, H) * G)
    rhs = np.sum(K * dV * V.expand(G, B, H))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_projection_of_a_constant_is_the_integral_of_the_basis():
    shape, coarse, H = (9, 13, 11), (5, 6, 5), 3
    B = V.bases(shape, coarse, H)
    G = V.project(np.ones(shape), np.ones(shape), B, H)
    # summed over every basis function of every grid: the number of forward nodes (unity)
    assert abs(G.sum() - np.prod(shape)) <= 1e-10


def test_normalisation_hand_values():
    K = np.array([8.0, -8.0, 2.0])
    Kd = np.array([3.0, 3.0, 0.0])
    np.testing.assert_allclose(V.normalize(K, Kd, 1.0, 0.5), [4.0, -4.0, 2.0], rtol=1e-15)
    np.testing.assert_allclose(V.normalize(K, Kd, 1.0, 0.0), K, rtol=0)
    np.testing.assert_allclose(V.normalize(K, Kd, 1.0, 1.0), [2.0, -2.0, 2.0], rtol=1e-15)


def test_update_with_constant_directions():
    s = np.full(4, 0.2); xi = np.full(4, 0.01); eta = np.full(4, -0.02)
    c = np.full(4, 3.0)
    s1, x1, e1 = V.update(s, xi, eta, c, c, -c, 0.05)
    np.testing.assert_allclose(s1, 0.2 * 0.95, rtol=1e-15)
    np.testing.assert_allclose(x1, 0.01 - 0.05, rtol=1e-15)
    np.testing.assert_allclose(e1, -0.02 + 0.05, rtol=1e-14)


def test_kernel_density_field_is_the_sum_of_unit_source_adjoints():
    """Eq. 5 is linear in its sources: the adjoint field with R = 1 at every receiver equals
    the sum of the fields with R = 1 at one receiver each, so K_d of Eq. 19 is a sum of
    single-receiver adjoints."""
    import oracle as O
    import tt_inputs as I
    w = I.small_case(71, shape=(9, 10, 11), n_src=1, n_rec=3)
    g = w.grid.as_dict()
    _, T, _, _, _ = O.forward(g, w.s, w.xi, w.eta, w.src[0], tol=1e-12, max_iter=500)
    P_all, _, ok, _ = O.adjoint(g, T, w.xi, w.eta, w.src[0], w.rec, np.ones(len(w.rec)),
                                tol=1e-13, max_iter=2000)
    assert ok
    parts = []
    for m in range(len(w.rec)):
        R = np.zeros(len(w.rec)); R[m] = 1.0
        P, _, ok, _ = O.adjoint(g, T, w.xi, w.eta, w.src[0], w.rec, R, tol=1e-13, max_iter=2000)
        assert ok
        parts.append(P)
    Kd = V.kernel_density(parts)
    assert np.abs(Kd - P_all).max() <= 1e-9 * np.abs(P_all).max()
