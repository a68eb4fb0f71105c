"""Pins of the teleseismic-boundary oracle (reading R17; oracle/tele.py and tt_oracle.c)
against facts outside its own code:
- 2-D, homogeneous 1-D model: the factor is exact, so T = s x chord to rounding;
- 2-D, v = c r: with rho = ln r the equation becomes |grad T| = 1/c in (rho, Delta), so
  T = sqrt(ln(r / r_s)^2 + Delta^2) / c exactly; the solve converges to it at first order;
- 3-D, homogeneous, exact times on the faces of a region 10 deg from the event: the
  interior converges to T = s x chord as h shrinks;
- 3-D, the whole chain in the v = c r model (2-D solve, faces by interpolation, 3-D solve):
  first order against the same closed form;
- the 3-D fixed point does not depend on the interior's start.
"""
import numpy as np
import pytest

import tt_inputs as I
from test_oracle import _cart, _node_points

RE = 6371.0
EVENT = (100.0, -6.0, 3.0)            # depth km, lat, lon: ~8.6 deg from the region


@pytest.fixture(scope="module")
def tl():
    import oracle.tele as TL
    return TL


def test_2d_homogeneous_is_exact(tl):
    n_r, n_d, r_min, dmax = 41, 61, RE - 400.0, 12.0
    T, it, conv = tl.tele2d(r_min, RE, n_r, dmax, n_d, np.full(n_r, 1 / 8.0), RE - 100.0,
                            tol=1e-12)
    r = np.linspace(r_min, RE, n_r)[:, None]
    D = np.radians(np.linspace(0, dmax, n_d))[None, :]
    rs = RE - 100.0
    exact = np.sqrt(r ** 2 + rs ** 2 - 2 * r * rs * np.cos(D)) / 8.0
    assert conv and np.abs(T - exact).max() <= 1e-12 * exact.max()


def _closed_form_2d(tl, n):
    r_min, dmax, c, rs = RE - 400.0, 12.0, 8.0 / RE, RE - 100.0
    r = np.linspace(r_min, RE, n)
    T, it, conv = tl.tele2d(r_min, RE, n, dmax, 2 * n - 1, 1 / (c * r), rs, tol=1e-10,
                            max_iter=500)
    D = np.radians(np.linspace(0, dmax, 2 * n - 1))[None, :]
    exact = np.sqrt(np.log(r[:, None] / rs) ** 2 + D ** 2) / c
    assert conv
    e = np.abs(T - exact) / exact.max()
    return e.max(), e.mean()


def test_2d_linear_in_radius_converges_at_first_order(tl):
    errs = [_closed_form_2d(tl, n) for n in (21, 41, 81)]
    for (x0, m0), (x1, m1) in zip(errs[:-1], errs[1:]):
        assert np.log2(x0 / x1) >= 0.9 and np.log2(m0 / m1) >= 0.9
    assert errs[-1][0] <= 1e-3


def _region(n):
    return I.GridSpec(n, n, n, 0.0, 40.0, 0.0, 1.0, 0.0, 1.0)


def _faces_from(T_exact, start):
    for ax in range(3):
        for side in (0, -1):
            sl = [slice(None)] * 3
            sl[ax] = side
            start[tuple(sl)] = T_exact[tuple(sl)]
    return start


def test_3d_homogeneous_with_exact_faces(tl):
    errs = []
    for n in (11, 21, 41):
        g = _region(n)
        X = _cart(g, _node_points(g))
        exact = np.linalg.norm(X - _cart(g, np.array(EVENT))[0], axis=-1) / 6.0
        z = np.zeros(g.shape)
        start = _faces_from(exact, exact * 1.05)
        T, it, conv = tl.forward_tele(g.as_dict(), np.full(g.shape, 1 / 6.0), z, z, start,
                                      tol=1e-10, max_iter=2000)
        assert conv
        errs.append(np.abs(T - exact).max() / exact.max())
    assert errs[0] > errs[1] > errs[2] and errs[2] <= 0.7 * errs[1]
    assert errs[-1] <= 5e-4


def _chain(tl, n, start_noise=0.0):
    c, r_min, dmax = 6.0 / RE, RE - 300.0, 12.0
    g = _region(n)
    gd = g.as_dict()
    depth = np.linspace(40.0, 0.0, n)
    s = np.broadcast_to((1 / (c * (RE - depth)))[:, None, None], g.shape).copy()
    rr = np.linspace(r_min, RE, 8 * n)
    T2, _, conv2 = tl.tele2d(r_min, RE, 8 * n, dmax, 8 * n, 1 / (c * rr), RE - EVENT[0],
                             tol=1e-10, max_iter=500)
    assert conv2
    start = tl.region_times(gd, T2, r_min, RE, dmax, EVENT[1], EVENT[2])
    if start_noise:
        noisy = start * (1 + start_noise * np.random.default_rng(n).standard_normal(g.shape))
        start = _faces_from(start, noisy)
    z = np.zeros(g.shape)
    T, it, conv = tl.forward_tele(gd, s, z, z, start, tol=1e-10, max_iter=3000)
    assert conv
    R, LA, LO = np.meshgrid(RE - depth, np.linspace(0, 1, n), np.linspace(0, 1, n),
                            indexing="ij")
    D = tl.epicentral_angle(LA, LO, EVENT[1], EVENT[2])
    exact = np.sqrt(np.log(R / (RE - EVENT[0])) ** 2 + D ** 2) / c
    return T, exact


def test_3d_chain_in_a_one_dimensional_model(tl):
    errs = []
    for n in (11, 21, 41):
        T, exact = _chain(tl, n)
        errs.append(np.abs(T - exact).max() / exact.max())
    assert errs[0] > errs[1] > errs[2] and errs[2] <= 0.7 * errs[1]
    assert errs[-1] <= 5e-4


def test_3d_fixed_point_does_not_depend_on_the_start(tl):
    Ta, _ = _chain(tl, 15)
    Tb, _ = _chain(tl, 15, start_noise=0.03)
    assert np.abs(Ta - Tb).max() <= 1e-8 * np.abs(Ta).max()
