"""Pin of the upwind-side rule of reading R16 (oracle/tt_oracle.c) against the exact monotone
formulation it abbreviates.

The Godunov update is the smallest causal root over every choice of upwind side per axis
and every axis subset. The oracle takes r's side from the neighbours' first-order
estimates of T (M has no cross term on r). Along theta and phi it takes the side the
characteristic M g comes from, which leaves 7 candidates instead of 17.

This file re-implements the sweep in plain Python on a small anisotropic grid (flat test
geometry) with either rule:
- With the oracle's rule it must reproduce the oracle's traveltime to rounding. That
  checks the Python harness (factor, fixed set, orderings, face rule).
- With every side of theta and phi tried, the fixed point must agree with the oracle's to
  far below the discretisation error. Measured: 1.2e-14 of max T here, and 1.5e-7 on a
  41 x 55 x 55 spherical grid with the benchmark's anisotropic model.
"""
import numpy as np
import pytest

import tt_inputs as I

DEG = np.pi / 180.0


def _setup(g, src):
    re_ = g.earth_radius_km
    dr = (g.depth_max_km - g.depth_min_km) / (g.n_r - 1)
    dt = (g.lat_max_deg - g.lat_min_deg) * DEG / (g.n_t - 1)
    dp = (g.lon_max_deg - g.lon_min_deg) * DEG / (g.n_p - 1)
    r0 = re_ - g.depth_max_km
    f = [((re_ - src[0]) - r0) / dr, (src[1] * DEG - g.lat_min_deg * DEG) / dt,
         (src[2] * DEG - g.lon_min_deg * DEG) / dp]
    n = g.shape
    c = [min(max(int(np.floor(f[a] + 0.5)), 0), n[a] - 1) for a in range(3)]
    return (dr, dt, dp), r0, c


def _update(tau, i, j, k, T0, p0, s, xi, eta, h, dl, all_sides):
    tp = [tau[i + 1, j, k], tau[i, j + 1, k], tau[i, j, k + 1]]
    tm = [tau[i - 1, j, k], tau[i, j - 1, k], tau[i, j, k - 1]]
    M = np.array([[1.0, 0.0, 0.0], [0.0, 1 - 2 * xi, 2 * eta], [0.0, 2 * eta, 1 + 2 * xi]])
    Mi = np.linalg.inv(M)
    u = [p0[d] / T0 for d in range(3)]
    e = [1.0 / (dl[d] * h[d]) for d in range(3)]
    gc = [u[d] * tau[i, j, k] + 0.5 * e[d] * (tp[d] - tm[d]) for d in range(3)]
    opts = []
    for d in range(3):
        if d == 0:
            lower = tm[0] * (1 - u[0] / e[0]) <= tp[0] * (1 + u[0] / e[0])
            sides = [lower]
        elif all_sides:
            sides = [True, False]
        else:
            sides = [M[d] @ np.array(gc) >= 0.0]
        opts.append([(1.0 if lo else -1.0, tm[d] if lo else tp[d]) for lo in sides])
    rhs = s / T0
    best = None
    for mask in range(1, 8):
        ax = [d for d in range(3) if mask >> d & 1]
        if len(ax) == 3:
            W = M
        else:
            W = np.linalg.inv(Mi[np.ix_(ax, ax)])
        for choice in np.ndindex(*[len(opts[d]) for d in ax]):
            sg = np.array([opts[d][q][0] for d, q in zip(ax, choice)])
            nb = np.array([opts[d][q][1] for d, q in zip(ax, choice)])
            a = np.array([u[d] for d in ax]) + sg * np.array([e[d] for d in ax])
            b = sg * np.array([e[d] for d in ax]) * nb
            A, B, C = a @ W @ a, a @ W @ b, b @ W @ b - rhs * rhs
            disc = B * B - A * C
            if not A > 0 or disc < 0:
                continue
            t = (B + np.sqrt(disc)) / A
            if np.all(sg * (W @ (a * t - b)) >= 0) and (best is None or t < best):
                best = t
    return tau[i, j, k] if best is None else best


def _solve(g, s, xi, eta, src, all_sides, tol=1e-11, max_iter=60):
    """Fast sweeping with the R16 update in the flat test geometry (h2 = h3 = R_E)."""
    import oracle as O
    assert g.flat
    T0, p0 = O.T0(g.as_dict(), s, xi, eta, src)
    dl, r0, c = _setup(g, src)
    n = g.shape
    tau = np.ones(n)

    def fixed(i, j, k):
        return abs(i - c[0]) <= 1 and abs(j - c[1]) <= 1 and abs(k - c[2]) <= 1

    re_ = g.earth_radius_km
    for it in range(max_iter):
        err = 0.0
        for o in range(8):
            dr_, dt_, dp_ = (-1 if o & 4 else 1), (-1 if o & 2 else 1), (-1 if o & 1 else 1)
            ii = range(1, n[0] - 1) if dr_ > 0 else range(n[0] - 2, 0, -1)
            jj = range(1, n[1] - 1) if dt_ > 0 else range(n[1] - 2, 0, -1)
            kk = range(1, n[2] - 1) if dp_ > 0 else range(n[2] - 2, 0, -1)
            for i in ii:
                for j in jj:
                    for k in kk:
                        if fixed(i, j, k):
                            continue
                        h = (1.0, re_, re_)
                        v = _update(tau, i, j, k, T0[i, j, k], p0[i, j, k], s[i, j, k],
                                    xi[i, j, k], eta[i, j, k], h, dl, all_sides)
                        err = max(err, abs(v - tau[i, j, k]))
                        tau[i, j, k] = v
            # faces: r, theta, phi, low then high (fixed nodes exempt)
            for ax in range(3):
                for hi in (False, True):
                    sl = [slice(None)] * 3
                    a1, a2 = [slice(None)] * 3, [slice(None)] * 3
                    sl[ax] = n[ax] - 1 if hi else 0
                    a1[ax] = n[ax] - 2 if hi else 1
                    a2[ax] = n[ax] - 3 if hi else 2
                    new = np.maximum(2 * tau[tuple(a1)] - tau[tuple(a2)], tau[tuple(a2)])
                    face = tau[tuple(sl)]
                    idx = np.argwhere(np.ones(face.shape, bool))
                    for q in idx:
                        full = list(q)
                        full.insert(ax, sl[ax])
                        if not fixed(*full):
                            face[tuple(q)] = new[tuple(q)]
        if err < tol:
            break
    return T0 * tau, it + 1


@pytest.mark.slow
def test_python_harness_reproduces_the_oracle_and_all_sides_agree():
    import oracle as O
    g = I.GridSpec(9, 10, 11, 0.0, 10.0, 0.0, 0.09, 0.0, 0.1, flat=1)
    i, j, k = np.meshgrid(*[np.linspace(0, 1, n) for n in g.shape], indexing="ij")
    s = (1 / 6.0) * (1 + 0.04 * np.sin(4 * i) * np.cos(3 * j + 2 * k))
    xi = 0.04 * np.sin(3 * j) * np.cos(2 * k + i)
    eta = 0.04 * np.cos(2 * j + i) * np.sin(3 * k)
    src = np.array([4.2, 0.041, 0.055])
    _, To, it_o, conv, _ = O.forward(g.as_dict(), s, xi, eta, src, tol=1e-11, max_iter=60,
                                     scheme="godunov_aniso")
    assert conv
    Tc, it_c = _solve(g, s, xi, eta, src, all_sides=False)
    assert np.abs(Tc - To).max() <= 1e-12 * To.max()
    assert it_c == it_o
    Ta, _ = _solve(g, s, xi, eta, src, all_sides=True)
    print("\nall sides against the characteristic rule: %.2e of max T"
          % (np.abs(Ta - To).max() / To.max()))
    assert np.abs(Ta - To).max() <= 1e-6 * To.max()
