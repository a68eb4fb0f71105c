"""Single-node finite-difference pins of the oracle's adjoint and kernels (Eqs. 5-9).

Eq. 9 states that a model change moves the misfit by the volume integral of the kernels
times the change: dchi = sum_n (K_s dln s + K_xi dxi + K_eta deta)_n dV_n. Here every interior
node of a small spherical grid is perturbed on its own, in s, xi and eta in turn, and the
central difference of the misfit (forward solve, receiver times and Eqs. 2-3, all tightly
converged) is compared with K dV at that node. The two sides share no code beyond the forward
solve: the kernels come from the adjoint sweep (Eq. 5) and Eqs. 6-8.

The continuous adjoint is not the exact gradient of the discrete misfit, and three parts of
the discrete misfit have no continuous counterpart, so the comparison leaves them out and
compares at the scale of a few cells:
- nodes on the faces: the forward sweep never reads the model there (the faces are
  extrapolated from the interior), so the discrete derivative is exactly zero;
- nodes within two cells of the source's fixed set: the model there enters the factor T0
  (its s0, xi0, eta0 are interpolated at the source) and the fixed set, where T = T0;
- node-scale oscillation: the Lax-Friedrichs update couples each node to both neighbours
  along each axis, so the discrete sensitivity of one node alternates around the smooth
  continuous one. Both fields are therefore summed over the same w x w x w node boxes, which
  by linearity is the response to perturbing each box as a block.
Thresholds were computed once from the oracle (values in the parameter list) and frozen.

A second pin checks the kernels' gradient of T directly: for a traveltime field linear in
(theta, phi) every difference of Eqs. 7-8, central or one-sided on a face, is exact.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import tt_inputs as I


def _case(n, xi0, eta0, amp):
    """Heterogeneous anisotropic n^3 spherical grid (20 km deep, 0.18 x 0.18 deg), one
    source at 16 km, four surface receivers with absolute times and two common-source
    pairs."""
    g = I.GridSpec(n, n, n, 0.0, 20.0, 0.0, 0.18, 0.0, 0.18)
    s = 1.0 / (I.background_velocity(g) * (1 + 0.03 * I.checker(g, 1, 1, 1)))
    xi = xi0 + amp * I.checker(g, 1, 1, 1)
    eta = eta0 + amp * I.checker(g, 1, 1, 1, phase_cos_phi=True)
    src = np.array([16.0, 0.05, 0.06])
    rec = np.array([[0.0, 0.14, 0.12], [0.0, 0.12, 0.15], [0.0, 0.15, 0.05],
                    [0.0, 0.03, 0.16]])
    data = dict(abs_rec=np.arange(4), abs_tobs=np.array([3.0, 3.1, 2.9, 3.05]),
                abs_w=np.ones(4), cs_m=np.array([0, 2]), cs_i=np.array([1, 3]),
                cs_dtobs=np.array([0.05, -0.04]), cs_w=np.ones(2))
    return g, s, xi, eta, src, rec, data


def _single_node_fd(oracle, case, eps=1e-4, tol=1e-14):
    """Central differences of chi = chi_t + chi_cs with respect to ln s, xi and eta at each
    interior node, one node at a time. Every perturbed solve starts from the unperturbed tau
    (the fixed point does not depend on the start). The oracle's C calls release the GIL, so
    a thread pool runs the solves in parallel."""
    g, s, xi, eta, src, rec, data = case
    gd = g.as_dict()
    tau0 = oracle.forward(gd, s, xi, eta, src, tol, 5000)[0]

    def chi(m):
        _, T, _, conv, _ = oracle.forward(gd, m[0], m[1], m[2], src, tol, 5000, tau_init=tau0)
        assert conv
        ct, cc, _ = oracle.misfit(oracle.receiver_times(gd, T, rec), **data)
        return ct + cc

    def one(job):
        which, node = job
        out = []
        for sign in (1.0, -1.0):
            m = [s.copy(), xi.copy(), eta.copy()]
            if which == 0:
                m[0][node] *= 1.0 + sign * eps
            else:
                m[which][node] += sign * eps
            out.append(chi(m))
        return (out[0] - out[1]) / (2.0 * eps)

    jobs = [(w, node) for w in range(3) for node in np.ndindex(g.shape)
            if all(0 < node[d] < g.shape[d] - 1 for d in range(3))]
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        vals = list(ex.map(one, jobs))
    fd = np.zeros((3,) + g.shape)
    for (w, node), v in zip(jobs, vals):
        fd[(w,) + node] = v
    return fd


_FD_CACHE = {}


def _fd_and_kernels(oracle, xi0, eta0, amp):
    """(case, single-node differences, K dV) of the 13^3 case, computed once per module."""
    key = (xi0, eta0, amp)
    if key not in _FD_CACHE:
        case = _case(13, xi0, eta0, amp)
        _FD_CACHE[key] = (case, _single_node_fd(oracle, case), _kernels_dV(oracle, case))
    return _FD_CACHE[key]


def _kernels_dV(oracle, case):
    g, s, xi, eta, src, rec, data = case
    gd = g.as_dict()
    r = oracle.solve_source(gd, s, xi, eta, src, rec, data, tol_fwd=1e-14, tol_adj=1e-14,
                            max_iter=5000)
    assert r["conv_fwd"] and r["conv_adj"]
    K = [np.zeros(g.shape) for _ in range(3)]
    oracle.kernel_add(gd, s, r["T"], r["P"], *K)
    dV = oracle.node_volumes(gd)
    return np.stack([k * dV for k in K])


def _compare_mask(g, src, dmin):
    """Interior nodes at index (Chebyshev) distance >= dmin from the node nearest the
    source, the centre of the 3 x 3 x 3 fixed set."""
    depth, lat, lon = g.axes()
    c = [int(np.argmin(np.abs(a - v))) for a, v in zip((depth, lat, lon), src)]
    ii = np.meshgrid(*[np.arange(n) for n in g.shape], indexing="ij")
    dist = np.max([np.abs(ii[d] - c[d]) for d in range(3)], axis=0)
    inner = np.all([(ii[d] > 0) & (ii[d] < g.shape[d] - 1) for d in range(3)], axis=0)
    return inner & (dist >= dmin)


def _box_sums(f, w):
    """Sum of f over the w x w x w box centred on each node (zero outside the grid)."""
    h = w // 2
    p = np.pad(f, h)
    out = np.zeros_like(f)
    n0, n1, n2 = f.shape
    for a in range(w):
        for b in range(w):
            for c in range(w):
                out += p[a:a + n0, b:b + n1, c:c + n2]
    return out


def _agreement(fd, pred, mask, w):
    a, b = np.where(mask, fd, 0.0), np.where(mask, pred, 0.0)
    corr = np.corrcoef(_box_sums(a, w)[mask], _box_sums(b, w)[mask])[0, 1]
    summed = abs(b.sum() - a.sum()) / np.abs(a).sum()
    return corr, summed


@pytest.mark.parametrize(
    "xi0,eta0,amp,min_corr,max_sum",
    [
        # the benchmark's anisotropy (checkerboards of +-0.03): oracle 0.910 / 0.938 / 0.936
        # correlation, 0.006 / 0.029 / 0.025 summed disagreement (s, xi, eta)
        (0.0, 0.0, 0.03, 0.90, 0.10),
        # strong anisotropy (xi = 0.1, eta = 0.15, +-0.05): the O(h) difference between the
        # discrete and continuous gradients grows with the anisotropy; oracle 0.879 / 0.890 /
        # 0.861 and 0.011 / 0.151 / 0.136. This case is the one that separates a wrong sign
        # or axis of the adjoint's cross term or its xi factor (correlation 0.50-0.85).
        (0.1, 0.15, 0.05, 0.85, 0.20),
    ],
    ids=["benchmark-anisotropy", "strong-anisotropy"])
def test_single_node_fd_matches_kernels(oracle, xi0, eta0, amp, min_corr, max_sum):
    case, fd, pred = _fd_and_kernels(oracle, xi0, eta0, amp)
    mask = _compare_mask(case[0], case[4], 3)
    for which, name in enumerate(("s", "xi", "eta")):
        corr, summed = _agreement(fd[which], pred[which], mask, 3)
        assert corr >= min_corr, (name, corr)
        assert summed <= max_sum, (name, summed)


def test_single_node_fd_of_slowness_has_the_kernels_total(oracle):
    """Over every interior node outside the source's neighbourhood, the summed single-node
    derivatives in s equal the summed K_s dV within 3 % (13^3, benchmark anisotropy)."""
    case, fd, pred = _fd_and_kernels(oracle, 0.0, 0.0, 0.03)
    mask = _compare_mask(case[0], case[4], 3)
    assert np.sum(pred[0][mask]) / np.sum(fd[0][mask]) == pytest.approx(1.0, abs=0.03)


@pytest.mark.parametrize("flat", [0, 1])
def test_kernel_gradient_exact_for_linear_traveltime(oracle, flat):
    """T = a theta + b phi + c r (angles in radians): the index-space differences of Eqs. 7-8
    are exact for a linear field on every node, faces included, so with P = 1 the kernels
    are K_xi = g_t^2 - g_p^2 and K_eta = -2 g_t g_p with g_t = a / r, g_p = b / (r cos theta)
    (flat geometry: the metric factors are R_E)."""
    g = I.GridSpec(7, 9, 11, 0.0, 30.0, 40.0, 40.4, 10.0, 10.6, flat=flat)
    depth, lat, lon = g.axes()
    r = g.earth_radius_km - depth
    th, ph = np.deg2rad(lat), np.deg2rad(lon)
    a, b, c = 37.0, -23.0, 0.11
    R, TH, PH = np.meshgrid(r, th, ph, indexing="ij")
    T = a * TH + b * PH + c * R
    P = np.ones(g.shape)
    s = np.full(g.shape, 0.2)
    Ks, Kx, Ke = (np.zeros(g.shape) for _ in range(3))
    oracle.kernel_add(g.as_dict(), s, T, P, Ks, Kx, Ke)
    if flat:
        gt, gp = a / g.earth_radius_km, b / g.earth_radius_km
    else:
        gt, gp = a / R, b / (R * np.cos(TH))
    np.testing.assert_allclose(Kx, gt * gt - gp * gp, rtol=1e-9, atol=0)
    np.testing.assert_allclose(Ke, -2.0 * gt * gp * np.ones(g.shape), rtol=1e-9, atol=0)
    np.testing.assert_allclose(Ks, 0.04, rtol=1e-14)
