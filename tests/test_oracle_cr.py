"""Pins of the common-receiver misfit oracle (oracle/cr.py): the adjoint source is the
derivative of the misfit (central differences, exact for a quadratic), the misfit vanishes
for perfect data and under receiver statics (Eq. 4 only sees differences between sources at
one receiver), and the pair count and sign for two sources by hand."""
import numpy as np

from oracle.cr import misfit_cr


def _case(seed, ns=4, nr=3):
    rng = np.random.default_rng(seed)
    Tr = rng.uniform(5, 20, (ns, nr))
    Tobs = Tr + rng.normal(0, 0.3, (ns, nr))
    W = rng.uniform(0, 1, (ns, ns, nr)) * (rng.uniform(size=(ns, ns, nr)) > 0.3)
    W = 0.5 * (W + W.transpose(1, 0, 2))
    for n in range(ns):
        W[n, n] = 0.0
    return Tr, Tobs, W


def test_adjoint_source_is_the_derivative():
    Tr, Tobs, W = _case(1)
    chi, _, R = misfit_cr(Tr, Tobs, W, gamma=1.0)
    h = 1e-4
    for n in range(Tr.shape[0]):
        for m in range(Tr.shape[1]):
            Tp, Tm = Tr.copy(), Tr.copy()
            Tp[n, m] += h; Tm[n, m] -= h
            fd = (misfit_cr(Tp, Tobs, W)[0] - misfit_cr(Tm, Tobs, W)[0]) / (2 * h)
            assert abs(fd - R[n, m]) <= 1e-7 * max(1.0, abs(fd))


def test_perfect_data_and_receiver_statics():
    Tr, _, W = _case(2)
    chi, share, R = misfit_cr(Tr, Tr.copy(), W)
    assert chi == 0.0 and not R.any()
    # a time shift common to every source at one receiver (a receiver static) cancels in
    # every difference of Eq. 4
    statics = np.array([0.7, -1.3, 2.5])
    chi, _, R = misfit_cr(Tr + statics[None, :], Tr, W)
    assert chi <= 1e-20 and np.abs(R).max() <= 1e-12
    # a shift of one source's times does not
    shifted = Tr.copy()
    shifted[1] += 0.5
    assert misfit_cr(shifted, Tr, W)[0] > 1e-3


def test_two_sources_by_hand():
    Tr = np.array([[10.0], [12.0]])
    Tobs = np.array([[10.5], [12.0]])
    W = np.zeros((2, 2, 1)); W[0, 1, 0] = W[1, 0, 0] = 0.5
    chi, share, R = misfit_cr(Tr, Tobs, W, gamma=2.0)
    e = (10.0 - 12.0) - (10.5 - 12.0)             # -0.5, and +0.5 for the pair (1, 0)
    assert abs(chi - 2 * 0.5 * 0.5 * e * e) <= 1e-15      # two ordered terms
    assert abs(share[0] - share[1]) <= 1e-15
    assert abs(R[0, 0] - 2.0 * 2 * 0.5 * e) <= 1e-15 and abs(R[1, 0] + R[0, 0]) <= 1e-15
