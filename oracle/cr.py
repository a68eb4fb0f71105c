"""FP64 oracle of the common-receiver differential-time misfit (test infrastructure only).

Eq. 4: chi_cr = sum over ordered source pairs (n, j) and receivers m of
w_{nj,m} / 2 ((T_n(x_m) - T_j(x_m)) - (T_n^obs(x_m) - T_j^obs(x_m)))^2, and its adjoint
source, Eq. A4: dchi_cr / dT_n(x_m) = 2 sum_j w_{nj,m} (...), for symmetric weights. Written
as those sums, one term at a time.
"""
import numpy as np


def misfit_cr(Tr, Tobs, W, gamma=1.0):
    """Tr, Tobs: [n_src][n_rec] synthetic and observed receiver times; W: [n_src][n_src][n_rec]
    symmetric weights w_{nj,m} (W[n, n] = 0). Returns (chi_cr, share, R): the misfit, each
    source's ordered terms (share[n] = the terms with first index n; they sum to chi_cr) and
    gamma dchi_cr / dT (Eq. A4)."""
    ns, nr = Tr.shape
    share = np.zeros(ns)
    R = np.zeros((ns, nr))
    for n in range(ns):
        for j in range(ns):
            for m in range(nr):
                w = W[n, j, m]
                if w == 0.0:
                    continue
                e = (Tr[n, m] - Tr[j, m]) - (Tobs[n, m] - Tobs[j, m])
                share[n] += 0.5 * w * e * e
                R[n, m] += gamma * 2.0 * w * e
    return share.sum(), share, R
