"""FP64 numpy oracle of the regularisation and model update of the inversion step (test
infrastructure only: the test suite, the smoke check and the benchmark's CPU-baseline leg
use it; the product never imports it).

Sec. 3.3 of the paper, written as its equations state them:
- inversion grids and their basis functions, Eqs. 11-14;
- projection of a kernel onto the basis, Eq. 17, and the expansion of coefficients back onto
  the forward grid, Eq. 15;
- kernel density, Eq. 19, and the normalisation of the kernels by it, Eq. 18;
- the model update of step 4 (Sec. 2).

Readings, where the paper leaves a choice open:
- Grid h of H (h = 0..H-1) has N nodes per axis at x_a = x_min + (a - h / H) dc,
  a = 0..N-1, with dc = (x_max - x_min) / (N - 2). Every grid then covers the forward
  domain, and the H grids are offset by dc / H from each other.
- The integral of Eq. 17 is the sum over the forward nodes of K B dV, with dV the node
  volume r^2 cos(theta) dr dtheta dphi.
- The update: s <- s (1 - a D_s / max|D_s|), xi <- xi - a D_xi / max|D_xi|, and likewise
  eta. D is the expansion (Eq. 15) of the projected kernels, and a is the step size. The
  kernels are derivatives with respect to ln s, xi and eta (Eq. 9). Step control: a step
  that raises chi is undone and a is halved.
"""
import numpy as np


def axis_basis(n_fine, n_coarse, H):
    """U[h, a, i]: the hat function of node a of inversion grid h (Eqs. 12-14) at forward node
    i of one axis, in the axis coordinate scaled to [0, 1]. The rising part exists only when
    node a - 1 belongs to the grid and the falling part only when node a + 1 does (the
    conditions of Eq. 12)."""
    x = np.arange(n_fine, dtype=np.float64) / (n_fine - 1)
    dc = 1.0 / (n_coarse - 2)
    U = np.zeros((H, n_coarse, n_fine))
    for h in range(H):
        xc = (np.arange(n_coarse, dtype=np.float64) - h / H) * dc
        for a in range(n_coarse):
            if a > 0:
                m = (x >= xc[a - 1]) & (x <= xc[a])
                U[h, a, m] = (x[m] - xc[a - 1]) / (xc[a] - xc[a - 1])
            if a < n_coarse - 1:
                m = (x >= xc[a]) & (x <= xc[a + 1])
                U[h, a, m] = (xc[a + 1] - x[m]) / (xc[a + 1] - xc[a])
    return U


def bases(shape, coarse, H):
    """Per-axis basis tables (r, theta, phi) of H grids of coarse = (N_r, N_t, N_p) nodes."""
    return tuple(axis_basis(n, c, H) for n, c in zip(shape, coarse))


def project(K, dV, B, H):
    """Eq. 17: G[h, a, b, c] = sum over forward nodes of K B^h_abc dV, with
    B^h_abc = u_a v_b w_c / H (Eq. 11)."""
    Ur, Ut, Up = B
    return np.stack([np.einsum("ijk,ai,bj,ck->abc", K * dV, Ur[h], Ut[h], Up[h]) / H
                     for h in range(H)])


def expand(G, B, H):
    """Eq. 15: D(x) = sum over h and l of G[h, l] B^h_l(x) at the forward nodes."""
    Ur, Ut, Up = B
    return sum(np.einsum("abc,ai,bj,ck->ijk", G[h], Ur[h], Ut[h], Up[h]) for h in range(H)) / H


def kernel_density(P_hat_list):
    """Eq. 19: K_d = sum over sources of the adjoint fields computed with R = 1."""
    return np.sum(np.stack(P_hat_list), axis=0)


def normalize(K, Kd, eps, zeta):
    """Eq. 18: K / (K_d + eps)^zeta."""
    return K / (Kd + eps) ** zeta


def update(s, xi, eta, Ds, Dxi, Deta, step):
    """The model update (reading in the module header)."""
    return (s * (1.0 - step * Ds / np.abs(Ds).max()),
            xi - step * Dxi / np.abs(Dxi).max(),
            eta - step * Deta / np.abs(Deta).max())
