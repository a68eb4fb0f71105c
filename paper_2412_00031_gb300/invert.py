"""Gradient-descent inversion loop (step 4 of Sec. 2, with the regularisation of Sec. 3.3) as
a host driver of the C ABI. Each evaluation of a model:
- solves the batch (tt_forward, tt_misfit, and tt_misfit_cr when common-receiver pairs are
  given, Eqs. 2-4; tt_adjoint) and accumulates the kernels (tt_kernel, Eqs. 6-8);
- solves the adjoint again with R = 1 at every record of each source and sums those fields
  into the kernel density (tt_kernel_density, Eq. 19).

A descent direction is then formed:
- normalise the kernels (tt_kernel_normalize, Eq. 18), with eps = eps_rel max K_d;
- project each onto the inversion grids and expand it back (tt_mgrid_project /
  tt_mgrid_expand, Eqs. 15 and 17).

The model moves along the direction (tt_model_update). Step-size control (the reading of
the cited method, which the paper does not spell out): a step that raises chi is undone and
the step size halved.

Every step of the arithmetic runs in the library's kernels. This module sequences the calls
and holds the buffers; it reads back chi (n_src x 2) and the largest K_d to set eps.
"""
import numpy as np

from . import (default_opts, mgrid, tt_adjoint, tt_forward, tt_kernel, tt_kernel_density,
               tt_kernel_normalize, tt_mgrid_expand, tt_mgrid_project, tt_misfit,
               tt_misfit_cr, tt_model_update)


class Inversion:
    """Buffers and calls of the loop for one batch of sources, data and inversion grids."""

    def __init__(self, ctx, model, src, data, grid_shape, mg, opts=None, eps_rel=1e-2,
                 zeta=0.5, cr=None):
        import torch
        self.torch = torch
        self.ctx, self.model, self.src, self.data, self.mg = ctx, model, src, data, mg
        s = model[0]
        self.opts = opts if opts is not None else default_opts(0 if s.dtype == torch.float32 else 1)
        self.eps_rel, self.zeta = float(eps_rel), float(zeta)
        B, dev, F = len(src), s.device, s.dtype
        shape = tuple(grid_shape) + (B,)
        self.tau = torch.empty(shape, dtype=F, device=dev)
        self.T = torch.empty_like(self.tau)
        self.P = torch.empty_like(self.tau)
        self.Phat = torch.empty_like(self.tau)
        f64 = dict(dtype=torch.float64, device=dev)
        self.chi = torch.empty((B, 2), **f64)
        self.R = torch.empty((B, data.n_rec), **f64)
        self.cr = cr                                    # CrData or None
        self.Tr = torch.empty((B, data.n_rec), **f64)
        self.chi_cr = torch.zeros(B, **f64)
        # R = 1 at every record of each source (Eq. 19's adjoint sources)
        Rhat = np.zeros((B, data.n_rec))
        for b in range(B):
            Rhat[b, data.h_abs_rec[data.h_abs_off[b]:data.h_abs_off[b + 1]]] = 1.0
        self.Rhat = torch.as_tensor(Rhat, **f64)
        self.K = [torch.empty(tuple(grid_shape), **f64) for _ in range(3)]
        self.Kd = torch.empty(tuple(grid_shape), **f64)
        self.D = [torch.empty(tuple(grid_shape), **f64) for _ in range(3)]
        self.G = torch.empty((mg.n_grids, mg.n_r, mg.n_t, mg.n_p), **f64)

    def evaluate(self):
        """chi of the current model; leaves its kernels and kernel density in the buffers."""
        c, m, s = self.ctx, self.model, self.src
        tt_forward(c, m, s, self.tau, self.T, self.opts)
        tt_misfit(c, self.T, self.data, self.Tr, self.chi, self.R)
        if self.cr is not None:
            tt_misfit_cr(c, self.cr, self.Tr, self.chi_cr, self.R)
        tt_adjoint(c, m, s, self.T, self.data.rec, self.R, self.P, self.opts)
        for K in self.K:
            K.zero_()
        tt_kernel(c, m, self.T, self.P, *self.K)
        tt_adjoint(c, m, s, self.T, self.data.rec, self.Rhat, self.Phat, self.opts)
        self.Kd.zero_()
        tt_kernel_density(c, self.Phat, self.Kd)
        chi = self.chi.cpu().numpy()
        total = self.data.alpha * chi[:, 0].sum() + self.data.beta * chi[:, 1].sum()
        if self.cr is not None:
            total += self.cr.gamma * self.chi_cr.cpu().numpy().sum()
        return float(total)

    def direction(self):
        """The smoothed, density-normalised descent direction from the last evaluation."""
        eps = self.eps_rel * float(self.Kd.max())
        tt_kernel_normalize(self.ctx, *self.K, self.Kd, max(eps, 1e-300), self.zeta)
        for K, D in zip(self.K, self.D):
            tt_mgrid_project(self.ctx, self.mg, K, self.G)
            tt_mgrid_expand(self.ctx, self.mg, self.G, D)

    def run(self, n_iter, step):
        """n_iter step attempts; returns the history [(chi, step, accepted)], first entry the
        starting model's chi."""
        chi = self.evaluate()
        hist = [(chi, step, True)]
        self.direction()
        for _ in range(n_iter):
            saved = [a.clone() for a in self.model]
            tt_model_update(self.ctx, self.model, *self.D, step)
            new = self.evaluate()
            if new < chi:
                chi = new
                hist.append((chi, step, True))
                self.direction()
            else:
                for a, b in zip(self.model, saved):
                    a.copy_(b)
                hist.append((new, step, False))
                step *= 0.5
        return hist


def invert(ctx, model, src, data, grid_shape, n_r=11, n_t=11, n_p=11, n_grids=5, n_iter=10,
           step=0.02, opts=None, eps_rel=1e-2, zeta=0.5, cr=None):
    """The loop on n_grids offset inversion grids of n_r x n_t x n_p nodes; the model tensors
    are updated in place. Returns the history of Inversion.run."""
    inv = Inversion(ctx, model, src, data, grid_shape, mgrid(n_r, n_t, n_p, n_grids), opts,
                    eps_rel, zeta, cr)
    return inv.run(n_iter, step)
