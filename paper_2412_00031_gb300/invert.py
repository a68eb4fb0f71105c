"""Gradient-descent inversion loop (step 4 of Sec. 2, with the regularisation of Sec. 3.3) as
a host driver of the C ABI. Each evaluation of a model:
- solves each batch of sources (tt_forward, tt_misfit, and tt_misfit_cr when
  common-receiver pairs are given, Eqs. 2-4; tt_adjoint) and accumulates the kernels
  (tt_kernel, Eqs. 6-8);
- solves the adjoint again with R = 1 at every record of each source and sums those fields
  into the kernel density (tt_kernel_density, Eq. 19).

A descent direction is then formed:
- normalise the kernels (tt_kernel_normalize_rel, Eq. 18), with eps = eps_rel max K_d (the
  maximum taken on the device);
- project each onto the inversion grids and expand it back (tt_mgrid_project /
  tt_mgrid_expand, Eqs. 15 and 17).

The model moves along the direction (tt_model_update). Step-size control (the reading of
the cited method, which the paper does not spell out): a step that raises chi is undone and
the step size halved.

With relocate = (step_km, step_s) the hypocentres and origin times are updated during the
inversion too (Sec. 2, Eq. 10). The arrivals become T_n(x_m) + tau_n, so the misfit of each
batch is taken from the table of receiver times plus origin times (tt_misfit_table). After
each model step, the receivers are solved as sources in the current model (tt_forward,
reciprocity) and each batch's events take one gradient step (tt_field_at_points,
tt_reloc_kernels, tt_reloc_update). A step that raises that batch's chi is undone and its
step sizes halved.

Every step of the arithmetic runs in the library's kernels, the step-control reductions
included (tt_misfit_total: each batch's total misfit as an FP64 sum on the device; the largest
K_d inside tt_kernel_normalize_rel). This module sequences the calls and holds the buffers;
it reads back one total misfit per batch.
"""
import numpy as np

from . import (default_opts, mgrid, tt_adjoint, tt_field_at_points, tt_forward, tt_kernel,
               tt_kernel_density, tt_kernel_normalize_rel, tt_mgrid_expand, tt_mgrid_project,
               tt_misfit, tt_misfit_cr, tt_misfit_table, tt_misfit_total, tt_model_update,
               tt_reloc_kernels, tt_reloc_update)


class _Batch:
    """One batch's sources, data and per-batch buffers."""

    def __init__(self, torch, src, data, cr, dev):
        B = len(src)
        f64 = dict(dtype=torch.float64, device=dev)
        self.src, self.data, self.cr = src, data, cr
        self.chi = torch.empty((B, 2), **f64)
        self.R = torch.empty((B, data.n_rec), **f64)
        self.Tr = torch.empty((B, data.n_rec), **f64)
        self.chi_cr = torch.zeros(B, **f64)
        # R = 1 at every record of each source (Eq. 19's adjoint sources)
        Rhat = np.zeros((B, data.n_rec))
        for b in range(B):
            Rhat[b, data.h_abs_rec[data.h_abs_off[b]:data.h_abs_off[b + 1]]] = 1.0
        self.Rhat = torch.as_tensor(Rhat, **f64)

    def enable_relocation(self, torch, dev, step_km, step_s):
        """Device copies of the event positions and origin times, and the relocation
        buffers."""
        B, nr = len(self.src), self.data.n_rec
        f64 = dict(dtype=torch.float64, device=dev)
        self.pts = torch.as_tensor(np.asarray(self.src, dtype=np.float64), **f64).contiguous()
        self.otime = torch.zeros(B, **f64)
        self.rstep = [float(step_km), float(step_s)]
        self.Tra = torch.empty((B, nr), **f64)
        self.val = torch.empty((B, nr), **f64)
        self.grad = torch.empty((B, nr, 3), **f64)
        self.chi_r = torch.empty((B, 2), **f64)
        self.R_r = torch.empty((B, nr), **f64)
        self.chi_cr_r = torch.zeros(B, **f64)
        self.Kx = torch.empty((B, 3), **f64)
        self.Kt = torch.empty(B, **f64)


class Inversion:
    """Buffers and calls of the loop for the sources, data and inversion grids. The sources
    come as one batch (src, data, cr) or as several: batches = [(src, data, cr), ...], each
    solved in turn on shared field buffers, with the kernels, kernel density and chi summed
    over all of them. A batch's cr pairs stay within it; cr_all (a CrData over all sources,
    numbered in batch order) holds pairs across batches. Then every batch's traveltime field
    is kept until the receiver-time tables of all batches give the common-receiver adjoint
    sources (Eq. A4), and the adjoints follow."""

    def __init__(self, ctx, model, src, data, grid_shape, mg, opts=None, eps_rel=1e-2,
                 zeta=0.5, cr=None, batches=None, relocate=None, cr_all=None):
        import torch
        self.torch = torch
        self.ctx, self.model, self.mg = ctx, model, mg
        s = model[0]
        self.opts = opts if opts is not None else default_opts(0 if s.dtype == torch.float32 else 1)
        self.eps_rel, self.zeta = float(eps_rel), float(zeta)
        dev, F = s.device, s.dtype
        if batches is None:
            batches = [(src, data, cr)]
        self.batches = [_Batch(torch, b_src, b_data, b_cr, dev) for b_src, b_data, b_cr in batches]
        Bmax = max(len(b.src) for b in self.batches)
        self.shape = tuple(grid_shape)
        self.buf = [torch.empty(self.shape + (Bmax,), dtype=F, device=dev) for _ in range(4)]
        f64 = dict(dtype=torch.float64, device=dev)
        self.K = [torch.empty(self.shape, **f64) for _ in range(3)]
        self.Kd = torch.empty(self.shape, **f64)
        self.D = [torch.empty(self.shape, **f64) for _ in range(3)]
        self.G = torch.empty((mg.n_grids, mg.n_r, mg.n_t, mg.n_p), **f64)
        self.cr_all = cr_all
        if cr_all is not None:
            assert all(b.cr is None for b in self.batches), "cr pairs go in cr_all"
            n_all = sum(len(b.src) for b in self.batches)
            n_rec = self.batches[0].data.n_rec
            assert cr_all.n_src == n_all and cr_all.n_rec == n_rec
            # the traveltime fields of all batches, kept until the adjoints
            self.T_all = [torch.empty(self.shape + (len(b.src),), dtype=F, device=dev)
                          for b in self.batches]
            self.Tr_all = torch.empty((n_all, n_rec), **f64)
            self.R_all = torch.empty((n_all, n_rec), **f64)
            self.chi_cr_all = torch.zeros(n_all, **f64)
            self.chi_zero_all = torch.zeros((n_all, 2), **f64)   # no chi_t / chi_cs terms
        self.relocate = relocate is not None
        self.reloc_hist = []
        if self.relocate:
            rec = self.batches[0].data.rec
            for bt in self.batches:
                assert np.array_equal(bt.data.rec, rec), "batches must share the receiver list"
                bt.enable_relocation(torch, dev, *relocate)
            self.rec = rec
            self.tauG = torch.empty(self.shape + (len(rec),), dtype=F, device=dev)
            self.Gam = torch.empty_like(self.tauG)
            if cr_all is not None:
                # common-receiver pairs across batches in the relocation too: the events'
                # positions, origin times, arrival tables, adjoint sources and kernels of all
                # batches in joined arrays, each batch's buffers views of its rows
                def joined(name):
                    return torch.cat([getattr(b, name) for b in self.batches]).contiguous()
                self.pts_all, self.otime_all = joined("pts"), joined("otime")
                self.Tra_all, self.Rr_all = joined("Tra"), joined("R_r")
                self.Kx_all, self.Kt_all = joined("Kx"), joined("Kt")
                self.chi_cr_r_all = torch.zeros(n_all, **f64)
                self.rstep = [float(relocate[0]), float(relocate[1])]
                views = {"pts": self.pts_all, "otime": self.otime_all, "Tra": self.Tra_all,
                         "R_r": self.Rr_all, "Kx": self.Kx_all, "Kt": self.Kt_all}
                row = 0
                for bt in self.batches:
                    B = len(bt.src)
                    for name, buf in views.items():
                        setattr(bt, name, buf[row:row + B])
                    row += B

    def _fields(self, B):
        """tau, T, P, P_hat views for a batch of B sources (node-major, source fastest)."""
        return [b.view(-1)[:int(np.prod(self.shape)) * B].view(self.shape + (B,))
                for b in self.buf]

    def evaluate(self):
        """chi of the current model; leaves the kernels and kernel density of all batches in
        the buffers."""
        c, m = self.ctx, self.model
        for K in self.K:
            K.zero_()
        self.Kd.zero_()
        total = 0.0
        if self.cr_all is not None:
            total += self._forward_all()
        for q, bt in enumerate(self.batches):
            tau, T, P, Phat = self._fields(len(bt.src))
            if self.cr_all is not None:
                T = self.T_all[q]
            else:
                bt.iters_fwd = tt_forward(c, m, bt.src, tau, T, self.opts)
                self._misfit(bt, T)
            bt.iters_adj = tt_adjoint(c, m, bt.src, T, bt.data.rec, bt.R, P, self.opts)
            tt_kernel(c, m, T, P, *self.K)
            tt_adjoint(c, m, bt.src, T, bt.data.rec, bt.Rhat, Phat, self.opts)
            tt_kernel_density(c, Phat, self.Kd)
            total += tt_misfit_total(c, bt.chi, bt.data.alpha, bt.data.beta,
                                     bt.chi_cr if bt.cr is not None else None,
                                     bt.cr.gamma if bt.cr is not None else 0.0)
        return float(total)

    def _misfit(self, bt, T):
        """The batch's receiver times, misfit and adjoint sources (within-batch cr pairs);
        returns the table of arrivals."""
        c = self.ctx
        tt_misfit(c, T, bt.data, bt.Tr, bt.chi, bt.R)
        Tr = bt.Tr
        if self.relocate:                       # arrivals with the origin times
            tt_misfit_table(c, bt.Tr, bt.otime, bt.data, bt.Tra, bt.chi, bt.R)
            Tr = bt.Tra
        if bt.cr is not None:
            tt_misfit_cr(c, bt.cr, Tr, bt.chi_cr, bt.R)
        return Tr

    def _forward_all(self):
        """Forward solves and misfits of every batch, then the common-receiver terms across
        batches on the joined tables; each batch's R gets its rows back. Returns gamma chi_cr."""
        c, m = self.ctx, self.model
        row = 0
        for q, bt in enumerate(self.batches):
            tau = self._fields(len(bt.src))[0]
            bt.iters_fwd = tt_forward(c, m, bt.src, tau, self.T_all[q], self.opts)
            Tr = self._misfit(bt, self.T_all[q])
            B = len(bt.src)
            self.Tr_all[row:row + B].copy_(Tr)
            self.R_all[row:row + B].copy_(bt.R)
            row += B
        tt_misfit_cr(c, self.cr_all, self.Tr_all, self.chi_cr_all, self.R_all)
        row = 0
        for bt in self.batches:
            B = len(bt.src)
            bt.R.copy_(self.R_all[row:row + B])
            row += B
        return tt_misfit_total(c, self.chi_zero_all, 0.0, 0.0, self.chi_cr_all,
                               self.cr_all.gamma)

    def direction(self):
        """The smoothed, density-normalised descent direction from the last evaluation."""
        tt_kernel_normalize_rel(self.ctx, *self.K, self.Kd, self.eps_rel, self.zeta)
        for K, D in zip(self.K, self.D):
            tt_mgrid_project(self.ctx, self.mg, K, self.G)
            tt_mgrid_expand(self.ctx, self.mg, self.G, D)

    def _reloc_chi(self, bt):
        """chi of a batch's events from the receiver-started fields; leaves K_x, K_tau."""
        c = self.ctx
        tt_field_at_points(c, self.Gam, bt.pts, bt.val, bt.grad)
        tt_misfit_table(c, bt.val, bt.otime, bt.data, bt.Tra, bt.chi_r, bt.R_r)
        if bt.cr is not None:
            tt_misfit_cr(c, bt.cr, bt.Tra, bt.chi_cr_r, bt.R_r)
        tt_reloc_kernels(c, bt.R_r, bt.grad, bt.Kx, bt.Kt)
        return tt_misfit_total(c, bt.chi_r, bt.data.alpha, bt.data.beta,
                               bt.chi_cr_r if bt.cr is not None else None,
                               bt.cr.gamma if bt.cr is not None else 0.0)

    def _reloc_chi_all(self):
        """chi of all events when common-receiver pairs span batches: each batch's arrivals
        and misfit, then Eqs. 4 and A4 on the joined arrival table (adding into the joined
        adjoint sources), then each batch's K_x, K_tau. Returns the total chi."""
        c = self.ctx
        total = 0.0
        for bt in self.batches:
            tt_field_at_points(c, self.Gam, bt.pts, bt.val, bt.grad)
            tt_misfit_table(c, bt.val, bt.otime, bt.data, bt.Tra, bt.chi_r, bt.R_r)
            total += tt_misfit_total(c, bt.chi_r, bt.data.alpha, bt.data.beta)
        tt_misfit_cr(c, self.cr_all, self.Tra_all, self.chi_cr_r_all, self.Rr_all)
        total += tt_misfit_total(c, self.chi_zero_all, 0.0, 0.0, self.chi_cr_r_all,
                                 self.cr_all.gamma)
        for bt in self.batches:
            tt_reloc_kernels(c, bt.R_r, bt.grad, bt.Kx, bt.Kt)
        return total

    def relocate_events(self):
        """One relocation step of every batch's events in the current model. With pairs
        across batches (cr_all) all events take one joint step, normalised over all of them,
        and the step control acts on the total chi."""
        tt_forward(self.ctx, self.model, self.rec, self.tauG, self.Gam, self.opts)
        if self.cr_all is not None:
            before = self._reloc_chi_all()
            saved = (self.pts_all.clone(), self.otime_all.clone())
            tt_reloc_update(self.ctx, self.pts_all, self.otime_all, self.Kx_all, self.Kt_all,
                            *self.rstep)
            after = self._reloc_chi_all()
            if after >= before:
                self.pts_all.copy_(saved[0])
                self.otime_all.copy_(saved[1])
                self.rstep = [s * 0.5 for s in self.rstep]
            self.reloc_hist.append((before, after, after < before))
            for bt in self.batches:
                bt.src = bt.pts.cpu().numpy()
            return
        for bt in self.batches:
            before = self._reloc_chi(bt)
            saved = (bt.pts.clone(), bt.otime.clone())
            tt_reloc_update(self.ctx, bt.pts, bt.otime, bt.Kx, bt.Kt, *bt.rstep)
            after = self._reloc_chi(bt)
            if after >= before:
                bt.pts.copy_(saved[0])
                bt.otime.copy_(saved[1])
                bt.rstep = [s * 0.5 for s in bt.rstep]
            self.reloc_hist.append((before, after, after < before))
            bt.src = bt.pts.cpu().numpy()

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
            if self.relocate:                   # move the events, then refresh chi and kernels
                self.relocate_events()
                chi = self.evaluate()
                self.direction()
        return hist


def invert(ctx, model, src, data, grid_shape, n_r=11, n_t=11, n_p=11, n_grids=5, n_iter=10,
           step=0.02, opts=None, eps_rel=1e-2, zeta=0.5, cr=None, batches=None, relocate=None,
           cr_all=None):
    """The loop on n_grids offset inversion grids of n_r x n_t x n_p nodes; the model tensors
    are updated in place. Returns the history of Inversion.run."""
    inv = Inversion(ctx, model, src, data, grid_shape, mgrid(n_r, n_t, n_p, n_grids), opts,
                    eps_rel, zeta, cr, batches, relocate, cr_all)
    return inv.run(n_iter, step)
