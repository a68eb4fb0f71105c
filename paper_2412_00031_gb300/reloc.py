"""Earthquake relocation (Eq. 10, Appendix B, Eqs. B1-B11) as a host driver of the C ABI.

By reciprocity the traveltime from event n to receiver m is Gamma_m(x_n), the time of a
wavefront started at receiver m. One batched forward solve with the receivers as the sources
(tt_forward) gives every Gamma_m on the grid; the model does not change while the events
move, so it is solved once. Each evaluation of the event positions x_n and origin times
tau_n then:
- reads Gamma_m and its gradient at every event (tt_field_at_points);
- forms the arrivals Gamma_m(x_n) + tau_n and their misfit and adjoint sources
  (tt_misfit_table, and tt_misfit_cr when common-receiver pairs are given, Eqs. 2-4 and
  A2-A4);
- sums the location and origin-time kernels (tt_reloc_kernels, Eqs. B5-B11).

Events move along the normalised gradient (tt_reloc_update). Step-size control follows the
model loop: a step that raises chi is undone and both step sizes are halved.

Every step of the arithmetic runs in the library's kernels. This module sequences the calls
and holds the buffers; it reads back one double per evaluation, the total misfit that
tt_misfit_total sums on the device.
"""
from . import (default_opts, tt_field_at_points, tt_forward, tt_misfit_cr, tt_misfit_table,
               tt_misfit_total, tt_reloc_kernels, tt_reloc_update)


class Relocation:
    """Buffers and calls of the relocation loop for one set of events, receivers and data.
    pts: float64 CUDA tensor [n_src, 3] (depth km, lat deg, lon deg), updated in place;
    otime: float64 CUDA tensor [n_src] of origin times (updated in place) or None to keep
    them at zero; data: DeviceData over the receivers (its n_src = the events)."""

    def __init__(self, ctx, model, grid_shape, data, pts, otime=None, cr=None, opts=None):
        import torch
        self.ctx, self.data, self.pts, self.otime, self.cr = ctx, data, pts, otime, cr
        s = model[0]
        self.opts = opts if opts is not None else default_opts(0 if s.dtype == torch.float32 else 1)
        n_src, n_rec, dev = pts.shape[0], data.n_rec, pts.device
        shape = tuple(grid_shape) + (n_rec,)
        tau = torch.empty(shape, dtype=s.dtype, device=dev)
        self.Gamma = torch.empty_like(tau)
        self.iters = tt_forward(ctx, model, data.rec, tau, self.Gamma, self.opts)
        del tau
        f64 = dict(dtype=torch.float64, device=dev)
        self.val = torch.empty((n_src, n_rec), **f64)
        self.grad = torch.empty((n_src, n_rec, 3), **f64)
        self.Tr = torch.empty((n_src, n_rec), **f64)
        self.chi = torch.empty((n_src, 2), **f64)
        self.chi_cr = torch.zeros(n_src, **f64)
        self.R = torch.empty((n_src, n_rec), **f64)
        self.Kx = torch.empty((n_src, 3), **f64)
        self.Kt = torch.empty(n_src, **f64)

    def evaluate(self):
        """chi at the current events; leaves their kernels in Kx and Kt."""
        c = self.ctx
        tt_field_at_points(c, self.Gamma, self.pts, self.val, self.grad)
        tt_misfit_table(c, self.val, self.otime, self.data, self.Tr, self.chi, self.R)
        if self.cr is not None:
            tt_misfit_cr(c, self.cr, self.Tr, self.chi_cr, self.R)
        tt_reloc_kernels(c, self.R, self.grad, self.Kx, self.Kt)
        # the step control's total misfit, an FP64 sum on the device
        return tt_misfit_total(c, self.chi, self.data.alpha, self.data.beta,
                               self.chi_cr if self.cr is not None else None,
                               self.cr.gamma if self.cr is not None else 0.0)

    def run(self, n_iter, step_km, step_s=0.0):
        """n_iter step attempts; returns the history [(chi, step_km, accepted)], first entry
        the starting events' chi."""
        chi = self.evaluate()
        hist = [(chi, step_km, True)]
        for _ in range(n_iter):
            saved = (self.pts.clone(), None if self.otime is None else self.otime.clone())
            tt_reloc_update(self.ctx, self.pts, self.otime, self.Kx, self.Kt, step_km, step_s)
            new = self.evaluate()
            if new < chi:
                chi = new
                hist.append((chi, step_km, True))
            else:
                self.pts.copy_(saved[0])
                if self.otime is not None:
                    self.otime.copy_(saved[1])
                hist.append((new, step_km, False))
                step_km *= 0.5
                step_s *= 0.5
                self.evaluate()
        return hist


def relocate(ctx, model, grid_shape, data, pts, otime=None, n_iter=10, step_km=2.0,
             step_s=0.2, cr=None, opts=None):
    """The relocation loop; pts (and otime) are updated in place. Returns Relocation.run's
    history."""
    r = Relocation(ctx, model, grid_shape, data, pts, otime, cr, opts)
    return r.run(n_iter, step_km, step_s)

