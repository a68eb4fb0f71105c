"""Host logic of the inversion and relocation loops (paper_2412_00031_gb300/invert.py), with
the library's calls replaced by CPU stand-ins on a quadratic misfit (no GPU). The loop must:
- accept a step that lowers chi;
- undo a step that raises it, restoring the model bit for bit, and halve the step;
- move the events along the relocation direction, keep the moves that lower that batch's
  chi, undo the others and halve that batch's steps, and hand the new positions to the
  next forward solve.
"""
import numpy as np
import pytest
import torch


@pytest.fixture(scope="module")
def inv_mod():
    import __graft_entry__
    __graft_entry__._load_builder().build()
    import paper_2412_00031_gb300.invert as V
    return V


class _Data:
    """The fields of DeviceData that the loop reads."""

    def __init__(self, n_src, n_rec):
        self.n_rec = n_rec
        self.rec = np.zeros((n_rec, 3))
        self.h_abs_off = np.arange(n_src + 1) * n_rec
        self.h_abs_rec = np.tile(np.arange(n_rec), n_src)
        self.alpha, self.beta = 1.0, 1.0


def _mgrid():
    class M:
        n_grids, n_r, n_t, n_p = 1, 2, 2, 2
    return M()


def test_model_steps_are_accepted_or_undone_and_halved(inv_mod, monkeypatch):
    V = inv_mod
    shape = (3, 3, 3)
    target = torch.full(shape, 0.25, dtype=torch.float64)
    model = (torch.full(shape, 0.2, dtype=torch.float64), torch.zeros(shape, dtype=torch.float64),
             torch.zeros(shape, dtype=torch.float64))
    inv = V.Inversion(None, model, np.zeros((2, 3)), _Data(2, 4), shape, _mgrid(),
                      opts=object())
    chis = []

    def evaluate():
        chi = float(((model[0] - target) ** 2).sum())
        chis.append(chi)
        return chi

    def direction():                        # the descent direction of this quadratic misfit
        inv.D[0].copy_(model[0] - target)
        inv.D[1].zero_()
        inv.D[2].zero_()

    def update(ctx, m, Ds, Dxi, Deta, step):  # s <- s (1 - step Ds / max|Ds|)
        m[0].mul_(1 - step * Ds / Ds.abs().max())

    monkeypatch.setattr(inv, "evaluate", evaluate)
    monkeypatch.setattr(inv, "direction", direction)
    monkeypatch.setattr(V, "tt_model_update", update)
    before = model[0].clone()
    hist = inv.run(6, 0.8)
    # 0.2 -> 0.2 (1 + 0.8) = 0.36 overshoots the target 0.25 and raises chi: undone, halved
    assert hist[1][2] is False and hist[1][1] == 0.8
    assert hist[2][1] == 0.4
    accepted = [h for h in hist if h[2]]
    assert all(b[0] < a[0] for a, b in zip(accepted[:-1], accepted[1:]))
    assert accepted[-1][0] < 0.5 * accepted[0][0]
    # a rejected step leaves the model exactly as it was
    inv2 = V.Inversion(None, model, np.zeros((2, 3)), _Data(2, 4), shape, _mgrid(), opts=object())
    model[0].copy_(before)
    monkeypatch.setattr(inv2, "evaluate", lambda: float(((model[0] - target) ** 2).sum()))
    monkeypatch.setattr(inv2, "direction", lambda: inv2.D[0].copy_(model[0] - target))
    h2 = inv2.run(1, 0.8)
    assert h2[1][2] is False and torch.equal(model[0], before)


def test_relocation_steps_keep_what_lowers_chi(inv_mod, monkeypatch):
    V = inv_mod
    shape = (3, 3, 3)
    model = tuple(torch.zeros(shape, dtype=torch.float64) for _ in range(3))
    src = np.array([[10.0, 0.5, 0.5], [20.0, 0.4, 0.6]])
    true = torch.tensor([[12.0, 0.5, 0.5], [19.0, 0.4, 0.6]], dtype=torch.float64)
    inv = V.Inversion(None, model, src, _Data(2, 4), shape, _mgrid(), opts=object(),
                      relocate=(5.0, 0.1))
    bt = inv.batches[0]
    fwd_src = []
    monkeypatch.setattr(V, "tt_forward", lambda c, m, s, tau, T, o: fwd_src.append(np.array(s)))

    def reloc_chi(b):                       # chi and its gradient in depth
        d = b.pts[:, 0] - true[:, 0]
        b.Kx.zero_()
        b.Kx[:, 0] = 2 * d
        b.Kt.zero_()
        return float((d ** 2).sum())

    def update(ctx, pts, otime, Kx, Kt, step_km, step_s):   # normalised step in depth
        pts[:, 0] -= step_km * Kx[:, 0] / Kx.abs().max()

    monkeypatch.setattr(inv, "_reloc_chi", reloc_chi)
    monkeypatch.setattr(V, "tt_reloc_update", update)
    for _ in range(6):
        inv.relocate_events()
    hist = inv.reloc_hist
    # the first step of 5 km moves the 2 km-deep miss by 5 km (chi 5 -> 11.25): undone, halved
    assert hist[0][2] is False and bt.rstep[0] < 5.0
    assert all((after < before) == ok for before, after, ok in hist)
    assert any(ok for _, _, ok in hist)
    err = (torch.as_tensor(bt.src)[:, 0] - true[:, 0]).abs().max()
    assert err < 0.5
    # each relocation solves the receivers in the current model, and the next forward
    # solve of the batch sees the moved events
    assert len(fwd_src) == 6
    assert np.array_equal(bt.src, bt.pts.numpy())
