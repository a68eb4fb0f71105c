"""tt_misfit_noalloc against tt_misfit (needs a GB300).

tt_misfit_noalloc serves callers that cannot allocate device memory when they call it (a
process whose HBM already belongs to its own pool allocator, or a stage that must not pay
cudaMalloc's device-wide synchronisation); it keeps its scratch in a static device array.
This file is collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.
"""
import numpy as np
import pytest

import tt_inputs as I
from gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_00031_gb300 as m
    return m


def _forward_and_reference(tt, w, dtype):
    """T from tt_forward and the misfit outputs of the context-based tt_misfit."""
    import torch
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    model = tuple(to_dev(a, dtype) for a in (w.s, w.xi, w.eta))
    tau = torch.empty(w.grid.shape + (w.n_src,), dtype=dtype, device="cuda")
    T = torch.empty_like(tau)
    tt.tt_forward(ctx, model, w.src, tau, T)
    data = tt.DeviceData.from_workload(w)
    out = [torch.empty((w.n_src, data.n_rec), dtype=torch.float64, device="cuda"),
           torch.empty((w.n_src, 2), dtype=torch.float64, device="cuda"),
           torch.empty((w.n_src, data.n_rec), dtype=torch.float64, device="cuda")]
    tt.tt_misfit(ctx, T, data, *out)
    torch.cuda.synchronize()
    ctx.close()
    return T, data, [o.cpu().numpy() for o in out]


def _noalloc(tt, w, T, data):
    import torch
    out = [torch.full((w.n_src, data.n_rec), np.nan, dtype=torch.float64, device="cuda"),
           torch.full((w.n_src, 2), np.nan, dtype=torch.float64, device="cuda"),
           torch.full((w.n_src, data.n_rec), np.nan, dtype=torch.float64, device="cuda")]
    tt.tt_misfit_noalloc(w.grid.as_dict(), T, data, *out)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in out]


def test_noalloc_misfit_matches_context_misfit_on_two_calls_in_a_row(tt):
    import torch
    # two different workloads (different grids, receiver counts, precisions), called back to
    # back, so that a result left in the shared scratch by the first call would show
    wa = I.small_case(31, shape=(13, 15, 17), n_src=4, n_rec=9)
    wb = I.small_case(32, shape=(11, 14, 12), n_src=3, n_rec=5)
    Ta, da, ref_a = _forward_and_reference(tt, wa, torch.float32)
    Tb, db, ref_b = _forward_and_reference(tt, wb, torch.float64)
    got_a = _noalloc(tt, wa, Ta, da)
    got_b = _noalloc(tt, wb, Tb, db)
    for got, ref in ((got_a, ref_a), (got_b, ref_b)):
        for g, r in zip(got, ref):
            assert np.all(np.isfinite(g))
            np.testing.assert_allclose(g, r, rtol=1e-12, atol=1e-12)


def test_noalloc_rejects_too_many_receivers(tt):
    import torch
    w = I.small_case(33, shape=(9, 9, 9), n_src=1, n_rec=tt.TT_NOALLOC_MAX_REC + 1)
    T = torch.zeros(w.grid.shape + (1,), dtype=torch.float32, device="cuda")
    data = tt.DeviceData.from_workload(w)
    R = torch.empty((1, data.n_rec), dtype=torch.float64, device="cuda")
    with pytest.raises(tt.TTError) as e:
        tt.tt_misfit_noalloc(w.grid.as_dict(), T, data, None, None, R)
    assert e.value.status == tt.TT_EINVAL
    assert "TT_NOALLOC_MAX_REC" in str(e.value)


def test_noalloc_rejects_a_grid_that_tt_ctx_create_rejects(tt):
    """Both entry points validate the grid with the same rules: a spherical grid reaching
    latitude 89 is refused (TT_EINVAL) by each."""
    import torch
    w = I.small_case(34, shape=(9, 9, 9), n_src=1, n_rec=3)
    g = w.grid.as_dict()
    g.update(lat_min_deg=88.0, lat_max_deg=89.5)
    with pytest.raises(tt.TTError) as e:
        tt.tt_ctx_create(g)
    assert e.value.status == tt.TT_EINVAL
    T = torch.zeros(w.grid.shape + (1,), dtype=torch.float32, device="cuda")
    data = tt.DeviceData.from_workload(w)
    R = torch.empty((1, data.n_rec), dtype=torch.float64, device="cuda")
    with pytest.raises(tt.TTError) as e:
        tt.tt_misfit_noalloc(g, T, data, None, None, R)
    assert e.value.status == tt.TT_EINVAL
    assert "invalid grid" in str(e.value)
