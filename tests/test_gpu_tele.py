"""Teleseismic events on the GPU (reading R17) against the FP64 oracle (oracle/tele.py),
through the C ABI (needs a GB300): the 2-D traveltimes of several events in three 1-D models
(FP64 to 1e-10 of the largest time with the same iteration counts, FP32 to the 1e-5 bar),
their interpolation onto a region's nodes, and the region's solve with those faces held
fixed (the whole chain against the oracle's chain)."""
import numpy as np
import pytest

import tt_inputs as I

pytestmark = pytest.mark.gpu

RE = 6371.0


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_00031_gb300 as m
    return m


def _models(n_r, r_min):
    r = np.linspace(r_min, RE, n_r)
    return {"homogeneous": np.full(n_r, 1 / 8.0),
            "v = c r": 1 / ((8.0 / RE) * r),
            "layered": 1 / (5.8 + 3.0 * (RE - r) / (RE - r_min) + 0.2 * np.sin((RE - r) / 37.0))}


@pytest.mark.parametrize("name", ["homogeneous", "v = c r", "layered"])
def test_2d_times_match_the_oracle(tt, name):
    import torch
    import oracle.tele as TL
    n_r, n_d, r_min, dmax = 61, 97, RE - 400.0, 15.0
    s_r = _models(n_r, r_min)[name]
    r_src = np.array([RE - 35.0, RE - 120.0, RE - 333.3])
    for dtype, tol, bar in ((torch.float64, 1e-10, 1e-10), (torch.float32, 1e-6, 1e-5)):
        T = torch.empty((len(r_src), n_r, n_d), dtype=dtype, device="cuda")
        it = tt.tt_tele2d(_ctx(tt), torch.as_tensor(s_r, dtype=dtype, device="cuda"), r_min, RE,
                          dmax, r_src, T, tol=tol, max_iter=500)
        Tg = T.double().cpu().numpy()
        s_ref = torch.as_tensor(s_r, dtype=dtype).double().numpy()
        for e, rs in enumerate(r_src):
            ref, it_o, conv = TL.tele2d(r_min, RE, n_r, dmax, n_d, s_ref, rs, tol=1e-10,
                                        max_iter=500)
            assert conv
            assert np.abs(Tg[e] - ref).max() <= bar * ref.max(), (name, dtype, e)
            if dtype == torch.float64:
                assert abs(int(it[e]) - it_o) <= 1


_CTX = {}


def _ctx(tt):
    if "c" not in _CTX:
        _CTX["c"] = tt.tt_ctx_create(I.GridSpec(11, 11, 11, 0.0, 40.0, 0.0, 1.0, 0.0, 1.0).as_dict())
    return _CTX["c"]


def test_region_times_match_the_oracle(tt):
    import torch
    import oracle.tele as TL
    n_r, n_d, r_min, dmax = 61, 97, RE - 400.0, 15.0
    s_r = _models(n_r, r_min)["layered"]
    events = np.array([[100.0, -6.0, 3.0], [30.0, 9.0, -4.0]])
    g = I.GridSpec(13, 14, 15, 0.0, 40.0, 0.0, 1.0, 0.0, 1.2)
    ctx = tt.tt_ctx_create(g.as_dict())
    T2 = torch.empty((2, n_r, n_d), dtype=torch.float64, device="cuda")
    tt.tt_tele2d(ctx, torch.as_tensor(s_r, device="cuda"), r_min, RE, dmax, RE - events[:, 0],
                 T2, tol=1e-10)
    T = torch.empty(g.shape + (2,), dtype=torch.float64, device="cuda")
    tt.tt_tele_region_times(ctx, T2, r_min, RE, dmax, events, T)
    T2h = T2.cpu().numpy()
    for e in range(2):
        ref = TL.region_times(g.as_dict(), T2h[e], r_min, RE, dmax, events[e, 1], events[e, 2])
        assert np.abs(T.cpu().numpy()[..., e] - ref).max() <= 1e-12 * ref.max()
    # an event beyond the 2-D grid's reach is refused
    with pytest.raises(tt.TTError, match="farther"):
        tt.tt_tele_region_times(ctx, T2, r_min, RE, 2.0, events, T)
    ctx.close()


def test_region_solve_matches_the_oracle_chain(tt):
    """The whole chain on the GPU (2-D solves, face data, the region's solve with the faces
    held fixed) against the oracle's own chain, on a heterogeneous anisotropic region with
    two events: FP64 to 1e-9 of the largest time with iteration counts within 1, FP32 to
    the 1e-5 bar."""
    import torch
    import oracle.tele as TL
    n_r, n_d, r_min, dmax = 61, 97, RE - 400.0, 15.0
    s_r = _models(n_r, r_min)["layered"]
    events = np.array([[100.0, -6.0, 3.0], [30.0, 9.0, -4.0]])
    w = I.small_case(97, shape=(11, 12, 13), n_src=1, depth_max=40.0, extent_deg=1.0)
    g = w.grid
    gd = g.as_dict()
    ref, ref_it = [], []
    for e in range(2):
        T2o, _, conv = TL.tele2d(r_min, RE, n_r, dmax, n_d, s_r, RE - events[e, 0], tol=1e-10)
        assert conv
        start = TL.region_times(gd, T2o, r_min, RE, dmax, events[e, 1], events[e, 2])
        To, it, conv = TL.forward_tele(gd, w.s, w.xi, w.eta, start, tol=1e-11, max_iter=500)
        assert conv
        ref.append(To)
        ref_it.append(it)
    ctx = tt.tt_ctx_create(gd)
    for dtype, code, bar in ((torch.float64, tt.TT_F64, 1e-9), (torch.float32, tt.TT_F32, 1e-5)):
        T2 = torch.empty((2, n_r, n_d), dtype=dtype, device="cuda")
        tt.tt_tele2d(ctx, torch.as_tensor(s_r, dtype=dtype, device="cuda"), r_min, RE, dmax,
                     RE - events[:, 0], T2, tol=1e-11 if code == tt.TT_F64 else 1e-6)
        T = torch.empty(g.shape + (2,), dtype=dtype, device="cuda")
        tt.tt_tele_region_times(ctx, T2, r_min, RE, dmax, events, T)
        model = tuple(torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")
                      for a in (w.s, w.xi, w.eta))
        # FP32 resolves T of order 100 s to ~1e-5 s (one unit in the last place): its
        # convergence tolerance is a few of those
        o = tt.default_opts(code, tol_fwd=1e-11 if code == tt.TT_F64 else 3e-5,
                            max_iter_fwd=500)
        it = tt.tt_forward_tele(ctx, model, T, o)
        Tg = T.double().cpu().numpy()
        for e in range(2):
            assert np.abs(Tg[..., e] - ref[e]).max() <= bar * ref[e].max(), (dtype, e)
            if code == tt.TT_F64:
                assert abs(int(it[e]) - ref_it[e]) <= 1
    ctx.close()
