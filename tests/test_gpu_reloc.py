"""Earthquake location and origin-time kernels on the GPU (Eq. 10, Eqs. B1-B11, reading R15)
against the FP64 oracle (oracle/reloc.py), through the C ABI (needs a GB300).

- values and gradients of batched fields at points (interior, on nodes, faces and corners;
  FP32 and FP64 fields), element by element; a point outside the grid is refused;
- the misfit and adjoint sources from a table of arrivals with origin times, with absolute,
  common-source and common-receiver data;
- the kernel sums and the event update;
- the loop: observations from the oracle's FP64 solves from the true events; the GPU
  relocates perturbed events (receiver-started solves, then kernels and updates) and the
  oracle's kernels at the start (from its own receiver-started solves) match the GPU's.
"""
import numpy as np
import pytest

import tt_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_00031_gb300 as m
    return m


def _dev(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def _grid():
    return I.GridSpec(9, 13, 11, 0.0, 40.0, 10.0, 11.0, 20.0, 21.5)


def _special_points(g, rng, n):
    lo = np.array([g.depth_min_km, g.lat_min_deg, g.lon_min_deg])
    hi = np.array([g.depth_max_km, g.lat_max_deg, g.lon_max_deg])
    pts = list(lo + (hi - lo) * rng.uniform(0, 1, (n, 3)))
    pts += [lo, hi, [lo[0], hi[1], lo[2]], [hi[0], lo[1], hi[2]]]              # corners
    pts += [[g.depth_min_km, 10.4, 20.6], [g.depth_max_km, 10.7, 21.1]]           # faces
    node = [g.depth_max_km - 3 * (g.depth_max_km - g.depth_min_km) / (g.n_r - 1),
            g.lat_min_deg + 5 * (g.lat_max_deg - g.lat_min_deg) / (g.n_t - 1),
            g.lon_min_deg + 7 * (g.lon_max_deg - g.lon_min_deg) / (g.n_p - 1)]
    pts.append(node)                                                             # on a node
    return np.array(pts)


def test_field_at_points_matches_oracle(tt):
    import torch
    import oracle.reloc as L
    g = _grid()
    rng = np.random.default_rng(91)
    M = 37
    fields = rng.uniform(2.0, 20.0) + rng.standard_normal(g.shape + (M,))
    pts = _special_points(g, rng, 40)
    ref_v, ref_g = L.table(g.as_dict(), [fields[..., m] for m in range(M)], pts)
    ctx = tt.tt_ctx_create(g.as_dict())
    for dtype in (torch.float64, torch.float32):
        G = _dev(fields, dtype)
        Fr = G.double().cpu().numpy()
        if dtype == torch.float32:
            ref_v, ref_g = L.table(g.as_dict(), [Fr[..., m] for m in range(M)], pts)
        val = _dev(np.zeros((len(pts), M)))
        grad = _dev(np.zeros((len(pts), M, 3)))
        tt.tt_field_at_points(ctx, G, _dev(pts), val, grad)
        assert np.abs(val.cpu().numpy() - ref_v).max() <= 1e-13 * np.abs(ref_v).max()
        for a in range(3):
            assert np.abs(grad.cpu().numpy()[..., a] - ref_g[..., a]).max() <= \
                1e-12 * np.abs(ref_g[..., a]).max()
    bad = pts.copy()
    bad[3, 0] = g.depth_max_km + 1.0
    with pytest.raises(tt.TTError, match="outside"):
        tt.tt_field_at_points(ctx, _dev(fields), _dev(bad), val, grad)
    ctx.close()


def _data(tt, rng, ns, nr):
    abs_off, abs_rec, abs_tobs, abs_w = [0], [], [], []
    cs_off, cs_m, cs_i, cs_d, cs_w = [0], [], [], [], []
    abs_recs, cs_recs = [], []
    for n in range(ns):
        m = np.sort(rng.choice(nr, rng.integers(3, nr + 1), replace=False))
        t = rng.uniform(5, 15, len(m))
        w = rng.uniform(0.5, 2.0, len(m))
        abs_rec += list(m); abs_tobs += list(t); abs_w += list(w); abs_off.append(len(abs_rec))
        abs_recs.append((m, t, w))
        pairs = [(a, b) for a in range(nr) for b in range(a + 1, nr) if rng.uniform() < 0.3]
        pm = np.array([a for a, _ in pairs], int)
        pi = np.array([b for _, b in pairs], int)
        pd = rng.normal(0, 1.0, len(pairs))
        pw = rng.uniform(0.5, 2.0, len(pairs))
        cs_m += list(pm); cs_i += list(pi); cs_d += list(pd); cs_w += list(pw)
        cs_off.append(len(cs_m))
        cs_recs.append((pm, pi, pd, pw))
    rec = np.zeros((nr, 3))
    data = tt.DeviceData(rec, abs_off, abs_rec, abs_tobs, abs_w, cs_off, cs_m, cs_i, cs_d, cs_w,
                         alpha=0.8, beta=1.3)
    return data, abs_recs, cs_recs


def test_misfit_table_kernels_and_update_match_oracle(tt):
    import oracle.reloc as L
    g = _grid()
    rng = np.random.default_rng(92)
    ns, nr = 45, 29
    data, abs_recs, cs_recs = _data(tt, rng, ns, nr)
    val = rng.uniform(5, 15, (ns, nr))
    otime = rng.normal(0, 0.5, ns)
    Tobs = rng.uniform(5, 15, (ns, nr))
    pairs, W = [], np.zeros((ns, ns, nr))
    for m in range(nr):
        for b in range(ns):
            for j in range(b + 1, ns):
                if rng.uniform() < 0.05:
                    wq = rng.uniform(0.2, 2.0)
                    pairs.append((b, j, m, Tobs[b, m] - Tobs[j, m], wq))
                    W[b, j, m] = W[j, b, m] = wq / 2
    gamma = 0.6
    cr = tt.CrData(ns, nr, pairs, gamma)
    ct, cc, ccr, R_ref = L.misfit_table(val + otime[:, None], abs_recs, cs_recs, 0.8, 1.3,
                                        (Tobs, W, gamma))
    ctx = tt.tt_ctx_create(g.as_dict())
    Tr, chi, R = _dev(np.zeros((ns, nr))), _dev(np.zeros((ns, 2))), _dev(np.zeros((ns, nr)))
    chi_cr = _dev(np.zeros(ns))
    tt.tt_misfit_table(ctx, _dev(val), _dev(otime), data, Tr, chi, R)
    assert np.array_equal(Tr.cpu().numpy(), val + otime[:, None])
    tt.tt_misfit_cr(ctx, cr, Tr, chi_cr, R)
    c = chi.cpu().numpy()
    assert abs(c[:, 0].sum() - ct) <= 1e-12 * ct
    assert abs(c[:, 1].sum() - cc) <= 1e-12 * cc
    assert abs(chi_cr.cpu().numpy().sum() - ccr) <= 1e-12 * ccr
    assert np.abs(R.cpu().numpy() - R_ref).max() <= 1e-12 * np.abs(R_ref).max()
    # kernels (Eqs. B5-B11) from the oracle's R and a random gradient table
    grad = rng.standard_normal((ns, nr, 3))
    Kx, Kt = _dev(np.zeros((ns, 3))), _dev(np.zeros(ns))
    tt.tt_reloc_kernels(ctx, _dev(R_ref), _dev(grad), Kx, Kt)
    Kx_ref, Kt_ref = L.kernels(R_ref, grad)
    assert np.abs(Kx.cpu().numpy() - Kx_ref).max() <= 1e-12 * np.abs(Kx_ref).max()
    assert np.abs(Kt.cpu().numpy() - Kt_ref).max() <= 1e-12 * np.abs(Kt_ref).max()
    # the update (reading R15b), including events pushed against the grid's faces
    lo = np.array([g.depth_min_km, g.lat_min_deg, g.lon_min_deg])
    hi = np.array([g.depth_max_km, g.lat_max_deg, g.lon_max_deg])
    pts = lo + (hi - lo) * rng.uniform(0, 1, (ns, 3))
    p, t = _dev(pts), _dev(otime)
    tt.tt_reloc_update(ctx, p, t, _dev(Kx_ref), _dev(Kt_ref), 5.0, 0.2)
    p_ref, t_ref = L.update(g.as_dict(), pts, otime, Kx_ref, Kt_ref, 5.0, 0.2)
    assert np.abs(p.cpu().numpy() - p_ref).max() <= 1e-11
    assert np.abs(t.cpu().numpy() - t_ref).max() <= 1e-14
    assert ((p_ref == lo) | (p_ref == hi)).any(), "no event reached a face"
    with pytest.raises(tt.TTError):
        tt.tt_reloc_update(ctx, p, t, _dev(Kx_ref), _dev(Kt_ref), -1.0, 0.2)
    ctx.close()


def test_relocation_loop_moves_events_toward_the_truth(tt):
    """Observations: the oracle's FP64 solves from 6 true events (arrival + origin time) at
    12 surface receivers, with common-source pairs. Start: events moved 1.5-2 km, origin times
    zero. The GPU's kernels at the start match the oracle's (its own receiver-started FP64
    solves on the FP32-rounded model), and six steps lower chi and the location error."""
    import torch
    import oracle as O
    import oracle.reloc as L
    from paper_2412_00031_gb300.reloc import Relocation
    w = I.small_case(93, shape=(21, 19, 23), n_src=6, n_rec=12, depth_max=20.0,
                     extent_deg=0.2)
    g = w.grid.as_dict()
    rng = np.random.default_rng(93)
    true = np.array(w.src, dtype=np.float64)
    t_true = rng.normal(0, 0.3, len(true))
    rec = np.array(w.rec)
    rec[:, 0] = 0.0                                                   # surface receivers
    nr = len(rec)
    tobs = []
    for n in range(len(true)):
        _, T, _, ok, _ = O.forward(g, w.s, w.xi, w.eta, true[n], tol=1e-10, max_iter=1000)
        assert ok
        tobs.append(O.receiver_times(g, T, rec) + t_true[n])
    tobs = np.array(tobs)
    ns = len(true)
    pairs = [(m, i) for m in range(nr) for i in range(m + 1, nr)]
    cs_m = np.tile([p[0] for p in pairs], ns)
    cs_i = np.tile([p[1] for p in pairs], ns)
    cs_d = np.concatenate([tobs[n, [p[0] for p in pairs]] - tobs[n, [p[1] for p in pairs]]
                           for n in range(ns)])
    data = tt.DeviceData(rec, np.arange(ns + 1) * nr, np.tile(np.arange(nr), ns), tobs.ravel(),
                         np.ones(ns * nr), np.arange(ns + 1) * len(pairs), cs_m, cs_i, cs_d,
                         np.full(len(cs_m), 0.5))
    start = true.copy()
    start[:, 0] += rng.choice([-1, 1], ns) * rng.uniform(1.5, 2.0, ns)
    start[:, 1] += rng.choice([-1, 1], ns) * 0.015
    start[:, 2] += rng.choice([-1, 1], ns) * 0.015
    model = tuple(_dev(a, torch.float32) for a in (w.s, w.xi, w.eta))
    ctx = tt.tt_ctx_create(g)
    pts, otime = _dev(start), _dev(np.zeros(ns))
    rl = Relocation(ctx, model, w.grid.shape, data, pts, otime)
    rl.evaluate()
    # the oracle's kernels at the start, from its own receiver-started solves
    s32 = [a.double().cpu().numpy() for a in model]
    fields = []
    for m in range(nr):
        _, G, _, ok, _ = O.forward(g, *s32, rec[m], tol=1e-10, max_iter=1000)
        assert ok
        fields.append(G)
    val, grad = L.table(g, fields, start)
    abs_recs = [(np.arange(nr), tobs[n], np.ones(nr)) for n in range(ns)]
    cs_recs = [(np.array([p[0] for p in pairs]), np.array([p[1] for p in pairs]),
                tobs[n, [p[0] for p in pairs]] - tobs[n, [p[1] for p in pairs]],
                np.full(len(pairs), 0.5)) for n in range(ns)]
    _, _, _, R_ref = L.misfit_table(val, abs_recs, cs_recs)
    Kx_ref, Kt_ref = L.kernels(R_ref, grad)
    Kx = rl.Kx.cpu().numpy()
    assert np.linalg.norm(Kx - Kx_ref) <= 1e-3 * np.linalg.norm(Kx_ref)
    assert np.linalg.norm(rl.Kt.cpu().numpy() - Kt_ref) <= 1e-3 * np.linalg.norm(Kt_ref)
    err0 = np.abs(start[:, 0] - true[:, 0]).mean()
    hist = rl.run(6, 1.5, 0.2)
    print("\nchi, step, accepted:", [("%.4g" % c, s, a) for c, s, a in hist])
    err1 = np.abs(pts.cpu().numpy()[:, 0] - true[:, 0]).mean()
    print("mean depth error: %.3f -> %.3f km" % (err0, err1))
    ctx.close()
    chis = [h[0] for h in hist if h[2]]
    assert hist[1][2], "the first step along the computed direction raised chi"
    assert chis[-1] <= 0.5 * chis[0]
    assert err1 <= 0.7 * err0
