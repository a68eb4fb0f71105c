"""Parity of the inversion step's kernels with the FP64 oracle (oracle/inversion.py), and the
inversion loop on a small synthetic case (needs a GB300).

- kernel density (Eq. 19), normalisation (Eq. 18), projection (Eq. 17) and expansion
  (Eq. 15) on seeded inputs, element by element; grids of several inversion-grid cells and
  ragged fine / coarse ratios; one projection at the 201 x 201 x 101 configuration size;
- the model update (FP32 and FP64 models);
- the common-receiver misfit and adjoint source (Eqs. 4, A4) against the oracle;
- the loop: observations from the oracle's FP64 forward in a checkerboard model (absolute
  and common-receiver times), inversion from the background model: chi must fall.
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


def test_kernel_density_sums_sources(tt):
    import torch
    import oracle.inversion as V
    w = I.small_case(81, shape=(9, 10, 11), n_src=1)
    rng = np.random.default_rng(81)
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    for dtype, B in ((torch.float32, 37), (torch.float64, 5)):
        P = rng.standard_normal(w.grid.shape + (B,))
        Pd = _dev(P, dtype)
        Kd = _dev(np.full(w.grid.shape, 0.5))
        tt.tt_kernel_density(ctx, Pd, Kd)
        P64 = Pd.double().cpu().numpy()
        ref = 0.5 + V.kernel_density([P64[..., b] for b in range(B)])
        assert np.abs(Kd.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    ctx.close()


def test_normalisation_matches_oracle(tt):
    import oracle.inversion as V
    w = I.small_case(82, shape=(9, 10, 11), n_src=1)
    rng = np.random.default_rng(82)
    K = [rng.standard_normal(w.grid.shape) for _ in range(3)]
    Kd = rng.uniform(0.0, 5.0, w.grid.shape)
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    Kdev = [_dev(k) for k in K]
    tt.tt_kernel_normalize(ctx, *Kdev, _dev(Kd), 0.3, 0.7)
    for a, k in zip(Kdev, K):
        ref = V.normalize(k, Kd, 0.3, 0.7)
        assert np.abs(a.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
    ctx.close()


def test_relative_normalisation_takes_the_density_maximum_on_the_device(tt):
    """Eq. 18 with eps = eps_rel max(Kd): the oracle's normalisation with eps computed from
    the maximum of Kd (and the smallest positive eps when Kd is zero everywhere)."""
    import oracle.inversion as V
    w = I.small_case(83, shape=(9, 10, 11), n_src=1)
    rng = np.random.default_rng(83)
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    for Kd in (rng.uniform(0.0, 5.0, w.grid.shape), np.zeros(w.grid.shape)):
        K = [rng.standard_normal(w.grid.shape) for _ in range(3)]
        Kdev = [_dev(k) for k in K]
        tt.tt_kernel_normalize_rel(ctx, *Kdev, _dev(Kd), 0.02, 0.7)
        eps = max(0.02 * Kd.max(), 1e-300)
        for a, k in zip(Kdev, K):
            ref = V.normalize(k, Kd, eps, 0.7)
            assert np.abs(a.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
    ctx.close()


@pytest.mark.parametrize("n_src", [1, 37, 300, 4096])
def test_misfit_total_is_the_weighted_sum(tt, n_src):
    """The step control's total misfit: alpha sum chi_t + beta sum chi_cs + gamma sum chi_cr
    of a batch, an FP64 sum on the device, equals the exact sum (math.fsum) to 1e-14."""
    import math
    w = I.small_case(84, shape=(9, 10, 11), n_src=1)
    rng = np.random.default_rng(84 + n_src)
    chi = rng.uniform(0.0, 3.0, (n_src, 2))
    cr = rng.uniform(0.0, 1.0, n_src)
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    got = tt.tt_misfit_total(ctx, _dev(chi), 0.7, 1.3, _dev(cr), 0.4)
    ref = math.fsum(list(0.7 * chi[:, 0]) + list(1.3 * chi[:, 1]) + list(0.4 * cr))
    assert abs(got - ref) <= 1e-14 * ref
    got2 = tt.tt_misfit_total(ctx, _dev(chi), 1.0, 1.0)
    assert abs(got2 - math.fsum(chi.ravel())) <= 1e-14 * got2
    ctx.close()


@pytest.mark.parametrize("shape,coarse,H", [((9, 10, 11), (4, 5, 4), 3),
                                            ((17, 23, 19), (11, 11, 11), 5),
                                            ((13, 12, 33), (6, 3, 9), 2)])
def test_projection_and_expansion_match_oracle(tt, shape, coarse, H):
    import oracle as O
    import oracle.inversion as V
    w = I.small_case(83, shape=shape, n_src=1)
    g = w.grid.as_dict()
    rng = np.random.default_rng(83)
    K = rng.standard_normal(shape)
    Gin = rng.standard_normal((H,) + coarse)
    B = V.bases(shape, coarse, H)
    dV = O.node_volumes(g)
    ctx = tt.tt_ctx_create(g)
    mg = tt.mgrid(*coarse, H)
    G = _dev(np.zeros((H,) + coarse))
    tt.tt_mgrid_project(ctx, mg, _dev(K), G)
    ref = V.project(K, dV, B, H)
    assert np.abs(G.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    D = _dev(np.zeros(shape))
    tt.tt_mgrid_expand(ctx, mg, _dev(Gin), D)
    ref = V.expand(Gin, B, H)
    assert np.abs(D.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    ctx.close()


def test_projection_at_the_inversion_configuration_size(tt):
    """201 (lat) x 201 (lon) x 101 (depth) nodes, 5 grids of 11^3: against the oracle on a
    smooth kernel (the oracle contracts one axis at a time through einsum's path)."""
    import oracle as O
    import oracle.inversion as V
    g = I.GridSpec(101, 201, 201, 0.0, 200.0, 0.0, 5.0, 0.0, 5.0).as_dict()
    shape, coarse, H = (101, 201, 201), (11, 11, 11), 5
    i, j, k = np.meshgrid(*[np.linspace(0, 1, n) for n in shape], indexing="ij")
    K = np.sin(3 * i) * np.cos(2 * j) + k * k
    ctx = tt.tt_ctx_create(g)
    mg = tt.mgrid(*coarse, H)
    G = _dev(np.zeros((H,) + coarse))
    tt.tt_mgrid_project(ctx, mg, _dev(K), G)
    B = V.bases(shape, coarse, H)
    Ur, Ut, Up = B
    KV = K * O.node_volumes(g)
    ref = np.stack([np.einsum("ijk,ai,bj,ck->abc", KV, Ur[h], Ut[h], Up[h], optimize=True) / H
                    for h in range(H)])
    assert np.abs(G.cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()
    ctx.close()


def test_model_update_matches_oracle(tt):
    import torch
    import oracle.inversion as V
    w = I.small_case(84, shape=(9, 10, 11), n_src=1)
    rng = np.random.default_rng(84)
    D = [rng.standard_normal(w.grid.shape) for _ in range(3)]
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    for dtype, tol in ((torch.float32, 2e-7), (torch.float64, 1e-14)):
        model = tuple(_dev(a, dtype) for a in (w.s, w.xi, w.eta))
        before = [a.double().cpu().numpy() for a in model]
        tt.tt_model_update(ctx, model, *[_dev(d) for d in D], 0.03)
        ref = V.update(*before, *D, 0.03)
        for a, r in zip(model, ref):
            got = a.double().cpu().numpy()
            assert np.abs(got - r).max() <= tol * np.abs(r).max() + 1e-12
    ctx.close()


def test_common_receiver_misfit_matches_oracle(tt):
    import torch
    from oracle.cr import misfit_cr
    rng = np.random.default_rng(86)
    ns, nr = 37, 23
    Tr = rng.uniform(5, 30, (ns, nr))
    Tobs = Tr + rng.normal(0, 0.2, (ns, nr))
    pairs, W = [], np.zeros((ns, ns, nr))
    for m in range(nr):
        for b in range(ns):
            for j in range(b + 1, ns):
                if rng.uniform() < 0.15:
                    wq = rng.uniform(0.2, 2.0)
                    pairs.append((b, j, m, Tobs[b, m] - Tobs[j, m], wq))
                    W[b, j, m] = W[j, b, m] = wq / 2     # two ordered terms of weight w / 2
    gamma = 1.7
    _, share, R_ref = misfit_cr(Tr, Tobs, W, gamma)
    g = I.small_case(86, shape=(9, 10, 11), n_src=1).grid.as_dict()
    ctx = tt.tt_ctx_create(g)
    cr = tt.CrData(ns, nr, pairs, gamma)
    R0 = rng.standard_normal((ns, nr))
    R, chi = _dev(R0), _dev(np.zeros(ns))
    tt.tt_misfit_cr(ctx, cr, _dev(Tr), chi, R)
    assert np.abs(R.cpu().numpy() - (R0 + R_ref)).max() <= 1e-12 * np.abs(R_ref).max()
    assert np.abs(chi.cpu().numpy() - share).max() <= 1e-12 * np.abs(share).max()
    # an entry naming a source outside the batch is skipped and refused
    cr.other[0] = ns + 3
    with pytest.raises(tt.TTError):
        tt.tt_misfit_cr(ctx, cr, _dev(Tr), chi, _dev(R0))
    ctx.close()


def test_inversion_loop_reduces_the_misfit(tt):
    """Observations: the oracle's FP64 forward in a 5 % checkerboard model, as absolute and
    common-receiver differential times; start: the background. The first step along the
    computed direction must be accepted (a descent direction), and three step attempts must
    lower chi by at least 5 % (measured: 10 %; 29 % without the common-receiver terms)."""
    import torch
    import oracle as O
    from paper_2412_00031_gb300.invert import Inversion
    w = I.small_case(85, shape=(17, 17, 17), n_src=6, n_rec=12)
    g = w.grid.as_dict()
    shape = w.grid.shape
    i, j, k = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    cb = 0.05 * np.sin(np.pi * i / 8) * np.sin(np.pi * j / 8) * np.sin(np.pi * k / 8)
    s_true = w.s / (1.0 + cb)
    tobs = []
    for b in range(w.n_src):
        _, T, _, conv, _ = O.forward(g, s_true, w.xi, w.eta, w.src[b], tol=1e-9, max_iter=500)
        assert conv
        tobs.append(O.receiver_times(g, T, w.rec))
    rec_all = np.arange(len(w.rec))
    data = tt.DeviceData(w.rec, np.arange(w.n_src + 1) * len(w.rec), np.tile(rec_all, w.n_src),
                         np.concatenate(tobs), np.ones(w.n_src * len(w.rec)),
                         np.zeros(w.n_src + 1, dtype=np.int32), [], [], [], [])
    T_obs = np.stack(tobs)
    pairs = [(b, j, m, T_obs[b, m] - T_obs[j, m], 1.0) for m in range(len(w.rec))
             for b in range(w.n_src) for j in range(b + 1, w.n_src)]
    cr = tt.CrData(w.n_src, len(w.rec), pairs, gamma=0.5)
    model = tuple(_dev(a, torch.float32) for a in (w.s, w.xi, w.eta))
    ctx = tt.tt_ctx_create(g)
    inv = Inversion(ctx, model, w.src, data, shape, tt.mgrid(5, 5, 5, 3), cr=cr)
    hist = inv.run(3, 0.03)
    ctx.close()
    chis = [h[0] for h in hist if h[2]]
    print("\nchi, step, accepted:", [("%.4g" % c, s, a) for c, s, a in hist])
    assert hist[1][2], "the first step along the computed direction raised chi"
    assert chis[-1] <= 0.95 * chis[0]


def test_batches_sum_to_the_single_batch(tt):
    """The same sources as one batch or as two (kernels, kernel density and chi summed over
    batches): equal up to the order of the FP64 sums."""
    import torch
    from paper_2412_00031_gb300.invert import Inversion
    w = I.small_case(87, shape=(13, 15, 17), n_src=7, n_rec=9)
    g = w.grid.as_dict()
    model = tuple(_dev(a, torch.float32) for a in (w.s, w.xi, w.eta))
    ctx = tt.tt_ctx_create(g)
    mg = tt.mgrid(4, 4, 4, 2)
    one = Inversion(ctx, model, w.src, tt.DeviceData.from_workload(w), w.grid.shape, mg)
    c1 = one.evaluate()
    parts = [w.subset(range(0, 4)), w.subset(range(4, 7))]
    two = Inversion(ctx, model, None, None, w.grid.shape, mg,
                    batches=[(p.src, tt.DeviceData.from_workload(p), None) for p in parts])
    c2 = two.evaluate()
    assert abs(c1 - c2) <= 1e-12 * c1
    for a, b in zip(one.K + [one.Kd], two.K + [two.Kd]):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    ctx.close()


def test_joint_relocation_lowers_chi_below_the_model_only_loop(tt):
    """Hypocentres and origin times updated during the inversion (Sec. 2, Eq. 10).
    Observations: the oracle's FP64 solves in a 5 % checkerboard model from the true events,
    plus true origin times. Start: the background model, the events moved by 1-1.5 km in
    depth and 0.005 deg laterally, origin times zero. Three model steps with a relocation
    step after each must reach a lower chi than three model steps alone, and move the
    events toward the truth."""
    import torch
    import oracle as O
    from paper_2412_00031_gb300.invert import Inversion
    w = I.small_case(88, shape=(17, 17, 17), n_src=6, n_rec=12)
    g = w.grid.as_dict()
    shape = w.grid.shape
    rng = np.random.default_rng(88)
    i, j, k = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    cb = 0.05 * np.sin(np.pi * i / 8) * np.sin(np.pi * j / 8) * np.sin(np.pi * k / 8)
    s_true = w.s / (1.0 + cb)
    true = np.array(w.src, dtype=np.float64)
    t0 = rng.normal(0, 0.2, len(true))
    tobs = []
    for b in range(len(true)):
        _, T, _, conv, _ = O.forward(g, s_true, w.xi, w.eta, true[b], tol=1e-9, max_iter=500)
        assert conv
        tobs.append(O.receiver_times(g, T, w.rec) + t0[b])
    nr, ns = len(w.rec), len(true)
    data = tt.DeviceData(w.rec, np.arange(ns + 1) * nr, np.tile(np.arange(nr), ns),
                         np.concatenate(tobs), np.ones(ns * nr),
                         np.zeros(ns + 1, dtype=np.int32), [], [], [], [])
    start = true.copy()
    start[:, 0] += rng.choice([-1, 1], ns) * rng.uniform(1.0, 1.5, ns)
    start[:, 1:] += rng.choice([-1, 1], (ns, 2)) * 0.005
    ctx = tt.tt_ctx_create(g)
    out = {}
    for name, reloc in (("model", None), ("joint", (0.8, 0.1))):
        model = tuple(_dev(a, torch.float32) for a in (w.s, w.xi, w.eta))
        inv = Inversion(ctx, model, start.copy(), data, shape, tt.mgrid(5, 5, 5, 3),
                        relocate=reloc)
        hist = inv.run(3, 0.03)
        chi = inv.evaluate()
        out[name] = (chi, hist, inv)
        print("\n%s: chi %s -> %.4g" % (name, ["%.4g" % h[0] for h in hist], chi))
    inv = out["joint"][2]
    print("relocation steps (chi before, after, accepted):", inv.reloc_hist)
    err0 = np.abs(start[:, 0] - true[:, 0]).mean()
    err1 = np.abs(inv.batches[0].src[:, 0] - true[:, 0]).mean()
    print("mean depth error %.3f -> %.3f km" % (err0, err1))
    ctx.close()
    assert out["joint"][0] < 0.8 * out["model"][0]
    assert err1 < 0.8 * err0


def test_common_receiver_pairs_across_batches_equal_one_batch(tt):
    """Common-receiver pairs that span two batches (cr_all): the kept traveltime fields and
    the joined receiver-time tables give the single batch's chi, kernels and kernel density
    (up to the order of the FP64 sums)."""
    import torch
    from paper_2412_00031_gb300.invert import Inversion
    w = I.small_case(89, shape=(13, 15, 17), n_src=7, n_rec=9)
    g = w.grid.as_dict()
    rng = np.random.default_rng(89)
    nr = len(w.rec)
    pairs = [(b, j, m, rng.normal(0, 0.3), rng.uniform(0.5, 1.5)) for m in range(nr)
             for b in range(7) for j in range(b + 1, 7) if rng.uniform() < 0.5]
    assert any(b < 4 <= j for b, j, _, _, _ in pairs), "no pair spans the two batches"
    model = tuple(_dev(a, torch.float32) for a in (w.s, w.xi, w.eta))
    ctx = tt.tt_ctx_create(g)
    mg = tt.mgrid(4, 4, 4, 2)
    one = Inversion(ctx, model, w.src, tt.DeviceData.from_workload(w), w.grid.shape, mg,
                    cr=tt.CrData(7, nr, pairs, gamma=0.7))
    c1 = one.evaluate()
    parts = [w.subset(range(0, 4)), w.subset(range(4, 7))]
    two = Inversion(ctx, model, None, None, w.grid.shape, mg,
                    batches=[(p.src, tt.DeviceData.from_workload(p), None) for p in parts],
                    cr_all=tt.CrData(7, nr, pairs, gamma=0.7))
    c2 = two.evaluate()
    assert abs(c1 - c2) <= 1e-12 * c1
    for a, b in zip(one.K + [one.Kd], two.K + [two.Kd]):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    ctx.close()


def test_relocation_with_pairs_across_batches_equals_one_batch(tt):
    """Double-difference (common-receiver) relocation across batches: two batches with the
    pairs in cr_all move their events exactly as one batch with the same pairs does (joint
    step normalised over all events, step control on the total chi), to the order of the FP64
    sums, over two relocation steps."""
    import torch
    from paper_2412_00031_gb300.invert import Inversion
    w = I.small_case(90, shape=(13, 15, 17), n_src=7, n_rec=9)
    g = w.grid.as_dict()
    rng = np.random.default_rng(90)
    nr = len(w.rec)
    pairs = [(b, j, m, rng.normal(0, 0.3), rng.uniform(0.5, 1.5)) for m in range(nr)
             for b in range(7) for j in range(b + 1, 7) if rng.uniform() < 0.5]
    assert any(b < 4 <= j for b, j, _, _, _ in pairs), "no pair spans the two batches"
    model = tuple(_dev(a, torch.float32) for a in (w.s, w.xi, w.eta))
    ctx = tt.tt_ctx_create(g)
    mg = tt.mgrid(4, 4, 4, 2)
    one = Inversion(ctx, model, w.src, tt.DeviceData.from_workload(w), w.grid.shape, mg,
                    cr=tt.CrData(7, nr, pairs, gamma=0.7), relocate=(0.6, 0.1))
    parts = [w.subset(range(0, 4)), w.subset(range(4, 7))]
    two = Inversion(ctx, model, None, None, w.grid.shape, mg,
                    batches=[(p.src, tt.DeviceData.from_workload(p), None) for p in parts],
                    cr_all=tt.CrData(7, nr, pairs, gamma=0.7), relocate=(0.6, 0.1))
    for _ in range(2):
        one.relocate_events()
        two.relocate_events()
    for (b1, a1, ok1), (b2, a2, ok2) in zip(one.reloc_hist, two.reloc_hist):
        assert abs(b1 - b2) <= 1e-12 * b1 and abs(a1 - a2) <= 1e-12 * a1 and ok1 == ok2
    assert any(h[2] for h in one.reloc_hist)
    p1 = one.batches[0].pts.cpu().numpy()
    p2 = np.concatenate([bt.pts.cpu().numpy() for bt in two.batches])
    assert np.abs(p1 - p2).max() <= 1e-9
    t1 = one.batches[0].otime.cpu().numpy()
    t2 = np.concatenate([bt.otime.cpu().numpy() for bt in two.batches])
    assert np.abs(t1 - t2).max() <= 1e-12
    assert np.abs(p1 - w.src).max() > 1e-3          # the events did move
    ctx.close()
