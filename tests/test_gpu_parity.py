"""GPU path against the FP64 oracle, through the C ABI (needs a GB300)."""
import numpy as np
import pytest

import tt_inputs as I
from gpu_helpers import gpu_solve, oracle_solve, rel_l2, rel_linf, rounded_model, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_00031_gb300 as m
    return m


def test_homogeneous_41_fp64_is_closed_form(tt):
    """41^3 spherical grid, Vp = 6 km/s, surface source: T = s * chord (FP64, 1e-12)."""
    w = I.homogeneous_41()
    out = gpu_solve(w, "f64", opts=tt.default_opts(tt.TT_F64, tol_fwd=1e-7, tol_adj=1e-7))
    from test_oracle import _cart, _node_points
    exact = np.linalg.norm(_cart(w.grid, _node_points(w.grid)) - _cart(w.grid, w.src[0])[0],
                           axis=-1) / 6.0
    assert out["iters_fwd"][0] == 1
    assert rel_linf(out["T"][..., 0], exact) <= 1e-12
    res, K = oracle_solve(w, tol=1e-7)
    assert rel_l2(out["P"][..., 0], res[0]["P"]) <= 1e-9
    for a, b in zip(out["K"], K):
        assert rel_l2(a, b) <= 1e-9


@pytest.mark.parametrize("seed,shape,flat", [(1, (13, 15, 17), 0), (2, (9, 21, 11), 0),
                                              (3, (12, 11, 14), 1)])
def test_small_fp64_matches_oracle(tt, seed, shape, flat):
    """Ragged grids, several sources, anisotropic heterogeneous model: FP64 GPU = oracle up to
    rounding order."""
    w = I.small_case(seed, shape=shape, n_src=3, n_rec=6, flat=flat)
    o = tt.default_opts(tt.TT_F64, tol_fwd=1e-12, tol_adj=1e-12, max_iter_fwd=2000,
                        max_iter_adj=2000)
    out = gpu_solve(w, "f64", opts=o)
    res, K = oracle_solve(w, tol=1e-12)
    for b, r in enumerate(res):
        assert abs(int(out["iters_fwd"][b]) - r["iters_fwd"]) <= 1
        assert rel_linf(out["T"][..., b], r["T"]) <= 1e-10
        assert rel_linf(out["Tr"][b], r["Tr"]) <= 1e-10
        assert out["chi"][b] == pytest.approx([r["chi_t"], r["chi_cs"]], rel=1e-8, abs=1e-12)
        assert np.abs(out["R"][b] - r["R"]).max() <= 1e-8 * max(1.0, np.abs(r["R"]).max())
        assert rel_l2(out["P"][..., b], r["P"]) <= 1e-8
    for a, b in zip(out["K"], K):
        assert rel_l2(a, b) <= 1e-8


@pytest.mark.parametrize("seed,shape,flat", [(4, (13, 15, 17), 0), (5, (21, 19, 23), 0),
                                              (6, (11, 13, 9), 1)])
def test_small_fp32_within_tolerance(tt, seed, shape, flat):
    """FP32 sweeps with FP64 reductions against the FP64 oracle: relative L-infinity T error
    <= 1e-5 and relative L2 kernel error <= 1e-3."""
    w = I.small_case(seed, shape=shape, n_src=4, n_rec=7, flat=flat)
    out = gpu_solve(w, "f32")
    res, K = oracle_solve(w, model=rounded_model(w, "f32"), tol=1e-10)
    for b, r in enumerate(res):
        assert rel_linf(out["T"][..., b], r["T"]) <= 1e-5
        assert rel_l2(out["P"][..., b], r["P"]) <= 1e-3
    for a, b in zip(out["K"], K):
        assert rel_l2(a, b) <= 1e-3


def test_batch_equals_single_sources_bitwise(tt):
    """Each source's result does not depend on the rest of the batch (same arithmetic, same
    hyperplane order, own convergence test)."""
    w = I.small_case(7, shape=(14, 16, 15), n_src=5, n_rec=6)
    full = gpu_solve(w, "f32")
    for b in range(w.n_src):
        one = gpu_solve(w.subset([b]), "f32")
        assert one["iters_fwd"][0] == full["iters_fwd"][b]
        assert np.array_equal(one["tau"][..., 0], full["tau"][..., b])
        assert np.array_equal(one["P"][..., 0], full["P"][..., b])


@pytest.mark.parametrize("blocks", [1, 3, 7])
def test_launch_shape_does_not_change_bits(tt, blocks):
    """A 7-point Gauss-Seidel sweep gives the same bits under every schedule that respects
    the hyperplane order, whatever the number of blocks and slots."""
    w = I.small_case(8, shape=(15, 13, 17), n_src=3, n_rec=5)
    ref = gpu_solve(w, "f32")
    o = tt.default_opts(tt.TT_F32, launch_blocks=blocks)
    out = gpu_solve(w, "f32", opts=o)
    assert np.array_equal(out["tau"], ref["tau"])
    assert np.array_equal(out["P"], ref["P"])
    for a, b in zip(out["K"], ref["K"]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("schedule,blocks", [(1, 0), (2, 0), (2, 5), (3, 0), (4, 0), (4, 2)])
def test_sweep_schedules_give_identical_bits(tt, schedule, blocks):
    """Node hyperplanes and tile hyperplanes of every shape visit each node after its
    upstream neighbours and before its downstream ones, so the forward result is the same
    bits whatever the schedule, tile shape or launch size (ragged tiles included)."""
    w = I.small_case(14, shape=(14, 19, 23), n_src=37, n_rec=5)
    ref = gpu_solve(w, "f32", opts=tt.default_opts(tt.TT_F32, sweep_schedule=1),
                    steps=("fwd",))
    o = tt.default_opts(tt.TT_F32, sweep_schedule=schedule, launch_blocks=blocks)
    out = gpu_solve(w, "f32", opts=o, steps=("fwd",))
    assert np.array_equal(out["iters_fwd"], ref["iters_fwd"])
    assert np.array_equal(out["tau"], ref["tau"])


def test_kernels_bitwise_reproducible(tt):
    w = I.small_case(9, shape=(13, 13, 13), n_src=6, n_rec=6)
    a = gpu_solve(w, "f32")
    b = gpu_solve(w, "f32")
    for x, y in zip(a["K"], b["K"]):
        assert np.array_equal(x, y)
    assert np.array_equal(a["R"], b["R"])


def test_warm_start_from_converged_tau_takes_one_iteration(tt):
    w = I.small_case(10, shape=(13, 14, 15), n_src=2, n_rec=5)
    cold = gpu_solve(w, "f32", steps=("fwd",))
    o = tt.default_opts(tt.TT_F32, init=1)
    warm = gpu_solve(w, "f32", opts=o, steps=("fwd",), tau_init=cold["tau"])
    assert (warm["iters_fwd"] <= 2).all()
    assert rel_linf(warm["T"], cold["T"]) <= 1e-6


# ------------------------------------------------------------------------- error paths

def _ctx_and_model(tt, w, dt="f32"):
    import torch
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    d = torch.float32 if dt == "f32" else torch.float64
    return ctx, tuple(to_dev(a, d) for a in (w.s, w.xi, w.eta))


def test_invalid_inputs_are_rejected(tt):
    import torch
    w = I.small_case(11, shape=(9, 9, 9), n_src=1, n_rec=4)
    ctx, model = _ctx_and_model(tt, w)
    tau = torch.empty(w.grid.shape + (1,), device="cuda")
    bad_src = np.array([[500.0, 0.05, 0.05]])
    with pytest.raises(tt.TTError) as e:
        tt.tt_forward(ctx, model, bad_src, tau)
    assert e.value.status == tt.TT_EINVAL
    xi_bad = model[1].clone()
    xi_bad[3, 3, 3] = 0.6
    with pytest.raises(tt.TTError) as e:
        tt.tt_forward(ctx, (model[0], xi_bad, model[2]), w.src, tau)
    assert e.value.status == tt.TT_EINVAL
    s_bad = model[0].clone()
    s_bad[1, 2, 3] = -1.0
    with pytest.raises(tt.TTError) as e:
        tt.tt_forward(ctx, (s_bad, model[1], model[2]), w.src, tau)
    assert e.value.status == tt.TT_EINVAL
    # the context is still usable
    tt.tt_forward(ctx, model, w.src, tau)
    ctx.close()


def test_iteration_limit_reports_not_converged(tt):
    import torch
    w = I.small_case(12, shape=(11, 11, 11), n_src=2, n_rec=4)
    ctx, model = _ctx_and_model(tt, w)
    tau = torch.empty(w.grid.shape + (2,), device="cuda")
    o = tt.default_opts(tt.TT_F32, max_iter_fwd=1)
    with pytest.raises(tt.TTError) as e:
        tt.tt_forward(ctx, model, w.src, tau, None, o)
    assert e.value.status == tt.TT_ENOTCONVERGED
    it = tt.tt_forward(ctx, model, w.src, tau, None, o, allow_unconverged=True)
    assert (it == 1).all()
    ctx.close()


def test_device_wait_limit_returns_timeout(tt):
    """A wait limit far below a barrier's real duration makes the persistent launch give up
    with TT_ETIMEOUT; the kernel returns on its own and the context stays usable."""
    import torch
    w = I.small_case(13, shape=(40, 40, 40), n_src=64, n_rec=4)
    ctx, model = _ctx_and_model(tt, w)
    tau = torch.empty(w.grid.shape + (64,), device="cuda")
    o = tt.default_opts(tt.TT_F32, spin_limit_ns=1)
    with pytest.raises(tt.TTError) as e:
        tt.tt_forward(ctx, model, w.src, tau, None, o)
    assert e.value.status == tt.TT_ETIMEOUT
    tt.tt_forward(ctx, model, w.src, tau)
    ctx.close()


def test_plan_replays_the_step_bitwise(tt):
    """A captured plan gives the bits of the individual calls, run after run."""
    import torch
    w = I.small_case(15, shape=(13, 14, 16), n_src=33, n_rec=6)
    ref = gpu_solve(w, "f32")
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    model = tuple(to_dev(a, torch.float32) for a in (w.s, w.xi, w.eta))
    shape = w.grid.shape + (w.n_src,)
    tau, T, P = (torch.empty(shape, device="cuda") for _ in range(3))
    data = tt.DeviceData.from_workload(w)
    chi = torch.empty((w.n_src, 2), dtype=torch.float64, device="cuda")
    R = torch.empty((w.n_src, data.n_rec), dtype=torch.float64, device="cuda")
    K = [torch.empty(w.grid.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    plan = tt.tt_plan_create(ctx, model, w.src, data, tau, T, P, chi, R, *K)
    for _ in range(2):
        itf, ita = tt.tt_plan_run(plan)
        assert np.array_equal(itf, ref["iters_fwd"]) and np.array_equal(ita, ref["iters_adj"])
        assert np.array_equal(tau.cpu().numpy(), ref["tau"])
        assert np.array_equal(P.cpu().numpy(), ref["P"])
        assert np.array_equal(R.cpu().numpy(), ref["R"])
        for a, b in zip(K, ref["K"]):
            assert np.array_equal(a.cpu().numpy(), b)
    plan.close()
    ctx.close()


@pytest.mark.parametrize("init", [0, 3])
def test_plan_in_iteration_order_gives_the_same_bits(tt, init):
    """From its second run a plan sweeps the batch in the order of the previous run's forward
    iteration counts, fewest first (opts.fwd_order = 0, batches of 64 sources or more): every
    run gives the bits of the individual calls and of a plan that keeps the given order
    (fwd_order = 1), with the iteration counts in the batch's order."""
    import torch
    w = I.small_case(19, shape=(13, 14, 16), n_src=96, n_rec=6)
    ref = gpu_solve(w, "f32", opts=tt.default_opts(tt.TT_F32, init=init))
    assert len(set(ref["iters_fwd"].tolist())) > 1     # an order that differs from the given one
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    model = tuple(to_dev(a, torch.float32) for a in (w.s, w.xi, w.eta))
    shape = w.grid.shape + (w.n_src,)
    data = tt.DeviceData.from_workload(w)
    outs = []
    for order in (0, 1):
        tau, T, P = (torch.empty(shape, device="cuda") for _ in range(3))
        chi = torch.empty((w.n_src, 2), dtype=torch.float64, device="cuda")
        R = torch.empty((w.n_src, data.n_rec), dtype=torch.float64, device="cuda")
        K = [torch.empty(w.grid.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
        o = tt.default_opts(tt.TT_F32, init=init, fwd_order=order)
        plan = tt.tt_plan_create(ctx, model, w.src, data, tau, T, P, chi, R, *K, opts=o)
        for _ in range(3):
            itf, ita = tt.tt_plan_run(plan)
            assert np.array_equal(itf, ref["iters_fwd"]) and np.array_equal(ita, ref["iters_adj"])
            assert np.array_equal(tau.cpu().numpy(), ref["tau"])
            assert np.array_equal(T.cpu().numpy(), ref["T"])
            assert np.array_equal(P.cpu().numpy(), ref["P"])
            assert np.array_equal(R.cpu().numpy(), ref["R"])
            for a, b in zip(K, ref["K"]):
                assert np.array_equal(a.cpu().numpy(), b)
        outs.append(chi.cpu().numpy())
        plan.close()
    assert np.array_equal(outs[0], outs[1])
    ctx.close()


def test_repeated_forward_calls_in_iteration_order_give_the_same_bits(tt):
    """A context remembers the forward iteration counts of a source set; the next tt_forward
    of the same sources sweeps them fewest first. The results are the given order's bits:
    from tau = 1, from a caller's start (opts.init = 1) and with T, with the counts in the
    batch's order."""
    import torch
    w = I.small_case(20, shape=(13, 14, 16), n_src=80, n_rec=4)
    model = tuple(to_dev(a, torch.float32) for a in (w.s, w.xi, w.eta))
    shape = w.grid.shape + (w.n_src,)
    rng = np.random.default_rng(20)
    start = torch.as_tensor((1.0 + 0.2 * rng.uniform(size=shape)).astype(np.float32), device="cuda")
    outs = {}
    for order in (1, 0):
        ctx = tt.tt_ctx_create(w.grid.as_dict())
        for rep in range(2):
            for init in (0, 1):
                tau = start.clone() if init == 1 else torch.empty(shape, device="cuda")
                T = torch.empty(shape, device="cuda")
                it = tt.tt_forward(ctx, model, w.src, tau, T,
                                   tt.default_opts(tt.TT_F32, init=init, fwd_order=order))
                outs[(order, rep, init)] = (it, tau.cpu().numpy(), T.cpu().numpy())
        ctx.close()
    assert len(set(outs[(1, 0, 0)][0].tolist())) > 1
    for key, (it, tau, T) in outs.items():
        ref = outs[(1, 0, key[2])]
        assert np.array_equal(it, ref[0]), key
        assert np.array_equal(tau, ref[1]) and np.array_equal(T, ref[2]), key


def test_autotuner_picks_a_measured_candidate_with_identical_results(tt):
    """The tuner times every launch configuration and keeps the fastest; the tuned solve
    gives the default solve's bits, and a second call reuses the cached choice."""
    import torch
    w = I.small_case(16, shape=(14, 17, 19), n_src=40, n_rec=5)
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    model = tuple(to_dev(a, torch.float32) for a in (w.s, w.xi, w.eta))
    o = tt.default_opts(tt.TT_F32)
    ms = tt.tt_autotune(ctx, model, w.src, o)
    timed = {k: v for k, v in ms.items() if v > 0}
    assert len(timed) == 7          # 40 sources: the tile schedules run too
    best = min(timed, key=timed.get)
    want = (1, [1, 2, 4, 8][list(ms).index(best)]) if best.startswith("nodes") else \
        (2 + ["tiles 2x4x8", "tiles 4x4x4", "tiles 2x8x8"].index(best), 0)
    assert (o.sweep_schedule, o.fwd_groups) == want
    ref = gpu_solve(w, "f32", steps=("fwd",), ctx=ctx)
    tuned = gpu_solve(w, "f32", opts=o, steps=("fwd",), ctx=ctx)
    assert np.array_equal(ref["tau"], tuned["tau"])
    o2 = tt.default_opts(tt.TT_F32)
    assert all(v == 0 for v in tt.tt_autotune(ctx, model, w.src, o2).values())
    assert (o2.sweep_schedule, o2.fwd_groups) == want
    for g in (1, 2, 3, 8):          # any group count gives the same bits
        out = gpu_solve(w, "f32", opts=tt.default_opts(tt.TT_F32, fwd_groups=g), steps=("fwd",),
                        ctx=ctx)
        assert np.array_equal(ref["tau"], out["tau"])
    ctx.close()


def test_adjoint_autotuner_picks_a_measured_candidate_with_identical_results(tt):
    """The adjoint tuner times whole adjoint solves in each launch configuration (source
    chunks, barrier groups) and keeps the fastest; every configuration gives the default
    solve's bits, and a second call reuses the cached choice."""
    import torch
    w = I.small_case(17, shape=(14, 17, 19), n_src=256, n_rec=7)
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    model = tuple(to_dev(a, torch.float32) for a in (w.s, w.xi, w.eta))
    ref = gpu_solve(w, "f32", ctx=ctx, steps=("fwd", "misfit", "adj"))
    T = to_dev(ref["T"], torch.float32)
    R = to_dev(ref["R"], torch.float64)
    o = tt.default_opts(tt.TT_F32)
    ms = tt.tt_autotune_adjoint(ctx, model, w.src, T, w.rec, R, o)
    timed = {k: v for k, v in ms.items() if v > 0}
    assert len(timed) == 6          # 256 sources: every candidate runs (8 groups of 32)
    best = min(timed, key=timed.get)
    c = list(ms).index(best)
    assert (o.adj_chunk, o.adj_groups) == ([0, 0, 0, 0, 128, 64][c], [1, 2, 4, 8, 0, 1][c])
    o2 = tt.default_opts(tt.TT_F32)
    assert all(v == 0 for v in tt.tt_autotune_adjoint(ctx, model, w.src, T, w.rec, R,
                                                       o2).values())
    assert (o2.adj_chunk, o2.adj_groups) == (o.adj_chunk, o.adj_groups)
    for chunk, groups in ((0, 1), (0, 8), (64, 1), (128, 0), (96, 3)):
        P = torch.empty_like(T)
        it = tt.tt_adjoint(ctx, model, w.src, T, w.rec, R, P,
                           tt.default_opts(tt.TT_F32, adj_chunk=chunk, adj_groups=groups))
        assert np.array_equal(P.cpu().numpy(), ref["P"]), (chunk, groups)
        assert np.array_equal(it, ref["iters_adj"])
    ctx.close()


@pytest.mark.parametrize("slots", [32, 64])
def test_retire_and_refill_gives_the_resident_bits(tt, slots):
    """One launch with `slots` sources in flight, each converged source handing its slot to
    the next queued one, performs every source's arithmetic as the all-resident launch:
    same tau, T and iteration counts, from tau = 1 and from a given tau, under an
    iteration cap (statuses and counts), and inside a captured plan."""
    import torch
    w = I.small_case(17, shape=(13, 15, 16), n_src=80, n_rec=5)
    ref = gpu_solve(w, "f32", steps=("fwd",))
    o = tt.default_opts(tt.TT_F32, fwd_slots=slots)
    out = gpu_solve(w, "f32", opts=o, steps=("fwd",))
    assert np.array_equal(out["iters_fwd"], ref["iters_fwd"])
    assert np.array_equal(out["tau"], ref["tau"]) and np.array_equal(out["T"], ref["T"])
    start = (1.0 + 0.97 * (ref["tau"] - 1.0)).astype(np.float32)
    a = gpu_solve(w, "f32", opts=tt.default_opts(tt.TT_F32, init=1), steps=("fwd",), tau_init=start)
    b = gpu_solve(w, "f32", opts=tt.default_opts(tt.TT_F32, init=1, fwd_slots=slots),
                  steps=("fwd",), tau_init=start)
    assert np.array_equal(a["iters_fwd"], b["iters_fwd"]) and np.array_equal(a["tau"], b["tau"])
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    model = tuple(to_dev(x, torch.float32) for x in (w.s, w.xi, w.eta))
    res = []
    for s in (0, slots):
        tau = torch.empty(w.grid.shape + (w.n_src,), device="cuda")
        oc = tt.default_opts(tt.TT_F32, max_iter_fwd=3, fwd_slots=s)
        with pytest.raises(tt.TTError) as e:
            tt.tt_forward(ctx, model, w.src, tau, None, oc)
        assert e.value.status == tt.TT_ENOTCONVERGED
        res.append((tt.tt_forward(ctx, model, w.src, tau, None, oc, allow_unconverged=True),
                    tau.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0]) and (res[1][0] == 3).all()
    assert np.array_equal(res[0][1], res[1][1])
    # a plan with refill replays the step with the same bits
    full = gpu_solve(w, "f32")
    shape = w.grid.shape + (w.n_src,)
    tau, T, P = (torch.empty(shape, device="cuda") for _ in range(3))
    data = tt.DeviceData.from_workload(w)
    chi = torch.empty((w.n_src, 2), dtype=torch.float64, device="cuda")
    R = torch.empty((w.n_src, data.n_rec), dtype=torch.float64, device="cuda")
    K = [torch.empty(w.grid.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    plan = tt.tt_plan_create(ctx, model, w.src, data, tau, T, P, chi, R, *K, opts=o)
    itf, _ = tt.tt_plan_run(plan)
    assert np.array_equal(itf, full["iters_fwd"])
    assert np.array_equal(tau.cpu().numpy(), full["tau"])
    assert np.array_equal(P.cpu().numpy(), full["P"])
    plan.close()
    ctx.close()


def test_plan_with_common_receiver_terms_equals_the_calls(tt):
    """A plan that includes the common-receiver terms (Eq. 4, A4) gives the bits of the
    individual calls: forward, misfit (receiver times), tt_misfit_cr, adjoint, kernels; and a
    plan whose entries name a source outside the batch is refused at creation."""
    import torch
    w = I.small_case(18, shape=(13, 14, 16), n_src=37, n_rec=9)
    rng = np.random.default_rng(18)
    pairs = [(b, j, m, rng.normal(0, 0.3), rng.uniform(0.5, 2.0))
             for m in range(9) for b in range(37) for j in range(b + 1, 37)
             if rng.uniform() < 0.1]
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    model = tuple(to_dev(a, torch.float32) for a in (w.s, w.xi, w.eta))
    shape = w.grid.shape + (w.n_src,)
    data = tt.DeviceData.from_workload(w)
    cr = tt.CrData(w.n_src, data.n_rec, pairs, gamma=0.8)
    f64 = dict(dtype=torch.float64, device="cuda")
    # the calls
    tau, T, P = (torch.empty(shape, device="cuda") for _ in range(3))
    Tr, chi, R = (torch.empty((w.n_src, data.n_rec), **f64), torch.empty((w.n_src, 2), **f64),
                  torch.empty((w.n_src, data.n_rec), **f64))
    chi_cr = torch.empty(w.n_src, **f64)
    itf = tt.tt_forward(ctx, model, w.src, tau, T)
    tt.tt_misfit(ctx, T, data, Tr, chi, R)
    tt.tt_misfit_cr(ctx, cr, Tr, chi_cr, R)
    ita = tt.tt_adjoint(ctx, model, w.src, T, w.rec, R, P)
    K = [torch.zeros(w.grid.shape, **f64) for _ in range(3)]
    tt.tt_kernel(ctx, model, T, P, *K)
    ref = [x.cpu().numpy() for x in (tau, P, Tr, chi, R, chi_cr, *K)]
    # the plan
    tau2, T2, P2 = (torch.empty(shape, device="cuda") for _ in range(3))
    Tr2, chi2, R2 = (torch.empty_like(Tr), torch.empty_like(chi), torch.empty_like(R))
    chi_cr2 = torch.empty_like(chi_cr)
    K2 = [torch.empty(w.grid.shape, **f64) for _ in range(3)]
    plan = tt.tt_plan_create(ctx, model, w.src, data, tau2, T2, P2, chi2, R2, *K2, cr=cr,
                             Tr=Tr2, chi_cr=chi_cr2)
    for _ in range(2):
        itf2, ita2 = tt.tt_plan_run(plan)
        assert np.array_equal(itf2, itf) and np.array_equal(ita2, ita)
        got = [x.cpu().numpy() for x in (tau2, P2, Tr2, chi2, R2, chi_cr2, *K2)]
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
    assert np.abs(ref[5]).max() > 0
    plan.close()
    cr.other[0] = w.n_src + 2
    with pytest.raises(tt.TTError, match="outside the batch"):
        tt.tt_plan_create(ctx, model, w.src, data, tau2, T2, P2, chi2, R2, *K2, cr=cr,
                          Tr=Tr2, chi_cr=chi_cr2)
    ctx.close()
