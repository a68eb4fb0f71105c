"""Warm-start network on the GPU against the FP64 oracle (oracle/net.py), through the C ABI:
features, forward pass, loss and gradient, the optimiser step, the zero network as a
no-op, and what a trained network gains over the cold start (needs a GB300)."""
import numpy as np
import pytest

import tt_inputs as I
from gpu_helpers import rel_linf, to_dev
from oracle import net as N

pytestmark = pytest.mark.gpu

# Tensor-core training (BF16 operands). With u = 2^-9, the unit roundoff of BF16, the input
# gradient reaching layer 1 has been rounded about 8 times (the output gradient, three
# transposed convolutions' BF16 weights and outputs, the activations that gate them), so the
# per-layer bar is 16 u, the whole gradient's 8 u and the loss's (one forward pass) 5 u.
# Measured: 8.5 u for layer 1's weights, 2.3 u in all, 0.34 u for the loss.
BF16_U = 2.0 ** -9
TC_LOSS_BAR = 5 * BF16_U
TC_GRAD_BAR_LAYER = 16 * BF16_U
TC_GRAD_BAR = 8 * BF16_U


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_00031_gb300 as m
    return m


def _theta(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in N.LAYERS:
        bound = scale * np.sqrt(6.0 / (27 * ci))
        parts += [rng.uniform(-bound, bound, 27 * ci * co), rng.uniform(-0.05, 0.05, co)]
    return np.concatenate(parts).astype(np.float32)


def _gpu_features(tt, w, dtype):
    import torch
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    model = tuple(to_dev(a, dtype) for a in (w.s, w.xi, w.eta))
    x = torch.empty((w.n_src,) + w.grid.shape + (6,), dtype=torch.float32, device="cuda")
    tt.tt_net_features(ctx, model, w.src, x)
    out = x.cpu().numpy()
    ctx.close()
    return out


@pytest.mark.parametrize("flat", [0, 1])
def test_features_match_oracle(tt, flat):
    import torch
    w = I.small_case(51 + flat, shape=(11, 13, 12), n_src=3, n_rec=4, flat=flat)
    ref = np.stack([N.features(w.grid.as_dict(), w.s, w.xi, w.eta, w.src[b])
                    for b in range(w.n_src)])
    for dt, tol in ((torch.float64, 1e-6), (torch.float32, 1e-5)):
        got = _gpu_features(tt, w, dt)
        assert np.abs(got - ref).max() <= tol * max(1.0, np.abs(ref).max())


def _oracle_inputs(seed, shape=(9, 10, 11), n=2):
    w = I.small_case(seed, shape=shape, n_src=n, n_rec=4)
    xs = [N.features(w.grid.as_dict(), w.s, w.xi, w.eta, w.src[b]).astype(np.float32)
          for b in range(n)]
    return w, xs


def test_forward_matches_oracle(tt):
    import torch
    w, xs = _oracle_inputs(61)
    theta = _theta(7)
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    x = torch.as_tensor(np.stack(xs), device="cuda")
    y = torch.empty(x.shape[:-1], dtype=torch.float32, device="cuda")
    tt.tt_net_forward(ctx, torch.as_tensor(theta, device="cuda"), x, y)
    ctx.close()
    for b in range(len(xs)):
        ref = N.forward(theta.astype(np.float64), xs[b].astype(np.float64))
        assert np.abs(y[b].cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()


def test_loss_gradient_matches_oracle(tt):
    """The GPU's backward pass (transposed convolutions, ReLU masks, weight-gradient
    reductions) gives the oracle's gradient of the masked MSE to FP32 accuracy."""
    import torch
    w, xs = _oracle_inputs(62, shape=(10, 9, 12), n=3)
    rng = np.random.default_rng(8)
    theta = _theta(9)
    taus = [(1.0 + 0.05 * rng.standard_normal(w.grid.shape)).astype(np.float32) for _ in xs]
    masks = [(rng.uniform(size=w.grid.shape) > 0.3).astype(np.float32) for _ in xs]
    loss_ref, g_ref = N.loss_and_grad(theta.astype(np.float64), [x.astype(np.float64) for x in xs],
                                      [t.astype(np.float64) - 1.0 for t in taus],
                                      [m.astype(np.float64) for m in masks])
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    d = lambda a: torch.as_tensor(np.ascontiguousarray(np.stack(a)), device="cuda")
    grad = torch.empty(tt.tt_net_param_count(), dtype=torch.float32, device="cuda")
    th = torch.as_tensor(theta, device="cuda")
    loss = tt.tt_net_loss_grad(ctx, th, d(xs), d(taus), d(masks), grad)
    g = grad.cpu().numpy().astype(np.float64)
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    k = 0
    for ci, co in N.LAYERS:   # every layer's weights and biases, not just the total
        for n in (27 * ci * co, co):
            a, b = g[k:k + n], g_ref[k:k + n]
            assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b) + 1e-12, (ci, co, n)
            k += n
    # deterministic: the same call gives the same bits
    grad2 = torch.empty_like(grad)
    loss2 = tt.tt_net_loss_grad(ctx, th, d(xs), d(taus), d(masks), grad2)
    assert loss2 == loss and torch.equal(grad, grad2)
    ctx.close()


def test_tensor_core_loss_gradient_matches_oracle_to_bf16_accuracy(tt):
    """Training with the convolutions on the tensor cores (tt_net_loss_grad_tc): BF16
    weights, activations and gradients, FP32 accumulation. Against the FP64 oracle's loss
    and gradient on the inputs of the FP32 test, per layer (weights and biases), and
    bitwise deterministic."""
    import torch
    w, xs = _oracle_inputs(62, shape=(10, 9, 12), n=3)
    rng = np.random.default_rng(8)
    theta = _theta(9)
    taus = [(1.0 + 0.05 * rng.standard_normal(w.grid.shape)).astype(np.float32) for _ in xs]
    masks = [(rng.uniform(size=w.grid.shape) > 0.3).astype(np.float32) for _ in xs]
    loss_ref, g_ref = N.loss_and_grad(theta.astype(np.float64), [x.astype(np.float64) for x in xs],
                                      [t.astype(np.float64) - 1.0 for t in taus],
                                      [m.astype(np.float64) for m in masks])
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    d = lambda a: torch.as_tensor(np.ascontiguousarray(np.stack(a)), device="cuda")
    grad = torch.empty(tt.tt_net_param_count(), dtype=torch.float32, device="cuda")
    th = torch.as_tensor(theta, device="cuda")
    loss = tt.tt_net_loss_grad_tc(ctx, th, d(xs), d(taus), d(masks), grad)
    g = grad.cpu().numpy().astype(np.float64)
    errs = []
    k = 0
    for ci, co in N.LAYERS:
        for n in (27 * ci * co, co):
            a, b = g[k:k + n], g_ref[k:k + n]
            errs.append(np.linalg.norm(a - b) / np.linalg.norm(b))
            k += n
    total = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    print("\ntensor-core gradient: loss rel err %.2e, total %.2e, per layer %s" % (
        abs(loss / loss_ref - 1), total, " ".join("%.2e" % e for e in errs)))
    assert abs(loss / loss_ref - 1) <= TC_LOSS_BAR
    assert total <= TC_GRAD_BAR and max(errs) <= TC_GRAD_BAR_LAYER
    grad2 = torch.empty_like(grad)
    loss2 = tt.tt_net_loss_grad_tc(ctx, th, d(xs), d(taus), d(masks), grad2)
    assert loss2 == loss and torch.equal(grad, grad2)
    ctx.close()


def test_adam_step(tt):
    import torch
    rng = np.random.default_rng(10)
    n = tt.tt_net_param_count()
    th, g = rng.standard_normal(n).astype(np.float32), rng.standard_normal(n).astype(np.float32)
    m0, v0 = (0.1 * rng.standard_normal(n)).astype(np.float32), rng.uniform(0, 0.1, n).astype(np.float32)
    ctx = tt.tt_ctx_create(I.small_case(1, shape=(5, 5, 5)).grid.as_dict())
    T, G, M, V = (torch.as_tensor(a, device="cuda") for a in (th, g, m0, v0))
    tt.tt_net_adam(ctx, T, G, M, V, 3, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)
    ctx.close()
    m1 = 0.9 * m0 + 0.1 * g
    v1 = 0.999 * v0 + 0.001 * g * g
    ref = th - 1e-2 * (m1 / (1 - 0.9 ** 3)) / (np.sqrt(v1 / (1 - 0.999 ** 3)) + 1e-8)
    assert np.allclose(T.cpu().numpy(), ref, rtol=1e-5, atol=1e-6)
    assert np.allclose(M.cpu().numpy(), m1, rtol=1e-6, atol=1e-7)


def test_zero_network_warm_start_is_the_cold_start(tt):
    """All-zero weights predict tau = 1: the warm-started solve is bit for bit the cold one."""
    import torch
    from gpu_helpers import gpu_solve
    w = I.small_case(63, shape=(13, 14, 15), n_src=5, n_rec=4)
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    tt.tt_net_set_weights(ctx, torch.zeros(tt.tt_net_param_count(), device="cuda"))
    cold = gpu_solve(w, "f32", steps=("fwd",), ctx=ctx)
    warm = gpu_solve(w, "f32", opts=tt.default_opts(tt.TT_F32, init=2), steps=("fwd",), ctx=ctx)
    ctx.close()
    assert np.array_equal(warm["iters_fwd"], cold["iters_fwd"])
    assert np.array_equal(warm["tau"], cold["tau"])


def test_warm_start_needs_weights(tt):
    import torch
    w = I.small_case(64, shape=(9, 9, 9), n_src=1, n_rec=3)
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    model = tuple(to_dev(a, torch.float32) for a in (w.s, w.xi, w.eta))
    tau = torch.empty(w.grid.shape + (1,), device="cuda")
    with pytest.raises(tt.TTError) as e:
        tt.tt_forward(ctx, model, w.src, tau, None, tt.default_opts(tt.TT_F32, init=2))
    assert e.value.status == tt.TT_EINVAL
    ctx.close()


@pytest.mark.parametrize("tensor_cores", [False, True], ids=["fp32-gradient", "tensor-core-gradient"])
def test_trained_network_gains_over_the_cold_start(tt, capsys, tensor_cores):
    """Trains the network on the GPU (forward solves of random-field models as data, the
    library's loss, gradient and Adam kernels; the gradient in FP32 or with the convolutions
    on the tensor cores) and measures on held-out models: the prediction is closer to the
    converged tau than tau = 1, the warm-started sweep meets the same tolerance, and it takes
    no more sweeps than the cold start."""
    import torch
    from paper_2412_00031_gb300 import warmstart as WS
    g, models = I.random_field_models(seed=I.SEED_BASE + 30, n_models=14, shape=(25, 25, 25),
                                      depth_km=24.0, extent_deg=0.3, n_src=4,
                                      depth_range=(4.0, 20.0))
    ctx = tt.tt_ctx_create(g.as_dict())
    x, t, m, _ = WS.make_samples(ctx, g.shape, models[:12])
    theta, losses = WS.train(ctx, x, t, m, WS.init_params(1), steps=300, batch=4, lr=2e-3, seed=2,
                             tensor_cores=tensor_cores)
    assert np.mean(losses[-20:]) < 0.2 * np.mean(losses[:5])
    tt.tt_net_set_weights(ctx, theta)
    xh, th, _, cold_iters = WS.make_samples(ctx, g.shape, models[12:])
    y = torch.empty(th.shape, dtype=torch.float32, device="cuda")
    tt.tt_net_forward(ctx, theta, xh, y)
    pred = 1.0 + y.clamp(-0.5, 1.0)
    err_net = (pred - th).abs().amax().item()
    err_one = (1.0 - th).abs().amax().item()
    assert err_net < 0.5 * err_one
    warm_iters = []
    for s, xi, eta, src in models[12:]:
        model = tuple(to_dev(a, torch.float32) for a in (s, xi, eta))
        tau_c = torch.empty(g.shape + (len(src),), device="cuda")
        tau_w = torch.empty_like(tau_c)
        tt.tt_forward(ctx, model, src, tau_c, None, tt.default_opts(tt.TT_F32))
        warm_iters.append(tt.tt_forward(ctx, model, src, tau_w, None,
                                        tt.default_opts(tt.TT_F32, init=2)))
        assert rel_linf(tau_w.cpu().numpy(), tau_c.cpu().numpy()) <= 1e-5
    warm_iters = np.concatenate(warm_iters)
    with capsys.disabled():
        print("\nwarm start (%s gradient): held-out max |tau - tau*| %.3e (tau = 1: %.3e); "
              "sweeps %.2f -> %.2f" % ("tensor-core" if tensor_cores else "FP32", err_net, err_one,
                                      cold_iters.mean(), warm_iters.mean()))
    assert warm_iters.mean() <= cold_iters.mean()
    ctx.close()


def _bf16(a):
    """Round float32 values to the nearest BF16 (ties to even), kept as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    r = (u + np.uint32(0x7FFF) + ((u >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)
    return r.view(np.float32)


def test_tensor_core_inference_matches_oracle(tt):
    """The warm start's inference (all four layers on the tensor cores with tcgen05: BF16
    operands, features and activations, FP32 accumulation) against the FP64 network with the
    same BF16 weights. Bound: four BF16 roundings of the layer inputs (2^-9 relative each)
    through layers of gain ~1 leave the output within 2 % of its range. 13 x 12 x 17 grids:
    24 tiles of 128 padded rows per grid, the last one ragged."""
    import torch
    w, xs = _oracle_inputs(65, shape=(13, 12, 17), n=2)
    theta = _theta(11)
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    tt.tt_net_set_weights(ctx, torch.as_tensor(theta, device="cuda"))
    x = torch.as_tensor(np.stack(xs), device="cuda")
    y = torch.empty(x.shape[:-1], dtype=torch.float32, device="cuda")
    tt.tt_net_infer(ctx, x, y)
    y32 = torch.empty_like(y)
    tt.tt_net_forward(ctx, torch.as_tensor(theta, device="cuda"), x, y32)
    ctx.close()
    tb = _bf16(theta).astype(np.float64)
    for b in range(len(xs)):
        ref = N.forward(tb, xs[b].astype(np.float64))
        scale = np.abs(ref).max()
        got = y[b].cpu().numpy()
        assert np.abs(got - ref).max() <= 2e-2 * scale
        assert np.corrcoef(got.ravel(), ref.ravel())[0, 1] > 0.9999
        assert np.abs(got - y32[b].cpu().numpy()).max() <= 2e-2 * scale


def test_tensor_core_inference_wide_and_small_grids(tt):
    """The tensor-core inference where the 126-row tile steps do not line up with the grid:
    a wide grid (260 phi nodes: a theta row spans three tiles) and a batch of three small
    grids (7 x 5 x 9: 420 rows each, ragged last tiles). Against the FP64 network with the
    same BF16 weights, to the bound of the test above."""
    import torch
    theta = _theta(12)
    tb = _bf16(theta).astype(np.float64)
    for seed, shape, n in ((66, (6, 5, 260), 1), (67, (7, 5, 9), 3)):
        w, xs = _oracle_inputs(seed, shape=shape, n=n)
        ctx = tt.tt_ctx_create(w.grid.as_dict())
        tt.tt_net_set_weights(ctx, torch.as_tensor(theta, device="cuda"))
        x = torch.as_tensor(np.stack(xs), device="cuda")
        y = torch.empty(x.shape[:-1], dtype=torch.float32, device="cuda")
        tt.tt_net_infer(ctx, x, y)
        ctx.close()
        for b in range(n):
            ref = N.forward(tb, xs[b].astype(np.float64))
            got = y[b].cpu().numpy()
            assert np.abs(got - ref).max() <= 2e-2 * np.abs(ref).max(), (shape, b)


@pytest.mark.parametrize("dt_name", ["f32", "f64"])
def test_coarse_grid_warm_start_matches_oracle(tt, dt_name):
    """The network on every other node (tt_net_set_stride(ctx, 2)) and its clamped prediction
    interpolated trilinearly to every node (tt_net_start), against the oracle: the features
    at the network nodes against the oracle's features of those nodes; the start against the
    oracle's FP64 network with the same BF16 weights on those features, interpolated
    (warm_start_coarse). 13 x 14 x 15 nodes: a 7 x 8 x 8 network grid, whose last interval
    along the even axis is half as long. Bound as for the inference (2 % of the prediction's
    range); tau = 1 at the node nearest each source (its fixed set)."""
    import torch
    w = I.small_case(68, shape=(13, 14, 15), n_src=3, n_rec=4)
    theta = _theta(13)
    dtype = torch.float32 if dt_name == "f32" else torch.float64
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    tt.tt_net_set_stride(ctx, 2)
    assert tt.tt_net_nodes(ctx) == 7 * 8 * 8 == tt.lib.tt_net_nodes(ctx.handle)
    model = tuple(to_dev(a, dtype) for a in (w.s, w.xi, w.eta))
    x = torch.empty((w.n_src, 7 * 8 * 8, 6), dtype=torch.float32, device="cuda")
    tt.tt_net_features(ctx, model, w.src, x)
    tt.tt_net_set_weights(ctx, torch.as_tensor(theta, device="cuda"))
    tau = torch.empty(w.grid.shape + (w.n_src,), dtype=dtype, device="cuda")
    tt.tt_net_start(ctx, model, w.src, tau)
    ctx.close()
    got = tau.cpu().numpy()
    idx = [N.coarse_nodes(n, 2) for n in w.grid.shape]
    tb = _bf16(theta).astype(np.float64)
    r, th, ph, re, _ = N._axes_rad(w.grid.as_dict())
    for b in range(w.n_src):
        xc = N.features(w.grid.as_dict(), w.s, w.xi, w.eta, w.src[b])[np.ix_(*idx)]
        xg = x[b].cpu().numpy().reshape(xc.shape)
        assert np.abs(xg - xc).max() <= 1e-5 * max(1.0, np.abs(xc).max())
        ref = N.warm_start_coarse(tb, xg.astype(np.float64), w.grid.shape, 2)
        depth, lat, lon = w.src[b]
        near = [int(round(v)) for v in ((re - depth - r[0]) / (r[1] - r[0]),
                                         (np.deg2rad(lat) - th[0]) / (th[1] - th[0]),
                                         (np.deg2rad(lon) - ph[0]) / (ph[1] - ph[0]))]
        I3 = np.meshgrid(*[np.arange(n) for n in w.grid.shape], indexing="ij")
        away = np.max([np.abs(I3[a] - near[a]) for a in range(3)], axis=0) > 2
        scale = np.abs(ref - 1).max()
        assert scale > 0.05
        assert np.abs(got[..., b][away] - ref[away]).max() <= 2e-2 * scale
        assert got[..., b][tuple(near)] == 1.0


def test_broken_network_costs_sweeps_not_accuracy(tt):
    """A network that predicts NaN everywhere (NaN weights) starts every node at tau = 1,
    so the warm-started solve is bit for bit the cold one. A network with huge weights
    (outputs overflow; the clamp keeps tau in [0.5, 2]) still converges to the cold solve's
    fixed point within the tolerance."""
    import torch
    from gpu_helpers import gpu_solve
    w = I.small_case(66, shape=(13, 14, 15), n_src=5, n_rec=4)
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    n = tt.tt_net_param_count()
    cold = gpu_solve(w, "f32", steps=("fwd",), ctx=ctx)
    warm_opts = tt.default_opts(tt.TT_F32, init=2)
    tt.tt_net_set_weights(ctx, torch.full((n,), float("nan"), device="cuda"))
    warm = gpu_solve(w, "f32", opts=warm_opts, steps=("fwd",), ctx=ctx)
    assert np.array_equal(warm["iters_fwd"], cold["iters_fwd"])
    assert np.array_equal(warm["tau"], cold["tau"])
    g = torch.Generator().manual_seed(66)
    tt.tt_net_set_weights(ctx, (1e3 * torch.randn(n, generator=g)).to("cuda"))
    warm = gpu_solve(w, "f32", opts=warm_opts, steps=("fwd",), ctx=ctx)
    ctx.close()
    assert np.all(np.isfinite(warm["tau"]))
    assert rel_linf(warm["tau"], cold["tau"]) <= 1e-5
