"""Training driver of the warm-start network (argument marshalling over the C ABI).

Every arithmetic step runs in libttgb's kernels. The steps are:
- the forward solves that produce the targets (tt_forward);
- the input features (tt_net_features);
- the loss and its gradient (tt_net_loss_grad in FP32, or tt_net_loss_grad_tc with the
  convolutions on the tensor cores);
- the optimiser (tt_net_adam).

This module only orders the calls, draws the seeded initial weights and the sample order,
and keeps the tensors. Samples are full grids: the network input x[n] is the feature array
of one (model, source) pair, the target t[n] the tau of its converged forward solve (the
loss compares the output with tau - 1), and
the mask m[n] is 1 everywhere (on the fixed set tau = 1 and the target is met exactly by
y = 0, which the clamp of the warm start does not need).
"""
import numpy as np

from . import (TT_F32, default_opts, tt_forward, tt_net_adam, tt_net_features,
               tt_net_loss_grad, tt_net_loss_grad_tc, tt_net_param_count)

LAYERS = ((6, 32), (32, 32), (32, 32), (32, 1))


def init_params(seed):
    """He-uniform weights (bound sqrt(6 / fan_in), fan_in = 27 C_in), zero biases, as one
    float32 vector in the C ABI's order."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in LAYERS:
        bound = np.sqrt(6.0 / (27 * ci))
        parts += [rng.uniform(-bound, bound, 27 * ci * co), np.zeros(co)]
    theta = np.concatenate(parts).astype(np.float32)
    assert theta.size == tt_net_param_count()
    return theta


def net_shape(grid_shape, stride):
    """Shape of the network's grid: every stride-th node along each axis, the last included."""
    return tuple(n if stride == 1 else (n + stride - 2) // stride + 1 for n in grid_shape)


def make_samples(ctx, grid_shape, models, device="cuda", opts=None):
    """Forward-solves every (model, source) pair in FP32 and returns device tensors
    x [n, Nr, Nt, Np, 6] (the features on the network's grid, tt_net_set_stride), t
    [n, Nr, Nt, Np] (the converged tau at those nodes), m (mask), and the forward iteration
    counts. models: list of (s, xi, eta, src) numpy arrays. The loss compares the network
    output with t - 1."""
    import torch
    xs, ts, ms, iters = [], [], [], []
    o = opts if opts is not None else default_opts(TT_F32)
    c = getattr(ctx, "net_stride", 1)
    shape = net_shape(grid_shape, c)
    # node indices of the network grid along each axis (min(a c, n - 1))
    idx = [torch.as_tensor(np.minimum(np.arange(m) * c, n - 1), device=device)
           for m, n in zip(shape, grid_shape)]
    for s, xi, eta, src in models:
        model = tuple(torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=device)
                      for a in (s, xi, eta))
        B = len(src)
        tau = torch.empty(tuple(grid_shape) + (B,), dtype=torch.float32, device=device)
        iters.append(tt_forward(ctx, model, src, tau, None, o))
        x = torch.empty((B,) + shape + (6,), dtype=torch.float32, device=device)
        tt_net_features(ctx, model, src, x)
        xs.append(x)
        if c > 1:
            tau = tau.index_select(0, idx[0]).index_select(1, idx[1]).index_select(2, idx[2])
        ts.append(tau.permute(3, 0, 1, 2).contiguous())
        ms.append(torch.ones_like(ts[-1]))
    return torch.cat(xs), torch.cat(ts), torch.cat(ms), np.concatenate(iters)


def train(ctx, x, t, m, theta0, steps, batch, lr=1e-3, seed=0, log_every=0,
          tensor_cores=False):
    """Adam on the masked MSE over mini-batches of whole grids. The sample order is a
    seeded permutation, re-drawn each epoch; a batch is a contiguous block of the permuted
    samples (gathered once per epoch). tensor_cores: gradients from tt_net_loss_grad_tc
    (convolutions on tcgen05, BF16 operands) instead of the FP32 tt_net_loss_grad. Returns
    (theta, losses)."""
    import torch
    theta = torch.as_tensor(theta0, dtype=torch.float32, device=x.device).clone()
    grad = torch.zeros_like(theta)
    mom1 = torch.zeros_like(theta)
    mom2 = torch.zeros_like(theta)
    rng = np.random.default_rng(seed)
    n = x.shape[0]
    losses = []
    step = 0
    while step < steps:
        perm = torch.as_tensor(rng.permutation(n), device=x.device)
        xp, tp, mp = x[perm].contiguous(), t[perm].contiguous(), m[perm].contiguous()
        for b0 in range(0, n - batch + 1, batch):
            if step >= steps:
                break
            fn = tt_net_loss_grad_tc if tensor_cores else tt_net_loss_grad
            loss = fn(ctx, theta, xp[b0:b0 + batch], tp[b0:b0 + batch], mp[b0:b0 + batch], grad)
            step += 1
            tt_net_adam(ctx, theta, grad, mom1, mom2, step, lr)
            losses.append(loss)
            if log_every and step % log_every == 0:
                print("step %d loss %.3e" % (step, loss), flush=True)
    return theta, losses
