"""Trains the warm-start network on the GPU and writes its weights.

The data are forward solves that the library itself computes, over random-field models
(Gaussian random fields of correlation length 10 km; sigma 3 % on Vp, 2 % on xi and eta
clipped to +-0.04; 5 -> 8 km/s background) on a grid of the given shape, depth and extents
(default 81 x 81 x 81, depth 0-60 km, 2 x 2 deg), with --sources sources per model (default
8). 10 % of the models are held out. The script reports:
- the training loss;
- the prediction error against the converged tau;
- the sweeps to convergence with and without the warm start on the held-out models.
With --stride 2 the network runs on every other node along each axis (its targets are the
converged tau there) and the warm start interpolates its prediction to the other nodes.

Run from the repository root (it draws the models with tt_inputs):

    python -m paper_2412_00031_gb300.train_warmstart --models 250 --out warmstart_81.npz

The committed weights: warmstart_81.npz (the network on every node) and warmstart_81_s2.npz
(every other node; the benchmark's warm start), the latter from

    python -m paper_2412_00031_gb300.train_warmstart --stride 2 --tensor-cores \
        --out paper_2412_00031_gb300/warmstart_81_s2.npz
"""
import argparse
import json
import os
import sys
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--models", type=int, default=250)
    ap.add_argument("--sources", type=int, default=8)
    ap.add_argument("--shape", type=int, nargs=3, default=(81, 81, 81))
    ap.add_argument("--depth-km", type=float, default=60.0)
    ap.add_argument("--extent-deg", type=float, nargs=2, default=(2.0, 2.0),
                    help="latitude and longitude extents of the grid")
    ap.add_argument("--src-depth", type=float, nargs=2, default=(5.0, 40.0),
                    help="source depth range in km")
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=20241203)
    ap.add_argument("--tensor-cores", action="store_true",
                    help="gradients with the convolutions on the tensor cores (BF16 operands)")
    ap.add_argument("--stride", type=int, default=1, choices=(1, 2),
                    help="the network's grid: 1 = every node, 2 = every other node along each "
                         "axis (the warm start interpolates to the others)")
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "warmstart_81.npz"))
    a = ap.parse_args(argv)
    sys.path.insert(0, os.getcwd())
    import torch
    import tt_inputs as I
    import paper_2412_00031_gb300 as tt
    from paper_2412_00031_gb300 import warmstart as WS

    t0 = time.time()
    g, models = I.random_field_models(seed=a.seed, n_models=a.models, shape=tuple(a.shape),
                                      depth_km=a.depth_km, extent_deg=tuple(a.extent_deg),
                                      n_src=a.sources, depth_range=tuple(a.src_depth))
    n_hold = max(1, a.models // 10)
    train_models, hold_models = models[:-n_hold], models[-n_hold:]
    ctx = tt.tt_ctx_create(g.as_dict())
    tt.tt_net_set_stride(ctx, a.stride)
    t1 = time.time()
    x, t, m, iters = WS.make_samples(ctx, g.shape, train_models)
    torch.cuda.synchronize()
    t2 = time.time()
    theta, losses = WS.train(ctx, x, t, m, WS.init_params(a.seed), steps=a.steps,
                             batch=a.batch, lr=a.lr, seed=a.seed, log_every=100,
                             tensor_cores=a.tensor_cores)
    torch.cuda.synchronize()
    t3 = time.time()
    del x, t, m
    # held-out: prediction error and sweeps with / without the warm start
    tt.tt_net_set_weights(ctx, theta)
    xh, th, _, cold = WS.make_samples(ctx, g.shape, hold_models)
    y = torch.empty(th.shape, dtype=torch.float32, device=th.device)
    tt.tt_net_forward(ctx, theta, xh, y)
    pred = 1.0 + y.clamp(-0.5, 1.0)
    err_net = float((pred - th).abs().amax())
    err_one = float((1.0 - th).abs().amax())
    rms_net = float(((pred - th) ** 2).mean().sqrt())
    rms_one = float(((1.0 - th) ** 2).mean().sqrt())
    warm = []
    for s, xi, eta, src in hold_models:
        model = tuple(torch.as_tensor(np.ascontiguousarray(f), dtype=torch.float32, device="cuda")
                      for f in (s, xi, eta))
        tau = torch.empty(g.shape + (len(src),), device="cuda")
        warm.append(tt.tt_forward(ctx, model, src, tau, None, tt.default_opts(tt.TT_F32, init=2)))
    warm = np.concatenate(warm)
    summary = {
        "grid": list(g.shape), "depth_km": a.depth_km, "extent_deg": list(a.extent_deg),
        "src_depth_km": list(a.src_depth), "sources_per_model": a.sources,
        "models_train": len(train_models), "models_held_out": n_hold,
        "solves_train": int(len(iters)), "steps": a.steps, "batch": a.batch, "lr": a.lr,
        "loss_first": float(np.mean(losses[:10])), "loss_last": float(np.mean(losses[-50:])),
        "held_out_max_err": err_net, "held_out_max_err_tau1": err_one,
        "held_out_rms_err": rms_net, "held_out_rms_err_tau1": rms_one,
        "held_out_sweeps_cold": float(cold.mean()), "held_out_sweeps_warm": float(warm.mean()),
        "seconds_data": t2 - t1, "seconds_train": t3 - t2, "seconds_models": t1 - t0,
        "gradient": "tensor cores (BF16 operands)" if a.tensor_cores else "FP32",
        "stride": a.stride,
    }
    np.savez(a.out, theta=theta.cpu().numpy(), losses=np.asarray(losses),
             summary=json.dumps(summary))
    print(json.dumps(summary))
    ctx.close()


if __name__ == "__main__":
    main()
