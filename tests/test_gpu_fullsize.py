"""Parity at the full sizes of the benchmark configurations, on sampled sources (needs a GB300;
the FP64 oracle runs one source at a time on the host).

- 81^3 isotropic checkerboard, 64 sources: the FP32 batch against complete oracle solves
  of sampled sources (traveltime, adjoint state, and that source's kernels).
- 121 x 161 x 161 anisotropic batch, 256 sources, in the benchmark's launch configuration
  (autotuned launch, one captured graph per step): a complete oracle solve of one source
  takes minutes there, so the oracle restarts its sweeps from the GPU's tau for the source
  that took the most iterations. The oracle must reach its own FP64 fixed point in fewer
  than half the GPU's iterations, and that fixed point must match the GPU's traveltime to
  the 1e-5 bar.
  The oracle's adjoint state, computed from its own traveltime, must match the GPU's P to
  the 1e-3 bar.
- the same batch with the anisotropic Godunov forward (the benchmark's godunov leg), in its
  launch configuration: sampled sources solved alone give their batch columns' bits.
"""
import numpy as np
import pytest

import tt_inputs as I
from gpu_helpers import gpu_solve, rel_l2, rel_linf, rounded_model, to_dev

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_00031_gb300 as m
    return m


def test_checkerboard_81_fp32_batch_against_oracle_solves(tt):
    import oracle as O
    w = I.checkerboard_81()
    out = gpu_solve(w, "f32")
    s, xi, eta = rounded_model(w, "f32")
    g = w.grid.as_dict()
    solved = {}
    for b in (0, w.n_src - 1):
        r = O.solve_source(g, s, xi, eta, w.src[b], w.rec, w.source_data(b), tol_fwd=1e-9,
                           tol_adj=1e-9, max_iter=1000)
        assert r["conv_fwd"] and r["conv_adj"]
        assert rel_linf(out["T"][..., b], r["T"]) <= 1e-5
        assert rel_l2(out["P"][..., b], r["P"]) <= 1e-3
        solved[b] = r
    # one source's kernels: the GPU on that source alone (bitwise its batch column)
    one = gpu_solve(w.subset([0]), "f32")
    assert np.array_equal(one["T"][..., 0], out["T"][..., 0])
    K = [np.zeros(w.grid.shape) for _ in range(3)]
    O.kernel_add(g, s, solved[0]["T"], solved[0]["P"], *K)
    for a, k in zip(one["K"], K):
        assert rel_l2(a, k) <= 1e-3


def test_anisotropic_batch_in_the_benchmark_configuration(tt):
    import torch
    import oracle as O
    w = I.anisotropic_batch()
    g = w.grid
    model = tuple(to_dev(a, torch.float32) for a in (w.s, w.xi, w.eta))
    ctx = tt.tt_ctx_create(g.as_dict())
    o = tt.default_opts(tt.TT_F32)
    tt.tt_autotune(ctx, model, w.src, o)
    shape = g.shape + (w.n_src,)
    tau, T, P = (torch.empty(shape, device="cuda") for _ in range(3))
    data = tt.DeviceData.from_workload(w)
    chi = torch.empty((w.n_src, 2), dtype=torch.float64, device="cuda")
    R = torch.empty((w.n_src, data.n_rec), dtype=torch.float64, device="cuda")
    K = [torch.empty(g.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    plan = tt.tt_plan_create(ctx, model, w.src, data, tau, T, P, chi, R, *K, opts=o)
    itf, ita = tt.tt_plan_run(plan)
    b = int(np.argmax(itf))                       # the slowest source
    tau_b = tau[..., b].contiguous().cpu().numpy().astype(np.float64)
    T_b = T[..., b].contiguous().cpu().numpy()
    P_b = P[..., b].contiguous().cpu().numpy()
    plan.close()
    ctx.close()
    s, xi, eta = rounded_model(w, "f32")
    gd = g.as_dict()
    # from the GPU's tau the oracle needs a fraction of the ~64 iterations of a cold start;
    # the rest is the distance between the FP32 and FP64 fixed points (contraction ~0.68
    # per iteration)
    _, To, it, conv, _ = O.forward(gd, s, xi, eta, w.src[b], tol=1e-7, max_iter=30,
                                   tau_init=tau_b)
    print("\nsource %d: GPU %d iterations; oracle from the GPU's tau: %d" % (b, itf[b], it))
    assert conv and it < itf[b] // 2
    assert rel_linf(T_b, To) <= 1e-5
    d = w.source_data(b)
    Tr = O.receiver_times(gd, To, w.rec)
    _, _, Ro = O.misfit(Tr, d["abs_rec"], d["abs_tobs"], d["abs_w"], d["cs_m"], d["cs_i"],
                        d["cs_dtobs"], d["cs_w"])
    Po, _, aconv, _ = O.adjoint(gd, To, xi, eta, w.src[b], w.rec, Ro, tol=1e-8, max_iter=200)
    assert aconv
    assert rel_l2(P_b, Po) <= 1e-3


def test_anisotropic_batch_with_the_godunov_solver_in_the_benchmark_configuration(tt):
    """The benchmark's godunov leg at full size: 121 x 161 x 161, 256 sources, anisotropic
    Godunov forward (R16) with the autotuned launch inside a captured graph. A cold oracle
    solve takes minutes here, so the check is one that holds at any size: the slowest and
    the fastest source, each solved alone with the default launch, give their batch
    columns' bits (traveltime, adjoint field and iteration counts). Their agreement with the
    oracle is tested at 81^3 (tests/test_gpu_godunov.py)."""
    import torch
    w = I.anisotropic_batch()
    g = w.grid
    model = tuple(to_dev(a, torch.float32) for a in (w.s, w.xi, w.eta))
    ctx = tt.tt_ctx_create(g.as_dict())
    o = tt.default_opts(tt.TT_F32, scheme=2)
    tt.tt_autotune(ctx, model, w.src, o)
    shape = g.shape + (w.n_src,)
    tau, T, P = (torch.empty(shape, device="cuda") for _ in range(3))
    data = tt.DeviceData.from_workload(w)
    chi = torch.empty((w.n_src, 2), dtype=torch.float64, device="cuda")
    R = torch.empty((w.n_src, data.n_rec), dtype=torch.float64, device="cuda")
    K = [torch.zeros(g.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    plan = tt.tt_plan_create(ctx, model, w.src, data, tau, T, P, chi, R, *K, opts=o)
    itf, ita = tt.tt_plan_run(plan)
    plan.close()
    assert int(np.max(itf)) <= 15
    for b in (int(np.argmax(itf)), int(np.argmin(itf))):
        one = gpu_solve(w.subset([b]), "f32", opts=tt.default_opts(tt.TT_F32, scheme=2),
                        ctx=ctx)
        assert np.array_equal(one["T"][..., 0], T[..., b].cpu().numpy())
        assert np.array_equal(one["P"][..., 0], P[..., b].cpu().numpy())
        assert int(one["iters_fwd"][0]) == int(itf[b])
    ctx.close()
