"""Parity at the full sizes of the benchmark configurations, on sampled sources (needs a GB300;
the FP64 oracle runs one source at a time on the host).

- 81^3 isotropic checkerboard, 64 sources: the FP32 batch against complete oracle solves
  of sampled sources (traveltime, adjoint state, and that source's kernels).
- 121 x 161 x 161 anisotropic batch, 256 sources, in the benchmark's launch configuration
  (autotuned launch, one captured graph per step), against cold FP64 oracle solves of 8
  seeded sources: traveltime, adjoint state, receiver times, misfits and adjoint sources
  per source, and the kernels summed over the 8. The oracle solves take a few minutes of
  host time; they run in threads while the GPU works.
- the same batch with the anisotropic Godunov forward (the benchmark's godunov leg), in its
  launch configuration: 2 seeded sources against cold oracle solves with the same update,
  and sampled sources solved alone give their batch columns' bits.
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


# Seeded sources of the 256 that the FP64 oracle solves cold at full size, and the ones it
# solves with the anisotropic Godunov update (R16).
C3_LF_SOURCES = sorted(np.random.default_rng(20241203).choice(256, 8, replace=False).tolist())
C3_GOD_SOURCES = sorted(np.random.default_rng(20241204).choice(256, 2, replace=False).tolist())


def _oracle_cold(w, b, scheme):
    """One cold FP64 oracle solve (tau = 1) of source b of the batch in the FP32-rounded
    model: forward, receiver times, misfit, adjoint."""
    import oracle as O
    s, xi, eta = rounded_model(w, "f32")
    gd = w.grid.as_dict()
    _, T, it, conv, _ = O.forward(gd, s, xi, eta, w.src[b], tol=1e-8, max_iter=400,
                                  scheme=scheme)
    d = w.source_data(b)
    Tr = O.receiver_times(gd, T, w.rec)
    ct, cc, R = O.misfit(Tr, d["abs_rec"], d["abs_tobs"], d["abs_w"], d["cs_m"], d["cs_i"],
                         d["cs_dtobs"], d["cs_w"])
    P, ita, aconv, _ = O.adjoint(gd, T, xi, eta, w.src[b], w.rec, R, tol=1e-8, max_iter=200)
    return dict(T=T, Tr=Tr, chi=np.array([ct, cc]), R=R, P=P, it=it, conv=conv and aconv)


@pytest.fixture(scope="module")
def c3_oracle():
    """The cold oracle solves of C3_LF_SOURCES (Lax-Friedrichs) and C3_GOD_SOURCES (R16),
    started in threads when the module's first test needs them, so they run on the host
    cores while the GPU works (the oracle's C calls release the GIL)."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    w = I.anisotropic_batch()
    ex = ThreadPoolExecutor(max(1, min(os.cpu_count() or 1,
                                       len(C3_LF_SOURCES) + len(C3_GOD_SOURCES))))
    jobs = {("lf", b): ex.submit(_oracle_cold, w, b, "lf") for b in C3_LF_SOURCES}
    jobs.update({("god", b): ex.submit(_oracle_cold, w, b, "godunov_aniso")
                 for b in C3_GOD_SOURCES})
    yield w, jobs
    ex.shutdown(wait=True)


def _run_plan(tt, w, o):
    """The benchmark step: autotuned launch, whole step in one captured graph."""
    import torch
    g = w.grid
    model = tuple(to_dev(a, torch.float32) for a in (w.s, w.xi, w.eta))
    ctx = tt.tt_ctx_create(g.as_dict())
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
    return ctx, model, T, P, chi, R, itf


def _misfit_tolerances(w, b, Tr_o, delta):
    """Bounds on |chi_gpu - chi_oracle| and |R_gpu - R_oracle| implied by receiver times
    that differ by at most delta (the traveltime bar times max T): chi is quadratic in the
    receiver times, R linear with coefficients the weights that touch each receiver."""
    d = w.source_data(b)
    n = len(w.rec)
    c = np.zeros(n)
    np.add.at(c, d["abs_rec"], np.abs(d["abs_w"]))
    np.add.at(c, d["cs_m"], 2 * np.abs(d["cs_w"]))
    np.add.at(c, d["cs_i"], 2 * np.abs(d["cs_w"]))
    r_abs = np.abs(Tr_o[d["abs_rec"]] - d["abs_tobs"])
    r_cs = np.abs(Tr_o[d["cs_m"]] - Tr_o[d["cs_i"]] - d["cs_dtobs"])
    dchi_t = np.sum(np.abs(d["abs_w"]) * (r_abs * delta + 0.5 * delta ** 2))
    dchi_cs = np.sum(np.abs(d["cs_w"]) * (r_cs * 2 * delta + 2 * delta ** 2))
    return np.array([dchi_t, dchi_cs]), c * delta


def test_anisotropic_batch_cold_oracle_parity_in_the_benchmark_configuration(tt, c3_oracle):
    """The benchmark step at full size (121 x 161 x 161, 256 sources, FP32, autotuned launch,
    one captured graph) against cold FP64 oracle solves of 8 seeded sources, per source:
    - T: relative L-inf <= 1e-5;
    - P: relative L2 <= 1e-3;
    - receiver times within the T bar, and chi_t, chi_cs and R element by element within the
      bounds those receiver-time differences imply (_misfit_tolerances); the oracle's misfit
      of the GPU's own receiver times gives the GPU's chi and R to 1e-12;
    - the kernels of the 8 sources (Eqs. 6-8, the library's tt_kernel on those columns)
      against the oracle's sum: relative L2 <= 1e-3 each."""
    import torch
    import oracle as O
    w, jobs = c3_oracle
    ctx, model, T, P, chi, R, itf = _run_plan(tt, w, tt.default_opts(tt.TT_F32))
    idx = torch.tensor(C3_LF_SOURCES, device="cuda")
    T8 = T.index_select(-1, idx).contiguous()
    P8 = P.index_select(-1, idx).contiguous()
    chi8, R8 = chi[idx].cpu().numpy(), R[idx].cpu().numpy()
    K8 = [torch.zeros(w.grid.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    tt.tt_kernel(ctx, model, T8, P8, *K8)
    sub = w.subset(C3_LF_SOURCES)
    data8 = tt.DeviceData.from_workload(sub)
    Tr8 = torch.empty((8, data8.n_rec), dtype=torch.float64, device="cuda")
    chi8b = torch.empty((8, 2), dtype=torch.float64, device="cuda")
    R8b = torch.empty_like(Tr8)
    tt.tt_misfit(ctx, T8, data8, Tr8, chi8b, R8b)
    torch.cuda.synchronize()
    T8, P8 = T8.cpu().numpy(), P8.cpu().numpy()
    K8 = [k.cpu().numpy() for k in K8]
    Tr8 = Tr8.cpu().numpy()
    # the misfit of the 8-source batch is the plan's own misfit of those sources
    assert np.array_equal(chi8b.cpu().numpy(), chi8) and np.array_equal(R8b.cpu().numpy(), R8)
    ctx.close()

    s, xi, eta = rounded_model(w, "f32")
    gd = w.grid.as_dict()
    Ko = [np.zeros(w.grid.shape) for _ in range(3)]
    for q, b in enumerate(C3_LF_SOURCES):
        r = jobs[("lf", b)].result()
        print("\nsource %d: GPU %d iterations, oracle %d (cold)" % (b, itf[b], r["it"]))
        assert r["conv"]
        assert rel_linf(T8[..., q], r["T"]) <= 1e-5
        assert rel_l2(P8[..., q], r["P"]) <= 1e-3
        delta = 1e-5 * np.abs(r["T"]).max()
        assert np.abs(Tr8[q] - r["Tr"]).max() <= delta
        tol_chi, tol_R = _misfit_tolerances(w, b, r["Tr"], delta)
        assert np.all(np.abs(chi8[q] - r["chi"]) <= tol_chi)
        assert np.all(np.abs(R8[q] - r["R"]) <= tol_R + 1e-15)
        d = w.source_data(b)
        ct, cc, Rg = O.misfit(Tr8[q], d["abs_rec"], d["abs_tobs"], d["abs_w"], d["cs_m"],
                              d["cs_i"], d["cs_dtobs"], d["cs_w"])
        assert np.allclose(chi8[q], [ct, cc], rtol=1e-12, atol=0)
        assert np.allclose(R8[q], Rg, rtol=1e-12, atol=1e-15)
        O.kernel_add(gd, s, r["T"], r["P"], *Ko)
    for a, k in zip(K8, Ko):
        assert rel_l2(a, k) <= 1e-3


@pytest.mark.parametrize("init", [0, 3])
def test_anisotropic_batch_with_the_godunov_solver_in_the_benchmark_configuration(tt, c3_oracle,
                                                                                  init):
    """The benchmark's godunov leg at full size: 121 x 161 x 161, 256 sources, anisotropic
    Godunov forward (R16) with the autotuned launch inside a captured graph, started from
    tau = 1 (init 0) and from above (init 3, the leg's start).
    - 2 seeded sources against cold FP64 oracle solves with the same update: T relative
      L-inf <= 1e-5, P relative L2 <= 1e-3, chi within the bound the T bar implies;
    - the slowest and the fastest source, each solved alone with the default launch, give
      their batch columns' bits (traveltime, adjoint field and iteration counts)."""
    w, jobs = c3_oracle
    g = w.grid
    o = tt.default_opts(tt.TT_F32, scheme=2, init=init)
    ctx, model, T, P, chi, R, itf = _run_plan(tt, w, o)
    assert int(np.max(itf)) <= (15 if init == 0 else 8)
    for b in C3_GOD_SOURCES:
        r = jobs[("god", b)].result()
        print("\nsource %d (Godunov): GPU %d iterations, oracle %d (cold)" % (b, itf[b], r["it"]))
        assert r["conv"]
        assert rel_linf(T[..., b].cpu().numpy(), r["T"]) <= 1e-5
        assert rel_l2(P[..., b].cpu().numpy(), r["P"]) <= 1e-3
        tol_chi, _ = _misfit_tolerances(w, b, r["Tr"], 1e-5 * np.abs(r["T"]).max())
        assert np.all(np.abs(chi[b].cpu().numpy() - r["chi"]) <= tol_chi)
    for b in (int(np.argmax(itf)), int(np.argmin(itf))):
        one = gpu_solve(w.subset([b]), "f32", opts=tt.default_opts(tt.TT_F32, scheme=2,
                                                                    init=init), ctx=ctx)
        assert np.array_equal(one["T"][..., 0], T[..., b].cpu().numpy())
        assert np.array_equal(one["P"][..., 0], P[..., b].cpu().numpy())
        assert int(one["iters_fwd"][0]) == int(itf[b])
    ctx.close()
