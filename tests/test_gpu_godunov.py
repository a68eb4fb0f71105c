"""The Godunov local solver on the GPU (opts.scheme = 1, isotropic models) against the
oracle's Godunov solver (reading R14), through the C ABI (needs a GB300).

- FP64 batch: traveltime to 1e-10 of the oracle and the same iteration counts;
- FP32 batch: traveltime to the 1e-5 bar of the FP32 path;
- retire-and-refill and barrier-group variants: bitwise the resident launch;
- an anisotropic model is refused;
- a 41^3 checkerboard: a few iterations where Lax-Friedrichs needs a count growing with the
  grid;
- the 81^3 isotropic checkerboard at full size (64 sources) against oracle solves of sampled
  sources;
- the anisotropic solver (opts.scheme = 2, reading R16): FP64 batch to 1e-10 of the oracle
  with the same iteration counts, FP32 batch to the 1e-5 bar with bitwise launch variants,
  and an anisotropic 81^3 checkerboard at full size;
- the start from above (opts.init = 3), with either update: FP64 batch to 1e-10 of the
  oracle started from the same value, with its iteration counts; FP32 batch to the 1e-5 bar
  of the oracle's converged solve, bitwise across launch variants.
"""
import numpy as np
import pytest

import tt_inputs as I
from gpu_helpers import gpu_solve, rel_linf, rounded_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_00031_gb300 as m
    return m


def _isotropic(seed, shape, n_src, amp=0.05):
    w = I.small_case(seed, shape=shape, n_src=n_src, n_rec=4)
    i, j, k = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    w.s = (1 / 6.0) * (1 + amp * np.sin(np.pi * i / 6) * np.sin(np.pi * j / 5) *
                       np.sin(np.pi * k / 7))
    w.xi = np.zeros(shape)
    w.eta = np.zeros(shape)
    return w


def _opts(tt, code, **kw):
    return tt.default_opts(code, scheme=1, **kw)


def test_fp64_batch_matches_the_oracle(tt):
    import oracle as O
    w = _isotropic(101, (13, 14, 15), 5)
    out = gpu_solve(w, "f64", opts=_opts(tt, tt.TT_F64, tol_fwd=1e-12, max_iter_fwd=200),
                    steps=("fwd",))
    g = w.grid.as_dict()
    for b in range(w.n_src):
        _, T, it, conv, _ = O.forward(g, w.s, w.xi, w.eta, w.src[b], tol=1e-12, max_iter=200,
                                      scheme="godunov")
        assert conv
        assert rel_linf(out["T"][..., b], T) <= 1e-10
        assert abs(int(out["iters_fwd"][b]) - it) <= 1


def test_fp32_batch_meets_the_bar(tt):
    import oracle as O
    w = _isotropic(102, (17, 16, 18), 40)
    out = gpu_solve(w, "f32", opts=_opts(tt, tt.TT_F32), steps=("fwd",))
    s, xi, eta = rounded_model(w, "f32")
    g = w.grid.as_dict()
    for b in (0, 17, 39):
        _, T, it, conv, _ = O.forward(g, s, xi, eta, w.src[b], tol=1e-10, max_iter=200,
                                      scheme="godunov")
        assert conv
        assert rel_linf(out["T"][..., b], T) <= 1e-5
    assert int(np.max(out["iters_fwd"])) <= 10


def test_launch_variants_are_bitwise(tt):
    w = _isotropic(103, (15, 13, 17), 96)
    ref = gpu_solve(w, "f32", opts=_opts(tt, tt.TT_F32), steps=("fwd",))
    for kw in ({"fwd_groups": 1}, {"fwd_groups": 3}, {"fwd_slots": 32}):
        out = gpu_solve(w, "f32", opts=_opts(tt, tt.TT_F32, **kw), steps=("fwd",))
        assert np.array_equal(out["tau"], ref["tau"]), kw
        assert np.array_equal(out["iters_fwd"], ref["iters_fwd"]), kw


def test_anisotropic_model_is_refused(tt):
    w = I.small_case(104, shape=(9, 10, 11), n_src=2, n_rec=3)
    assert np.abs(w.xi).max() > 0
    with pytest.raises(tt.TTError, match="isotropic"):
        gpu_solve(w, "f32", opts=_opts(tt, tt.TT_F32), steps=("fwd",))


def test_few_iterations_against_lax_friedrichs(tt):
    w = _isotropic(105, (41, 41, 41), 8)
    god = gpu_solve(w, "f32", opts=_opts(tt, tt.TT_F32), steps=("fwd",))
    lf = gpu_solve(w, "f32", steps=("fwd",))
    print("\nmean iterations: Godunov %.1f, Lax-Friedrichs %.1f" %
          (np.mean(god["iters_fwd"]), np.mean(lf["iters_fwd"])))
    assert np.max(god["iters_fwd"]) <= 8
    assert np.mean(lf["iters_fwd"]) >= 2 * np.mean(god["iters_fwd"])


@pytest.mark.slow
def test_checkerboard_81_batch_against_oracle_solves(tt):
    """The 81^3 isotropic checkerboard, 64 sources, FP32 Godunov batch: complete FP64 oracle
    Godunov solves of the first and last source (traveltime to the 1e-5 bar); the source
    alone gives its batch column's bits; no source needs more than 10 iterations."""
    import oracle as O
    w = I.checkerboard_81()
    out = gpu_solve(w, "f32", opts=_opts(tt, tt.TT_F32), steps=("fwd",))
    s, xi, eta = rounded_model(w, "f32")
    g = w.grid.as_dict()
    for b in (0, w.n_src - 1):
        _, T, it, conv, _ = O.forward(g, s, xi, eta, w.src[b], tol=1e-10, max_iter=200,
                                      scheme="godunov")
        assert conv
        assert rel_linf(out["T"][..., b], T) <= 1e-5
    one = gpu_solve(w.subset([w.n_src - 1]), "f32", opts=_opts(tt, tt.TT_F32), steps=("fwd",))
    assert np.array_equal(one["T"][..., 0], out["T"][..., -1])
    assert int(np.max(out["iters_fwd"])) <= 10


# ---- the anisotropic Godunov solver (opts.scheme = 2, reading R16) ----

def test_anisotropic_fp64_batch_matches_the_oracle(tt):
    import oracle as O
    w = I.small_case(111, shape=(13, 14, 15), n_src=5)
    assert np.abs(w.xi).max() > 0 and np.abs(w.eta).max() > 0
    o = tt.default_opts(tt.TT_F64, scheme=2, tol_fwd=1e-12, max_iter_fwd=200)
    out = gpu_solve(w, "f64", opts=o, steps=("fwd",))
    g = w.grid.as_dict()
    for b in range(w.n_src):
        _, T, it, conv, _ = O.forward(g, w.s, w.xi, w.eta, w.src[b], tol=1e-12, max_iter=200,
                                      scheme="godunov_aniso")
        assert conv
        assert rel_linf(out["T"][..., b], T) <= 1e-10
        assert abs(int(out["iters_fwd"][b]) - it) <= 1


def test_anisotropic_fp32_batch_meets_the_bar_and_variants_are_bitwise(tt):
    import oracle as O
    w = I.small_case(112, shape=(17, 16, 18), n_src=40)
    ref = gpu_solve(w, "f32", opts=tt.default_opts(tt.TT_F32, scheme=2), steps=("fwd",))
    s, xi, eta = rounded_model(w, "f32")
    g = w.grid.as_dict()
    for b in (0, 21, 39):
        _, T, it, conv, _ = O.forward(g, s, xi, eta, w.src[b], tol=1e-10, max_iter=200,
                                      scheme="godunov_aniso")
        assert conv
        assert rel_linf(ref["T"][..., b], T) <= 1e-5
    assert int(np.max(ref["iters_fwd"])) <= 10
    for kw in ({"fwd_groups": 1}, {"fwd_groups": 3}, {"fwd_slots": 32}):
        out = gpu_solve(w, "f32", opts=tt.default_opts(tt.TT_F32, scheme=2, **kw), steps=("fwd",))
        assert np.array_equal(out["tau"], ref["tau"]), kw
        assert np.array_equal(out["iters_fwd"], ref["iters_fwd"]), kw


@pytest.mark.slow
def test_anisotropic_81_batch_against_oracle_solves(tt):
    """81^3 checkerboard with xi and eta checkerboards of amplitude 0.04, 64 sources, FP32:
    complete FP64 oracle solves (R16) of the first and last source to the 1e-5 bar."""
    import oracle as O
    w = I.checkerboard_81()
    w.xi = 0.04 * I.checker(w.grid)
    w.eta = 0.04 * I.checker(w.grid, phase_cos_phi=True)
    out = gpu_solve(w, "f32", opts=tt.default_opts(tt.TT_F32, scheme=2), steps=("fwd",))
    s, xi, eta = rounded_model(w, "f32")
    g = w.grid.as_dict()
    for b in (0, w.n_src - 1):
        _, T, it, conv, _ = O.forward(g, s, xi, eta, w.src[b], tol=1e-10, max_iter=200,
                                      scheme="godunov_aniso")
        assert conv
        assert rel_linf(out["T"][..., b], T) <= 1e-5
    assert int(np.max(out["iters_fwd"])) <= 12


# ---- the start from above (opts.init = 3) ----

def _upper_start(w):
    """The value opts.init = 3 starts from, restated in FP32: twice max s / sqrt(1 - 2 g) over
    min s / sqrt(1 + 2 g), g = sqrt(xi^2 + eta^2) over the model's nodes."""
    s, xi, eta = (np.asarray(a, dtype=np.float32) for a in (w.s, w.xi, w.eta))
    g2 = np.sqrt(xi * xi + eta * eta) * np.float32(2)
    hi = np.max(s / np.sqrt(np.maximum(np.float32(1) - g2, np.float32(1e-6))))
    lo = np.min(s / np.sqrt(np.float32(1) + g2))
    return float(np.float32(2) * hi / lo)


@pytest.mark.parametrize("scheme,name", [(2, "godunov_aniso"), (0, "lf")])
def test_start_from_above_fp64_matches_the_oracle_from_the_same_start(tt, scheme, name):
    import oracle as O
    w = I.small_case(113, shape=(13, 14, 15), n_src=5)
    assert np.abs(w.xi).max() > 0 and np.abs(w.eta).max() > 0
    o = tt.default_opts(tt.TT_F64, scheme=scheme, init=tt.TT_INIT_ABOVE, tol_fwd=1e-12,
                        max_iter_fwd=500)
    out = gpu_solve(w, "f64", opts=o, steps=("fwd",))
    g = w.grid.as_dict()
    start = np.full(w.grid.shape, _upper_start(w))
    assert start.flat[0] > 1.5
    for b in range(w.n_src):
        _, T, it, conv, _ = O.forward(g, w.s, w.xi, w.eta, w.src[b], tol=1e-12, max_iter=500,
                                      tau_init=start, scheme=name)
        assert conv
        assert rel_linf(out["T"][..., b], T) <= 1e-10
        assert abs(int(out["iters_fwd"][b]) - it) <= 1


def test_start_from_above_fp32_meets_the_bar_and_variants_are_bitwise(tt):
    """On this small grid both starts need about 3 iterations; the saving from above shows
    at the benchmark size (the full-size test)."""
    import oracle as O
    w = I.small_case(114, shape=(17, 16, 18), n_src=40)
    one = gpu_solve(w, "f32", opts=tt.default_opts(tt.TT_F32, scheme=2), steps=("fwd",))
    ref = gpu_solve(w, "f32", opts=tt.default_opts(tt.TT_F32, scheme=2, init=tt.TT_INIT_ABOVE),
                    steps=("fwd",))
    s, xi, eta = rounded_model(w, "f32")
    g = w.grid.as_dict()
    for b in (0, 19, 39):
        _, T, _, conv, _ = O.forward(g, s, xi, eta, w.src[b], tol=1e-10, max_iter=200,
                                     scheme="godunov_aniso")
        assert conv
        assert rel_linf(ref["T"][..., b], T) <= 1e-5
    print("\nGodunov iterations: from tau = 1 mean %.2f max %d, from above mean %.2f max %d" %
          (np.mean(one["iters_fwd"]), np.max(one["iters_fwd"]), np.mean(ref["iters_fwd"]),
           np.max(ref["iters_fwd"])))
    assert np.max(ref["iters_fwd"]) <= np.max(one["iters_fwd"]) + 1
    for kw in ({"fwd_groups": 1}, {"fwd_groups": 3}, {"fwd_slots": 32}):
        out = gpu_solve(w, "f32", opts=tt.default_opts(tt.TT_F32, scheme=2,
                                                       init=tt.TT_INIT_ABOVE, **kw),
                        steps=("fwd",))
        assert np.array_equal(out["tau"], ref["tau"]), kw
        assert np.array_equal(out["iters_fwd"], ref["iters_fwd"]), kw
