"""Edge cases of the GPU path against the FP64 oracle, through the C ABI (needs a GB300):
- sources on the corners, edges and faces of the domain and on a node, on the smallest
  grid the library accepts (4 nodes per axis) and on a ragged one, receivers on corners
  and faces: FP64 traveltimes, misfits, adjoint fields and kernels to the oracle's bars;
- batch sizes: none and TT_MAX_BATCH + 1 are refused, TT_MAX_BATCH itself runs and each
  sampled column is the bits of its source solved alone;
- a grid with fewer than 4 nodes on an axis is refused.
"""
import numpy as np
import pytest

import tt_inputs as I
from gpu_helpers import gpu_solve, oracle_solve, rel_l2, rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_00031_gb300 as m
    return m


def _workload(shape, src, rec, seed=0):
    """Heterogeneous anisotropic model on a 12 km deep, 0.12 x 0.132 deg grid with the given
    sources and receivers; absolute times and common-source pairs as in the small cases."""
    g = I.GridSpec(shape[0], shape[1], shape[2], 0.0, 12.0, 0.0, 0.12, 0.0, 0.132)
    rng = np.random.default_rng(seed)
    v = I.background_velocity(g) * (1.0 + 0.04 * I.checker(g, 1.0, 1.0, 1.0))
    xi = 0.03 * I.checker(g, 1.0, 1.0, 1.0)
    eta = 0.03 * I.checker(g, 1.0, 1.0, 1.0, phase_cos_phi=True)
    src, rec = np.asarray(src, dtype=float), np.asarray(rec, dtype=float)
    tobs = I.synthetic_observations(g, src, rec, 6.0, 0.05, rng)
    d = I.build_data(g, src, rec, tobs, rng, cs_max_deg=0.2)
    return I.Workload(g, 1.0 / v, xi, eta, src, rec, name="edges-%dx%dx%d" % shape, **d)


def _boundary_points():
    """The 8 corners of the domain, the middle of an edge and of two faces, and a node."""
    corners = [[z, t, p] for z in (0.0, 12.0) for t in (0.0, 0.12) for p in (0.0, 0.132)]
    return corners + [[0.0, 0.06, 0.0], [6.0, 0.12, 0.05], [12.0, 0.03, 0.07]]


@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 7, 6)])
def test_sources_on_the_boundary_match_the_oracle(tt, shape):
    """Fixed sets clipped at the faces, edges and corners; receivers on the surface corners,
    a surface edge and the bottom corner. FP64: T to 1e-10 of the oracle with the same
    iteration counts (within 1), chi and R to 1e-8, P and the kernels to 1e-8."""
    src = _boundary_points()
    if shape == (5, 7, 6):   # a node: depth 3 km, the second latitude row, the third column
        src.append([3.0, 0.12 / 6, 2 * 0.132 / 5])
    rec = [[0.0, 0.0, 0.0], [0.0, 0.12, 0.132], [0.0, 0.06, 0.132], [0.0, 0.03, 0.05],
           [12.0, 0.12, 0.0]]
    w = _workload(shape, src, rec)
    o = tt.default_opts(tt.TT_F64, tol_fwd=1e-12, tol_adj=1e-12, max_iter_fwd=2000,
                        max_iter_adj=2000)
    out = gpu_solve(w, "f64", opts=o)
    res, K = oracle_solve(w, tol=1e-12)
    for b, r in enumerate(res):
        assert abs(int(out["iters_fwd"][b]) - r["iters_fwd"]) <= 1, b
        assert rel_linf(out["T"][..., b], r["T"]) <= 1e-10, b
        assert rel_linf(out["Tr"][b], r["Tr"]) <= 1e-10, b
        assert out["chi"][b] == pytest.approx([r["chi_t"], r["chi_cs"]], rel=1e-8, abs=1e-12)
        assert np.abs(out["R"][b] - r["R"]).max() <= 1e-8 * max(1.0, np.abs(r["R"]).max())
        if np.abs(r["P"]).max() > 0:
            assert rel_l2(out["P"][..., b], r["P"]) <= 1e-8, b
        else:
            assert np.abs(out["P"][..., b]).max() == 0.0, b
    for a, b in zip(out["K"], K):
        assert rel_l2(a, b) <= 1e-8


def test_batch_size_limits(tt):
    """No source and TT_MAX_BATCH + 1 sources are refused; a batch of TT_MAX_BATCH sources
    runs the whole step, and sampled columns are the bits of their sources solved alone."""
    import torch
    rng = np.random.default_rng(21)
    n = tt.TT_MAX_BATCH
    src = np.stack([rng.uniform(0.5, 11.5, n), rng.uniform(0.0, 0.12, n),
                    rng.uniform(0.0, 0.132, n)], 1)
    rec = [[0.0, 0.03, 0.04], [0.0, 0.09, 0.1], [0.0, 0.06, 0.066]]
    w = _workload((5, 6, 7), src, rec)
    ctx = tt.tt_ctx_create(w.grid.as_dict())
    model = tuple(torch.as_tensor(a, dtype=torch.float32, device="cuda") for a in (w.s, w.xi, w.eta))
    for bad in (np.zeros((0, 3)), np.concatenate([src, src[:1]])):
        tau = torch.empty(w.grid.shape + (max(1, len(bad)),), device="cuda")
        with pytest.raises(tt.TTError) as e:
            tt.tt_forward(ctx, model, bad, tau)
        assert e.value.status == tt.TT_EINVAL
    ctx.close()
    out = gpu_solve(w, "f32")
    assert np.isfinite(out["T"]).all() and np.isfinite(out["P"]).all()
    assert all(np.isfinite(k).all() for k in out["K"])
    for b in (0, 1777, n - 1):
        one = gpu_solve(w.subset([b]), "f32", steps=("fwd",))
        assert np.array_equal(one["tau"][..., 0], out["tau"][..., b]), b
        assert np.array_equal(one["T"][..., 0], out["T"][..., b]), b
        assert int(one["iters_fwd"][0]) == int(out["iters_fwd"][b]), b


@pytest.mark.parametrize("shape", [(3, 6, 6), (6, 3, 6), (6, 6, 3)])
def test_grid_with_fewer_than_four_nodes_on_an_axis_is_refused(tt, shape):
    g = I.GridSpec(shape[0], shape[1], shape[2], 0.0, 12.0, 0.0, 0.12, 0.0, 0.132)
    with pytest.raises(tt.TTError) as e:
        tt.tt_ctx_create(g.as_dict())
    assert e.value.status == tt.TT_EINVAL
