"""Pins of the FP64 warm-start network reference (oracle/net.py) against things other than
itself: torch's conv3d, finite differences of the loss, closed-form geometry."""
import numpy as np
import pytest

import tt_inputs as I
from oracle import net as N


def _theta(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in N.LAYERS:
        bound = scale * np.sqrt(6.0 / (27 * ci))
        parts += [rng.uniform(-bound, bound, 27 * ci * co), rng.uniform(-0.1, 0.1, co)]
    return np.concatenate(parts)


def test_parameter_count_is_the_four_layer_net():
    assert N.n_params() == 27 * (6 * 32 + 32 * 32 + 32 * 32 + 32) + 32 * 3 + 1


def test_conv3d_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = rng.standard_normal((5, 6, 7, 4))
    W = rng.standard_normal((27, 4, 3))
    b = rng.standard_normal(3)
    y = N.conv3d(x, W, b)
    wt = torch.tensor(W.reshape(3, 3, 3, 4, 3)).permute(4, 3, 0, 1, 2)   # [co][ci][dz][dy][dx]
    xt = torch.tensor(x).permute(3, 0, 1, 2)[None]
    ref = torch.nn.functional.conv3d(xt, wt, torch.tensor(b), padding=1)[0].permute(1, 2, 3, 0)
    assert np.abs(y - ref.numpy()).max() < 1e-12


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    theta = _theta(5)
    xs = [rng.standard_normal((4, 5, 6, 6)) * 0.5 for _ in range(2)]
    ts = [rng.standard_normal((4, 5, 6)) * 0.1 for _ in range(2)]
    ms = [(rng.uniform(size=(4, 5, 6)) > 0.2).astype(float) for _ in range(2)]
    loss, g = N.loss_and_grad(theta, xs, ts, ms)
    idx = np.concatenate([rng.choice(N.n_params(), 40, replace=False),
                          np.arange(N.n_params() - 40, N.n_params())])   # incl. every bias of layers 3-4
    h = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (N.loss_and_grad(tp, xs, ts, ms)[0] - N.loss_and_grad(tm, xs, ts, ms)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), k


def test_features_homogeneous_spherical_offsets_are_chords():
    w = I.homogeneous_41()
    x = N.features(w.grid.as_dict(), w.s, w.xi, w.eta, w.src[0])
    assert np.abs(x[..., 0]).max() < 1e-12          # s / s0 - 1 = 0
    assert np.abs(x[..., 1:3]).max() == 0.0
    g = w.grid
    d, la, lo = np.meshgrid(*g.axes(), indexing="ij")
    # law of cosines on the sphere (independent of the frame construction)
    re = g.earth_radius_km
    r, rs = re - d, re - w.src[0][0]
    th, ph = np.deg2rad(la), np.deg2rad(lo)
    ths, phs = np.deg2rad(w.src[0][1]), np.deg2rad(w.src[0][2])
    cosg = np.sin(th) * np.sin(ths) + np.cos(th) * np.cos(ths) * np.cos(ph - phs)
    chord = np.sqrt(np.maximum(r * r + rs * rs - 2 * r * rs * cosg, 0.0))
    dist = np.linalg.norm(x[..., 3:6], axis=-1) * N.FEATURE_SCALE_KM
    assert np.abs(dist - chord).max() < 1e-9 * chord.max()
    # the up component at the source's own column is the depth difference
    i = np.argmin(np.abs(d[:, 0, 0] - 20.0))
    col = x[:, 20, 20, 3] * N.FEATURE_SCALE_KM
    assert np.abs(col[i] - (w.src[0][0] - d[i, 0, 0])) < 1e-9


def test_features_flat_geometry_offsets_are_coordinate_differences():
    w = I.small_case(41, shape=(7, 8, 9), n_src=1, n_rec=3, flat=1)
    g = w.grid.as_dict()
    x = N.features(g, w.s, w.xi, w.eta, w.src[0])
    depth, lat, lon = w.grid.axes()
    re = w.grid.earth_radius_km
    up = (w.src[0][0] - depth)[:, None, None] / N.FEATURE_SCALE_KM
    north = re * np.deg2rad(lat - w.src[0][1])[None, :, None] / N.FEATURE_SCALE_KM
    east = re * np.deg2rad(lon - w.src[0][2])[None, None, :] / N.FEATURE_SCALE_KM
    assert np.abs(x[..., 3] - up).max() < 1e-12
    assert np.abs(x[..., 4] - north).max() < 1e-12
    assert np.abs(x[..., 5] - east).max() < 1e-12


def test_biases_only_network_is_constant():
    theta = np.zeros(N.n_params())
    theta[-1] = 0.25
    x = np.random.default_rng(6).standard_normal((3, 4, 5, 6))
    assert np.all(N.forward(theta, x) == 0.25)
    assert np.all(N.warm_start(theta, x) == 1.25)


# ---- the network on the stride-2 grid: node selection and the interpolation back


@pytest.mark.parametrize("n", [9, 10, 13, 2, 3])
def test_coarse_nodes_take_every_other_node_and_the_last(n):
    idx = N.coarse_nodes(n, 2)
    assert idx[0] == 0 and idx[-1] == n - 1
    assert np.all(np.diff(idx) >= 1) and np.all(np.diff(idx)[:-1] == 2)
    assert len(idx) == -(-(n - 1) // 2) + 1
    assert np.array_equal(N.coarse_nodes(n, 1), np.arange(n))


@pytest.mark.parametrize("shape", [(9, 10, 13), (8, 11, 6)])
def test_upsample_is_exact_for_trilinear_fields_and_keeps_the_network_nodes(shape):
    """A field a + b i + c j + d k + e i j k (trilinear in the node indices) sampled at the
    network nodes comes back exactly at every node, whether the last interval of an axis is
    whole or half; the network nodes keep their values; stride 1 is the identity."""
    rng = np.random.default_rng(5)
    co = rng.standard_normal(5)
    f = lambda i, j, k: co[0] + co[1] * i + co[2] * j + co[3] * k + co[4] * i * j * k
    I, J, K = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
    full = f(I, J, K)
    idx = [N.coarse_nodes(n, 2) for n in shape]
    yc = full[np.ix_(*idx)]
    up = N.upsample(yc, shape, 2)
    assert np.max(np.abs(up - full)) <= 1e-12 * np.max(np.abs(full))
    assert np.array_equal(up[np.ix_(*idx)], yc) or np.max(np.abs(up[np.ix_(*idx)] - yc)) <= 1e-13
    noise = rng.standard_normal(shape)
    assert np.array_equal(N.upsample(noise, shape, 1), noise)


def test_upsample_of_a_non_trilinear_field_stays_between_its_neighbours():
    """Every interpolated value lies within the range of the network values around it (the
    weights are non-negative and sum to one): a bump does not overshoot."""
    shape = (9, 11, 13)
    rng = np.random.default_rng(6)
    idx = [N.coarse_nodes(n, 2) for n in shape]
    yc = rng.uniform(-1, 1, [len(i) for i in idx])
    up = N.upsample(yc, shape, 2)
    assert up.min() >= yc.min() - 1e-15 and up.max() <= yc.max() + 1e-15
