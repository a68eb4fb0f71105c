"""FP64 reference of the warm-start network: its input features, forward pass, loss and
gradient (test infrastructure only; the product package never imports it).

The network predicts the factored correction tau of Sec. 3.1 (T = T0 tau) from local
quantities. Its input is six channels per node: s / s0 - 1 (slowness relative to the
slowness at the source), xi, eta (Eq. "4"), and the offset D to the source in the source's
local (up, north, east) frame, in units of 100 km (the offset that defines T0). Four 3x3x3
convolutions (6 -> 32 -> 32 -> 32 -> 1, zero padding outside the grid, ReLU between them)
give y, and the warm start is tau = 1 + clamp(y, -0.5, 1). Training minimises the masked
mean squared error between y and tau - 1.

Arrays are channels-last: a field on an (n_r, n_t, n_p) grid with C channels has shape
(n_r, n_t, n_p, C). Layer l has weights W[27][C_in][C_out] (tap index (dz * 3 + dy) * 3 + dx,
the tap reading the node at offset (dz - 1, dy - 1, dx - 1)) and bias b[C_out]. The flat
parameter vector concatenates W then b for layers 1 to 4.

Each step is the plain definition: a convolution is a sum over the 27 taps of
matrix products (numpy), and the gradient is the chain rule written out layer by layer.
"""
import numpy as np

LAYERS = ((6, 32), (32, 32), (32, 32), (32, 1))
FEATURE_SCALE_KM = 100.0
CLAMP_LO, CLAMP_HI = -0.5, 1.0


def n_params():
    return sum(27 * ci * co + co for ci, co in LAYERS)


def unpack(theta):
    """Flat parameter vector -> [(W, b), ...] (views, float64)."""
    theta = np.asarray(theta, dtype=np.float64)
    out, k = [], 0
    for ci, co in LAYERS:
        W = theta[k:k + 27 * ci * co].reshape(27, ci, co)
        k += 27 * ci * co
        b = theta[k:k + co]
        k += co
        out.append((W, b))
    assert k == theta.size
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


# ------------------------------------------------------------------------------ features

def _axes_rad(g):
    get = (lambda k: g[k]) if isinstance(g, dict) else (lambda k: getattr(g, k))
    nr, nt, np_ = get("n_r"), get("n_t"), get("n_p")
    re = get("earth_radius_km")
    r = re - get("depth_max_km") + np.arange(nr) * (get("depth_max_km") - get("depth_min_km")) / (nr - 1)
    th = np.deg2rad(get("lat_min_deg") + np.arange(nt) * (get("lat_max_deg") - get("lat_min_deg")) / (nt - 1))
    ph = np.deg2rad(get("lon_min_deg") + np.arange(np_) * (get("lon_max_deg") - get("lon_min_deg")) / (np_ - 1))
    return r, th, ph, re, int(get("flat"))


def _trilinear(field, fr, ft, fp):
    """Trilinear interpolation of a nodal field at fractional index (fr, ft, fp)."""
    n = field.shape
    i0 = min(max(int(np.floor(fr)), 0), n[0] - 2)
    j0 = min(max(int(np.floor(ft)), 0), n[1] - 2)
    k0 = min(max(int(np.floor(fp)), 0), n[2] - 2)
    a, b, c = fr - i0, ft - j0, fp - k0
    v = 0.0
    for di, wi in ((0, 1 - a), (1, a)):
        for dj, wj in ((0, 1 - b), (1, b)):
            for dk, wk in ((0, 1 - c), (1, c)):
                v += wi * wj * wk * field[i0 + di, j0 + dj, k0 + dk]
    return v


def features(g, s, xi, eta, src):
    """Six input channels for one source at (depth_km, lat_deg, lon_deg): (n_r, n_t, n_p, 6)."""
    r, th, ph, re, flat = _axes_rad(g)
    depth, lat, lon = (float(v) for v in src)
    rs = re - depth
    ths, phs = np.deg2rad(lat), np.deg2rad(lon)
    fr = (rs - r[0]) / (r[1] - r[0])
    ft = (ths - th[0]) / (th[1] - th[0])
    fp = (phs - ph[0]) / (ph[1] - ph[0])
    s0 = _trilinear(np.asarray(s, dtype=np.float64), fr, ft, fp)
    R, TH, PH = np.meshgrid(r, th, ph, indexing="ij")
    if flat:
        du, dn, de = R - rs, re * (TH - ths), re * (PH - phs)
    else:
        X = np.stack([R * np.cos(TH) * np.cos(PH), R * np.cos(TH) * np.sin(PH), R * np.sin(TH)], -1)
        Xs = rs * np.array([np.cos(ths) * np.cos(phs), np.cos(ths) * np.sin(phs), np.sin(ths)])
        e_up = np.array([np.cos(ths) * np.cos(phs), np.cos(ths) * np.sin(phs), np.sin(ths)])
        e_n = np.array([-np.sin(ths) * np.cos(phs), -np.sin(ths) * np.sin(phs), np.cos(ths)])
        e_e = np.array([-np.sin(phs), np.cos(phs), 0.0])
        d = X - Xs
        du, dn, de = d @ e_up, d @ e_n, d @ e_e
    x = np.empty(R.shape + (6,))
    x[..., 0] = np.asarray(s, dtype=np.float64) / s0 - 1.0
    x[..., 1] = xi
    x[..., 2] = eta
    x[..., 3] = du / FEATURE_SCALE_KM
    x[..., 4] = dn / FEATURE_SCALE_KM
    x[..., 5] = de / FEATURE_SCALE_KM
    return x


# ------------------------------------------------------------------------------ network

def conv3d(x, W, b):
    """y[p] = b + sum over taps t of x[p + offset(t)] @ W[t], zero outside the grid."""
    D, H, Wd, _ = x.shape
    xp = np.zeros((D + 2, H + 2, Wd + 2, x.shape[3]))
    xp[1:-1, 1:-1, 1:-1] = x
    y = np.broadcast_to(b, (D, H, Wd, W.shape[2])).copy()
    for t in range(27):
        dz, dy, dx = t // 9, (t // 3) % 3, t % 3
        y += xp[dz:dz + D, dy:dy + H, dx:dx + Wd] @ W[t]
    return y


def conv3d_backward(x, W, dy):
    """Gradients of sum(dy * conv3d(x, W, b)) with respect to x, W and b."""
    D, H, Wd, _ = x.shape
    xp = np.zeros((D + 2, H + 2, Wd + 2, x.shape[3]))
    xp[1:-1, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dW = np.empty_like(W)
    dy2 = dy.reshape(-1, dy.shape[3])
    for t in range(27):
        dz, dyy, dx = t // 9, (t // 3) % 3, t % 3
        win = xp[dz:dz + D, dyy:dyy + H, dx:dx + Wd]
        dW[t] = win.reshape(-1, win.shape[3]).T @ dy2
        dxp[dz:dz + D, dyy:dyy + H, dx:dx + Wd] += dy @ W[t].T
    return dxp[1:-1, 1:-1, 1:-1], dW, dy2.sum(axis=0)


def forward(theta, x, keep=False):
    """Network output y (n_r, n_t, n_p); with keep=True also the pre-activations."""
    layers = unpack(theta)
    h, pre = x, []
    for l, (W, b) in enumerate(layers):
        a = conv3d(h, W, b)
        pre.append(a)
        h = np.maximum(a, 0.0) if l + 1 < len(layers) else a
    y = h[..., 0]
    return (y, pre) if keep else y


def warm_start(theta, x):
    """tau = 1 + clamp(y, -0.5, 1)."""
    return 1.0 + np.clip(forward(theta, x), CLAMP_LO, CLAMP_HI)


# --------------------------------------------------------------- the network on a coarser grid

def coarse_nodes(n, c):
    """Node indices, along one axis of n nodes, of the network grid of stride c: every c-th
    node, the last node of the axis always included (index min(a c, n - 1))."""
    na = n if c == 1 else (n + c - 2) // c + 1
    return np.minimum(np.arange(na) * c, n - 1)


def _axis_weights(n, c):
    """For every node i of an axis: the lower network node a and the weight f of the upper
    one. Node i lies between the network nodes' positions p0 = a c and p1 = min(p0 + c, n - 1),
    a = min(i // c, na - 2), f = (i - p0) / (p1 - p0)."""
    na = len(coarse_nodes(n, c))
    i = np.arange(n)
    a = np.minimum(i // c, na - 2)
    p0 = a * c
    p1 = np.minimum(p0 + c, n - 1)
    return a, (i - p0) / (p1 - p0)


def upsample(yc, shape, c):
    """Trilinear interpolation of a field on the stride-c network grid to every node of a grid
    of `shape`: the sum over the eight surrounding network nodes of the products of the
    per-axis weights (1 - f or f) times their values."""
    (ar, fr), (at, ft), (ap, fp) = (_axis_weights(n, c) for n in shape)
    out = np.zeros(shape)
    for di in (0, 1):
        for dj in (0, 1):
            for dk in (0, 1):
                w = ((fr if di else 1 - fr)[:, None, None] * (ft if dj else 1 - ft)[None, :, None]
                     * (fp if dk else 1 - fp)[None, None, :])
                out += w * yc[np.ix_(ar + di, at + dj, ap + dk)]
    return out


def warm_start_coarse(theta, xc, shape, c):
    """The warm start with the network on the stride-c grid (xc: the features at its nodes):
    clamp(y) at the network nodes, interpolated to every node, plus 1."""
    return 1.0 + upsample(np.clip(forward(theta, xc), CLAMP_LO, CLAMP_HI), shape, c)


def loss_and_grad(theta, xs, targets, masks):
    """Masked mean squared error over a batch and its gradient.

    xs: list of feature arrays (n_r, n_t, n_p, 6); targets: tau - 1 on the same grids;
    masks: 0/1 weights. loss = sum_b sum_p m (y - t)^2 / sum_b sum_p m.
    """
    layers = unpack(theta)
    total = sum(float(np.sum(m)) for m in masks)
    grads = [(np.zeros_like(W), np.zeros_like(b)) for W, b in layers]
    loss = 0.0
    for x, t, m in zip(xs, targets, masks):
        y, pre = forward(theta, x, keep=True)
        r = y - t
        loss += float(np.sum(m * r * r)) / total
        d = (2.0 * m * r / total)[..., None]
        for l in range(len(layers) - 1, -1, -1):
            W, _ = layers[l]
            h_in = x if l == 0 else np.maximum(pre[l - 1], 0.0)
            dh, dW, db = conv3d_backward(h_in, W, d)
            grads[l][0][...] += dW
            grads[l][1][...] += db
            if l > 0:
                d = dh * (pre[l - 1] > 0.0)
    return loss, pack(grads)
