"""The Python binding refuses device arguments that hold fewer elements than a call touches,
before the library is called (the C ABI takes plain pointers and cannot check sizes). Runs
on the CPU: a correctly sized CPU tensor gets past the size check and is then refused for
not being a CUDA tensor, so neither case reaches a kernel."""
import numpy as np
import pytest
import torch


@pytest.fixture(scope="module")
def tt():
    import __graft_entry__
    __graft_entry__._load_builder().build()
    import paper_2412_00031_gb300 as m
    return m


class _Ctx:
    def __init__(self, tt, shape):
        self.handle = None
        self.grid = tt.TTGrid(shape[0], shape[1], shape[2], 0.0, 10.0, 0.0, 1.0, 0.0, 1.0,
                              6371.0, 0)


def _z(*shape):
    return torch.zeros(shape, dtype=torch.float64)


def test_fields_smaller_than_the_batch_are_refused(tt):
    shape = (4, 5, 6)
    ctx = _Ctx(tt, shape)
    model = (_z(*shape), _z(*shape), _z(*shape))
    src = np.zeros((3, 3))
    with pytest.raises(ValueError, match="tau holds 240 elements; the call touches 360"):
        tt.tt_forward(ctx, model, src, _z(*shape, 2), _z(*shape, 3))
    with pytest.raises(ValueError, match="CUDA"):
        tt.tt_forward(ctx, model, src, _z(*shape, 3), _z(*shape, 3))
    with pytest.raises(ValueError, match="s holds"):
        tt.tt_forward(ctx, (_z(3), model[1], model[2]), src, _z(*shape, 3))
    with pytest.raises(ValueError, match="Keta holds"):
        tt.tt_kernel(ctx, model, _z(*shape, 3), _z(*shape, 3), _z(*shape), _z(*shape), _z(5))


def test_tables_smaller_than_the_data_are_refused(tt):
    shape = (4, 5, 6)
    ctx = _Ctx(tt, shape)

    class D:
        n_src, n_rec = 3, 7
    with pytest.raises(ValueError, match="chi holds"):
        tt.tt_misfit_table(ctx, _z(3, 7), None, D(), None, _z(3), _z(3, 7))
    with pytest.raises(ValueError, match="grad holds"):
        tt.tt_field_at_points(ctx, _z(*shape, 7), _z(2, 3), _z(2, 7), _z(2, 7))
    with pytest.raises(ValueError, match="Kx holds"):
        tt.tt_reloc_kernels(ctx, _z(3, 7), _z(3, 7, 3), _z(3), _z(3))
    with pytest.raises(ValueError, match="T holds"):
        tt.tt_tele_region_times(ctx, _z(2, 5, 5), 6000.0, 6371.0, 10.0, np.zeros((2, 3)),
                                _z(*shape, 1))
    with pytest.raises(ValueError, match="CUDA"):
        tt.tt_tele_region_times(ctx, _z(2, 5, 5), 6000.0, 6371.0, 10.0, np.zeros((2, 3)),
                                _z(*shape, 2))


def _f(*shape):
    return torch.zeros(shape, dtype=torch.float32)


def test_arguments_of_the_wrong_element_type_are_refused(tt):
    """Sizes are counted in elements, so a buffer of the wrong float type would pass a size
    check and then be read or written with the other element size: every batched field must
    have the model's type, every double* argument must be float64."""
    shape = (4, 5, 6)
    ctx = _Ctx(tt, shape)
    m64 = (_z(*shape), _z(*shape), _z(*shape))
    m32 = (_f(*shape), _f(*shape), _f(*shape))
    src = np.zeros((3, 3))
    with pytest.raises(TypeError, match="tau is torch.float32"):
        tt.tt_forward(ctx, m64, src, _f(*shape, 3), _z(*shape, 3))
    with pytest.raises(TypeError, match="xi is torch.float32"):
        tt.tt_forward(ctx, (m64[0], m32[1], m64[2]), src, _z(*shape, 3))
    with pytest.raises(TypeError, match="Ks is torch.float32"):
        tt.tt_kernel(ctx, m32, _f(*shape, 3), _f(*shape, 3), _f(*shape), _z(*shape), _z(*shape))
    with pytest.raises(TypeError, match="R is torch.float32"):
        tt.tt_adjoint(ctx, m32, src, _f(*shape, 3), np.zeros((7, 3)), _f(3, 7), _f(*shape, 3))
    with pytest.raises(TypeError, match="P is torch.float64"):
        tt.tt_adjoint(ctx, m32, src, _f(*shape, 3), np.zeros((7, 3)), _z(3, 7), _z(*shape, 3))

    class D:
        n_src, n_rec = 3, 7
    with pytest.raises(TypeError, match="chi is torch.float32"):
        tt.tt_misfit(ctx, _f(*shape, 3), D(), None, _f(3, 2), _z(3, 7))
    with pytest.raises(TypeError, match="Kd is torch.float32"):
        tt.tt_kernel_normalize(ctx, _z(*shape), _z(*shape), _z(*shape), _f(*shape), 1.0, 1.0)
    with pytest.raises(TypeError, match="fields must be float32 or float64"):
        tt.tt_forward(ctx, tuple(a.half() for a in m32), src, _f(*shape, 3).half())


def test_no_alloc_misfit_and_network_buffers_are_size_checked(tt):
    shape = (4, 5, 6)
    grid = dict(n_r=4, n_t=5, n_p=6, depth_min_km=0.0, depth_max_km=10.0, lat_min_deg=0.0,
                lat_max_deg=1.0, lon_min_deg=0.0, lon_max_deg=1.0, earth_radius_km=6371.0,
                flat=0)

    class D:
        n_src, n_rec = 3, 7
    with pytest.raises(ValueError, match="T holds 240 elements; the call touches 360"):
        tt.tt_misfit_noalloc(grid, _f(*shape, 2), D(), None, _z(3, 2), _z(3, 7))
    with pytest.raises(ValueError, match="R holds"):
        tt.tt_misfit_noalloc(grid, _f(*shape, 3), D(), None, _z(3, 2), _z(3, 6))
    with pytest.raises(TypeError, match="Tr is torch.float32"):
        tt.tt_misfit_noalloc(grid, _f(*shape, 3), D(), _f(3, 7), _z(3, 2), _z(3, 7))
    ctx = _Ctx(tt, shape)
    n_par = tt.tt_net_param_count()
    N = 4 * 5 * 6
    with pytest.raises(ValueError, match="theta holds"):
        tt.tt_net_set_weights(ctx, _f(n_par - 1))
    with pytest.raises(ValueError, match="x holds"):
        tt.tt_net_forward(ctx, _f(n_par), _f(2, N * 6 - 1), _f(2, N))
    with pytest.raises(ValueError, match="y holds"):
        tt.tt_net_infer(ctx, _f(2, N, 6), _f(2, N - 1))
    with pytest.raises(ValueError, match="mask holds"):
        tt.tt_net_loss_grad(ctx, _f(n_par), _f(2, N, 6), _f(2, N), _f(N), _f(n_par))
    with pytest.raises(ValueError, match="v holds"):
        tt.tt_net_adam(ctx, _f(n_par), _f(n_par), _f(n_par), _f(3), 1)
    with pytest.raises(ValueError, match="x holds"):
        tt.tt_net_features(ctx, (_f(*shape),) * 3, np.zeros((2, 3)), _f(N * 6))
    with pytest.raises(ValueError, match="CUDA"):
        tt.tt_net_set_weights(ctx, _f(n_par))


def test_common_receiver_table_is_packed_by_the_library(tt):
    """tt_cr_pack (host side, no GPU): every unordered pair of Eq. 4 appears under both of its
    sources at its receiver, with dT_obs and -dT_obs, in the order the header states."""
    rng = np.random.default_rng(7)
    ns, nr = 5, 4
    rows = []
    for _ in range(23):
        b, j = rng.choice(ns, 2, replace=False)
        rows.append((b, j, rng.integers(nr), rng.normal(), rng.uniform(0.5, 2.0)))
    rows.append(rows[3][:3] + (0.25, 1.0))            # a repeated pair keeps its own entry
    off, other, dtobs, w = tt.cr_pack(ns, nr, rows)
    assert off.dtype == np.int32 and other.dtype == np.int32 and off[-1] == 2 * len(rows)
    for b in range(ns):
        for m in range(nr):
            want = [(j, dt, ww) for (bb, j, mm, dt, ww) in rows if bb == b and mm == m]
            want += [(bb, -dt, ww) for (bb, j, mm, dt, ww) in rows if j == b and mm == m]
            q0, q1 = off[b * nr + m], off[b * nr + m + 1]
            got = list(zip(other[q0:q1], dtobs[q0:q1], w[q0:q1]))
            assert [(int(g[0]), g[1], g[2]) for g in got] == [(int(a), c, d) for a, c, d in want]
    # refusals: a source out of range, b == j, a receiver out of range, a fractional index
    for bad in [(5, 0, 0, 0.1, 1.0), (2, 2, 0, 0.1, 1.0), (0, 1, 4, 0.1, 1.0),
                (0.5, 1, 0, 0.1, 1.0), (0, -1, 0, 0.1, 1.0)]:
        with pytest.raises(tt.TTError):
            tt.cr_pack(ns, nr, rows[:2] + [bad])
    off, other, dtobs, w = tt.cr_pack(ns, nr, [])
    assert len(other) == 0 and not off.any()
