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
