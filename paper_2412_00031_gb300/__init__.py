"""Python binding of libttgb, the GB300 adjoint-state traveltime tomography library.

Argument marshalling only: every step runs in the CUDA kernels behind the C ABI declared in
include/tt.h. Device arrays are torch CUDA tensors (PyTorch provides device memory and the
stream); host arrays are numpy. The functions carry the C names:

    ctx = tt_ctx_create(grid)                      # grid: dict / object with tt_grid fields
    iters = tt_forward(ctx, model, src, tau, T)    # model = (s, xi, eta) CUDA tensors
    tt_misfit(ctx, T, data, Tr, chi, R)            # data: DeviceData
    iters = tt_adjoint(ctx, model, src, T, rec, R, P)
    tt_kernel(ctx, model, T, P, Ks, Kxi, Keta)

Batched fields (tau, T, P) are tensors of shape (n_r, n_t, n_p, n_src), i.e. node-major with
the source index fastest, as the C ABI stores them. There is no CPU fallback: importing this
module fails if libttgb.so has not been built.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libttgb.so")

TT_OK, TT_EINVAL, TT_ENOTCONVERGED, TT_ECUDA, TT_ETIMEOUT, TT_ENOMEM = range(6)
TT_F32, TT_F64 = 0, 1
TT_INIT_ONE, TT_INIT_GIVEN, TT_INIT_NET, TT_INIT_ABOVE = 0, 1, 2, 3  # tt_opts.init
STATUS_NAMES = {0: "TT_OK", 1: "TT_EINVAL", 2: "TT_ENOTCONVERGED", 3: "TT_ECUDA",
                4: "TT_ETIMEOUT", 5: "TT_ENOMEM"}
TT_MAX_BATCH = 4096


class TTGrid(C.Structure):
    _fields_ = [("n_r", C.c_int), ("n_t", C.c_int), ("n_p", C.c_int),
                ("depth_min_km", C.c_double), ("depth_max_km", C.c_double),
                ("lat_min_deg", C.c_double), ("lat_max_deg", C.c_double),
                ("lon_min_deg", C.c_double), ("lon_max_deg", C.c_double),
                ("earth_radius_km", C.c_double), ("geometry", C.c_int)]


class TTModel(C.Structure):
    _fields_ = [("d_s", C.c_void_p), ("d_xi", C.c_void_p), ("d_eta", C.c_void_p),
                ("dtype", C.c_int)]


class TTMgrid(C.Structure):
    _fields_ = [("n_r", C.c_int), ("n_t", C.c_int), ("n_p", C.c_int), ("n_grids", C.c_int)]


class TTCrData(C.Structure):
    _fields_ = [("n_src", C.c_int), ("n_rec", C.c_int), ("n_entries", C.c_int),
                ("d_off", C.c_void_p), ("d_other", C.c_void_p), ("d_dtobs", C.c_void_p),
                ("d_w", C.c_void_p), ("gamma", C.c_double)]


class TTPoint(C.Structure):
    _fields_ = [("depth_km", C.c_double), ("lat_deg", C.c_double), ("lon_deg", C.c_double)]


class TTData(C.Structure):
    _fields_ = [("n_src", C.c_int), ("n_rec", C.c_int), ("h_rec", C.POINTER(TTPoint)),
                ("d_abs_off", C.c_void_p), ("d_abs_rec", C.c_void_p),
                ("d_abs_tobs", C.c_void_p), ("d_abs_w", C.c_void_p),
                ("d_cs_off", C.c_void_p), ("d_cs_m", C.c_void_p), ("d_cs_i", C.c_void_p),
                ("d_cs_dtobs", C.c_void_p), ("d_cs_w", C.c_void_p),
                ("alpha", C.c_double), ("beta", C.c_double)]


class TTOpts(C.Structure):
    _fields_ = [("tol_fwd", C.c_double), ("tol_adj", C.c_double),
                ("max_iter_fwd", C.c_int), ("max_iter_adj", C.c_int), ("init", C.c_int),
                ("spin_limit_ns", C.c_longlong), ("launch_blocks", C.c_int),
                ("sweep_schedule", C.c_int), ("adj_chunk", C.c_int), ("fwd_groups", C.c_int),
                ("fwd_slots", C.c_int), ("scheme", C.c_int), ("adj_groups", C.c_int),
                ("fwd_order", C.c_int)]


class TTStats(C.Structure):
    _fields_ = [("sweep_ms", C.c_double), ("node_updates", C.c_longlong),
                ("node_sweeps", C.c_longlong), ("iters_max", C.c_int), ("grid_blocks", C.c_int),
                ("block_threads", C.c_int), ("launches", C.c_longlong), ("warm_ms", C.c_double)]


TT_STATS_FORWARD, TT_STATS_ADJOINT, TT_STATS_KERNEL = 0, 1, 2

EXPORTED = ["tt_default_opts", "tt_ctx_create", "tt_ctx_destroy", "tt_last_error",
            "tt_forward", "tt_misfit", "tt_adjoint", "tt_kernel", "tt_get_stats",
            "tt_misfit_noalloc", "tt_plan_create", "tt_plan_run", "tt_plan_destroy",
            "tt_net_param_count", "tt_net_features", "tt_net_forward", "tt_net_loss_grad",
            "tt_net_adam", "tt_net_set_weights", "tt_autotune", "tt_net_infer",
            "tt_kernel_density", "tt_kernel_normalize", "tt_mgrid_project", "tt_mgrid_expand",
            "tt_model_update", "tt_misfit_cr", "tt_field_at_points", "tt_misfit_table",
            "tt_reloc_kernels", "tt_reloc_update", "tt_tele2d", "tt_tele_region_times",
            "tt_forward_tele", "tt_autotune_adjoint", "tt_kernel_normalize_rel",
            "tt_misfit_total", "tt_plan_create_cr", "tt_net_loss_grad_tc", "tt_net_set_stride",
            "tt_net_nodes", "tt_net_start", "tt_cr_pack"]
TT_NOALLOC_MAX_REC = 1024


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libttgb.so is not built; run __graft_entry__.build() first")
    L = C.CDLL(LIB_PATH)
    L.tt_default_opts.argtypes = [C.POINTER(TTOpts), C.c_int]
    L.tt_default_opts.restype = None
    L.tt_ctx_create.argtypes = [C.POINTER(C.c_void_p), C.POINTER(TTGrid), C.c_void_p]
    L.tt_ctx_destroy.argtypes = [C.c_void_p]
    L.tt_ctx_destroy.restype = None
    L.tt_last_error.argtypes = [C.c_void_p]
    L.tt_last_error.restype = C.c_char_p
    L.tt_forward.argtypes = [C.c_void_p, C.POINTER(TTModel), C.POINTER(TTPoint), C.c_int,
                             C.c_void_p, C.c_void_p, C.POINTER(TTOpts), C.POINTER(C.c_int)]
    L.tt_misfit.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(TTData), C.c_void_p,
                            C.c_void_p, C.c_void_p]
    L.tt_adjoint.argtypes = [C.c_void_p, C.POINTER(TTModel), C.POINTER(TTPoint), C.c_int,
                             C.c_void_p, C.c_int, C.POINTER(TTPoint), C.c_void_p, C.c_void_p,
                             C.POINTER(TTOpts), C.POINTER(C.c_int)]
    L.tt_kernel.argtypes = [C.c_void_p, C.POINTER(TTModel), C.c_int, C.c_void_p, C.c_void_p,
                            C.c_void_p, C.c_void_p, C.c_void_p]
    L.tt_get_stats.argtypes = [C.c_void_p, C.c_int, C.POINTER(TTStats)]
    L.tt_misfit_noalloc.argtypes = [C.POINTER(TTGrid), C.c_void_p, C.c_int, C.POINTER(TTData),
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_char_p,
                                    C.c_int]
    L.tt_plan_create.argtypes = [C.POINTER(C.c_void_p), C.c_void_p, C.POINTER(TTModel),
                                 C.POINTER(TTPoint), C.c_int, C.POINTER(TTData),
                                 C.POINTER(TTOpts)] + [C.c_void_p] * 8
    L.tt_plan_create_cr.argtypes = [C.POINTER(C.c_void_p), C.c_void_p, C.POINTER(TTModel),
                                    C.POINTER(TTPoint), C.c_int, C.POINTER(TTData),
                                    C.POINTER(TTCrData), C.POINTER(TTOpts)] + [C.c_void_p] * 10
    L.tt_plan_run.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.tt_plan_destroy.argtypes = [C.c_void_p]
    L.tt_plan_destroy.restype = None
    L.tt_net_param_count.argtypes = []
    L.tt_net_features.argtypes = [C.c_void_p, C.POINTER(TTModel), C.POINTER(TTPoint), C.c_int,
                                  C.c_void_p]
    L.tt_net_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
    L.tt_net_loss_grad.argtypes = [C.c_void_p] + [C.c_void_p] * 4 + [C.c_int, C.c_void_p,
                                                                       C.POINTER(C.c_double)]
    L.tt_net_loss_grad_tc.argtypes = [C.c_void_p] + [C.c_void_p] * 4 + [C.c_int, C.c_void_p,
                                                                          C.POINTER(C.c_double)]
    L.tt_net_adam.argtypes = [C.c_void_p] + [C.c_void_p] * 4 + [C.c_int] + [C.c_float] * 4
    L.tt_net_set_weights.argtypes = [C.c_void_p, C.c_void_p]
    L.tt_net_infer.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
    L.tt_net_set_stride.argtypes = [C.c_void_p, C.c_int]
    L.tt_net_nodes.argtypes = [C.c_void_p]
    L.tt_net_nodes.restype = C.c_int
    L.tt_net_start.argtypes = [C.c_void_p, C.POINTER(TTModel), C.POINTER(TTPoint), C.c_int,
                               C.c_void_p]
    L.tt_autotune.argtypes = [C.c_void_p, C.POINTER(TTModel), C.POINTER(TTPoint), C.c_int,
                              C.POINTER(TTOpts), C.POINTER(C.c_double)]
    L.tt_kernel_normalize_rel.argtypes = [C.c_void_p] * 5 + [C.c_double, C.c_double]
    L.tt_misfit_total.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_double, C.c_double,
                                  C.c_void_p, C.c_double, C.POINTER(C.c_double)]
    L.tt_autotune_adjoint.argtypes = [C.c_void_p, C.POINTER(TTModel), C.POINTER(TTPoint),
                                      C.c_int, C.c_void_p, C.c_int, C.POINTER(TTPoint),
                                      C.c_void_p, C.POINTER(TTOpts), C.POINTER(C.c_double)]
    L.tt_misfit_cr.argtypes = [C.c_void_p, C.POINTER(TTCrData)] + [C.c_void_p] * 3
    L.tt_cr_pack.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int] + [C.c_void_p] * 5
    L.tt_kernel_density.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
    L.tt_kernel_normalize.argtypes = [C.c_void_p] + [C.c_void_p] * 4 + [C.c_double] * 2
    L.tt_mgrid_project.argtypes = [C.c_void_p, C.POINTER(TTMgrid), C.c_void_p, C.c_void_p]
    L.tt_mgrid_expand.argtypes = [C.c_void_p, C.POINTER(TTMgrid), C.c_void_p, C.c_void_p]
    L.tt_model_update.argtypes = [C.c_void_p, C.POINTER(TTModel)] + [C.c_void_p] * 3 + [C.c_double]
    L.tt_field_at_points.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int] + \
        [C.c_void_p] * 3
    L.tt_misfit_table.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(TTData)] + \
        [C.c_void_p] * 3
    L.tt_reloc_kernels.argtypes = [C.c_void_p, C.c_int, C.c_int] + [C.c_void_p] * 4
    L.tt_reloc_update.argtypes = [C.c_void_p, C.c_int] + [C.c_void_p] * 4 + [C.c_double] * 2
    L.tt_tele2d.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                            C.c_double, C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_double,
                            C.c_int, C.c_void_p, C.POINTER(C.c_int)]
    L.tt_forward_tele.argtypes = [C.c_void_p, C.POINTER(TTModel), C.c_int, C.c_void_p,
                                  C.POINTER(TTOpts), C.POINTER(C.c_int)]
    L.tt_tele_region_times.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double,
                                       C.c_double, C.c_double, C.c_void_p, C.c_int,
                                       C.POINTER(TTPoint), C.c_void_p]
    for name in ("tt_ctx_create", "tt_forward", "tt_misfit", "tt_adjoint", "tt_kernel",
                 "tt_get_stats", "tt_misfit_noalloc", "tt_plan_create", "tt_plan_run",
                 "tt_net_param_count", "tt_net_features", "tt_net_forward", "tt_net_loss_grad",
                 "tt_net_adam", "tt_net_set_weights", "tt_autotune", "tt_net_infer",
                 "tt_kernel_density", "tt_kernel_normalize", "tt_mgrid_project",
                 "tt_mgrid_expand", "tt_model_update", "tt_misfit_cr", "tt_field_at_points",
                 "tt_misfit_table", "tt_reloc_kernels", "tt_reloc_update", "tt_tele2d",
                 "tt_tele_region_times", "tt_forward_tele", "tt_autotune_adjoint",
                 "tt_kernel_normalize_rel", "tt_misfit_total", "tt_plan_create_cr",
                 "tt_net_loss_grad_tc", "tt_net_set_stride", "tt_net_start", "tt_cr_pack"):
        getattr(L, name).restype = C.c_int
    return L


lib = _load()


class TTError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


def _check(ctx, status, allow=()):
    if status != TT_OK and status not in allow:
        msg = lib.tt_last_error(ctx.handle if ctx is not None else None)
        raise TTError(status, msg.decode() if msg else "")
    return status


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dtype_code(t):
    import torch
    if t.dtype == torch.float32:
        return TT_F32
    if t.dtype == torch.float64:
        return TT_F64
    raise TypeError("fields must be float32 or float64, got %s" % t.dtype)


def _points(pts):
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    arr = (TTPoint * len(pts))()
    for q, p in enumerate(pts):
        arr[q] = TTPoint(*p)
    return arr, len(pts)


def _nodes(ctx):
    g = ctx.grid
    return int(g.n_r) * int(g.n_t) * int(g.n_p)


def _room(**named):
    """Each value is (tensor or None, elements the call touches[, element type]). Raises
    ValueError when a device argument holds fewer elements than that, and TypeError when its
    element type is not the one the library reads or writes through that pointer, before the
    library is called (the C ABI takes plain pointers and cannot check sizes or types). The
    element type is a torch dtype or None (any); _F64 marks the double* arguments."""
    for name, spec in named.items():
        t, need = spec[0], spec[1]
        want = spec[2] if len(spec) > 2 else None
        if t is None:
            continue
        if want is not None and t.dtype != want:
            raise TypeError("%s is %s; the call reads or writes it as %s" % (name, t.dtype, want))
        if t.numel() < need:
            raise ValueError("%s holds %d elements; the call touches %d" % (name, t.numel(), need))


def _f64():
    import torch
    return torch.float64


def _model_room(ctx, model):
    """The three model arrays: N elements each, all of the slowness's float type (the type
    every batched field of the call must have too). Returns that type."""
    N = _nodes(ctx)
    ft = model[0].dtype
    _dtype_code(model[0])
    _room(s=(model[0], N), xi=(model[1], N, ft), eta=(model[2], N, ft))
    return ft


def _cuda_ok(*tensors):
    for t in tensors:
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError("device arguments must be contiguous CUDA tensors")


def default_opts(dtype=TT_F32, **kw):
    o = TTOpts()
    lib.tt_default_opts(C.byref(o), dtype)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Context:
    """Owns a tt_ctx (one grid, one CUDA stream)."""

    def __init__(self, handle, grid):
        self.handle = handle
        self.grid = grid

    def close(self):
        if self.handle:
            lib.tt_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_grid(g):
    get = (lambda k: g[k]) if isinstance(g, dict) else (lambda k: getattr(g, k))
    return TTGrid(get("n_r"), get("n_t"), get("n_p"), get("depth_min_km"), get("depth_max_km"),
                  get("lat_min_deg"), get("lat_max_deg"), get("lon_min_deg"), get("lon_max_deg"),
                  get("earth_radius_km"), int(get("flat")))


def tt_ctx_create(grid, stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    h = C.c_void_p()
    G = make_grid(grid)
    st = lib.tt_ctx_create(C.byref(h), C.byref(G), C.c_void_p(stream.cuda_stream))
    if st != TT_OK:
        raise TTError(st, "tt_ctx_create rejected the grid or failed to allocate")
    return Context(h, G)


def _model(model):
    s, xi, eta = model
    _cuda_ok(s, xi, eta)
    return TTModel(_ptr(s), _ptr(xi), _ptr(eta), _dtype_code(s))


def tt_forward(ctx, model, src, tau, T=None, opts=None, allow_unconverged=False):
    """Forward solve; tau (in/out) and T have shape (n_r, n_t, n_p, n_src). Returns the
    per-source iteration counts (numpy int32)."""
    pts, n = _points(src)
    ft = _model_room(ctx, model)
    _room(tau=(tau, _nodes(ctx) * n, ft), T=(T, _nodes(ctx) * n, ft))
    M = _model(model)
    _cuda_ok(tau, T)
    if opts is None:
        opts = default_opts(M.dtype)
    iters = (C.c_int * n)()
    st = lib.tt_forward(ctx.handle, C.byref(M), pts, n, _ptr(tau), _ptr(T), C.byref(opts), iters)
    _check(ctx, st, (TT_ENOTCONVERGED,) if allow_unconverged else ())
    return np.frombuffer(iters, dtype=np.int32).copy()


class DeviceData:
    """Observations on the device, in the layout of tt_data."""

    def __init__(self, rec, abs_off, abs_rec, abs_tobs, abs_w, cs_off, cs_m, cs_i, cs_dtobs,
                 cs_w, alpha=1.0, beta=1.0, device="cuda"):
        import torch
        i32 = lambda a: torch.as_tensor(np.asarray(a, dtype=np.int32), device=device)
        f64 = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), device=device)
        self.rec = np.asarray(rec, dtype=np.float64).reshape(-1, 3)
        self.abs_off, self.abs_rec = i32(abs_off), i32(abs_rec)
        self.abs_tobs, self.abs_w = f64(abs_tobs), f64(abs_w)
        self.cs_off, self.cs_m, self.cs_i = i32(cs_off), i32(cs_m), i32(cs_i)
        self.cs_dtobs, self.cs_w = f64(cs_dtobs), f64(cs_w)
        self.alpha, self.beta = float(alpha), float(beta)
        self.h_abs_off = np.asarray(abs_off, dtype=np.int64)    # host copies (record masks)
        self.h_abs_rec = np.asarray(abs_rec, dtype=np.int64)
        self.n_src = len(abs_off) - 1
        self.n_rec = len(self.rec)
        self._pts, _ = _points(self.rec)

    @classmethod
    def from_workload(cls, w, alpha=1.0, beta=1.0, device="cuda"):
        return cls(w.rec, w.abs_off, w.abs_rec, w.abs_tobs, w.abs_w, w.cs_off, w.cs_m, w.cs_i,
                   w.cs_dtobs, w.cs_w, alpha, beta, device)

    def c_struct(self):
        return TTData(self.n_src, self.n_rec, self._pts, _ptr(self.abs_off), _ptr(self.abs_rec),
                      _ptr(self.abs_tobs), _ptr(self.abs_w), _ptr(self.cs_off), _ptr(self.cs_m),
                      _ptr(self.cs_i), _ptr(self.cs_dtobs), _ptr(self.cs_w), self.alpha,
                      self.beta)


def tt_misfit(ctx, T, data, Tr=None, chi=None, R=None):
    """Receiver times, misfits and adjoint sources; Tr, chi, R are float64 CUDA tensors of
    shape (n_src, n_rec), (n_src, 2), (n_src, n_rec)."""
    nb = data.n_src * data.n_rec
    f64 = _f64()
    _dtype_code(T)
    _room(T=(T, _nodes(ctx) * data.n_src), Tr=(Tr, nb, f64), chi=(chi, 2 * data.n_src, f64),
          R=(R, nb, f64))
    _cuda_ok(T, Tr, chi, R)
    D = data.c_struct()
    _check(ctx, lib.tt_misfit(ctx.handle, _ptr(T), _dtype_code(T), C.byref(D), _ptr(Tr),
                              _ptr(chi), _ptr(R)))


def tt_adjoint(ctx, model, src, T, rec, R, P, opts=None, allow_unconverged=False):
    pts, n = _points(src)
    rpts, nr = _points(rec)
    ft = _model_room(ctx, model)
    _room(T=(T, _nodes(ctx) * n, ft), R=(R, n * nr, _f64()), P=(P, _nodes(ctx) * n, ft))
    M = _model(model)
    _cuda_ok(T, R, P)
    if opts is None:
        opts = default_opts(M.dtype)
    iters = (C.c_int * n)()
    st = lib.tt_adjoint(ctx.handle, C.byref(M), pts, n, _ptr(T), nr, rpts, _ptr(R), _ptr(P),
                        C.byref(opts), iters)
    _check(ctx, st, (TT_ENOTCONVERGED,) if allow_unconverged else ())
    return np.frombuffer(iters, dtype=np.int32).copy()


def tt_kernel(ctx, model, T, P, Ks, Kxi, Keta):
    n_src = T.shape[-1]
    N = _nodes(ctx)
    ft, f64 = _model_room(ctx, model), _f64()
    _room(T=(T, N * n_src, ft), P=(P, N * n_src, ft), Ks=(Ks, N, f64), Kxi=(Kxi, N, f64),
          Keta=(Keta, N, f64))
    M = _model(model)
    _cuda_ok(T, P, Ks, Kxi, Keta)
    _check(ctx, lib.tt_kernel(ctx.handle, C.byref(M), n_src, _ptr(T), _ptr(P), _ptr(Ks),
                              _ptr(Kxi), _ptr(Keta)))


def cr_pack(n_src, n_rec, pairs):
    """tt_cr_pack on host arrays: (off, other, dtobs, w) numpy arrays of tt_cr_data's table
    from rows (b, j, m, dT_obs, w) of unordered pairs."""
    P = np.ascontiguousarray(np.asarray(pairs, dtype=np.float64).reshape(-1, 5))
    n = P.shape[0]
    off = np.zeros(int(n_src) * int(n_rec) + 1, dtype=np.int32)
    other = np.zeros(2 * n, dtype=np.int32)
    dtobs = np.zeros(2 * n, dtype=np.float64)
    w = np.zeros(2 * n, dtype=np.float64)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    st = lib.tt_cr_pack(None, int(n_src), int(n_rec), n, p(P), p(off), p(other), p(dtobs), p(w))
    if st != 0:
        raise TTError(st, "tt_cr_pack refused the pair list (sources, receiver or b == j)")
    return off, other, dtobs, w


class CrData:
    """Common-receiver differential times (Eq. 4) of one batch, in the layout of tt_cr_data.
    pairs: rows (b, j, m, dT_obs, w), an unordered source pair {b, j} observed at receiver m
    with T_b^obs - T_j^obs = dT_obs and weight w; each is listed under both sources."""

    def __init__(self, n_src, n_rec, pairs, gamma=1.0, device="cuda"):
        import torch
        off, other, dtobs, w = cr_pack(n_src, n_rec, pairs)
        self.n_src, self.n_rec, self.n_entries = int(n_src), int(n_rec), int(len(other))
        self.off = torch.as_tensor(off, device=device)
        self.other = torch.as_tensor(other, device=device)
        self.dtobs = torch.as_tensor(dtobs, device=device)
        self.w = torch.as_tensor(w, device=device)
        self.gamma = float(gamma)

    def c_struct(self):
        return TTCrData(self.n_src, self.n_rec, self.n_entries, _ptr(self.off), _ptr(self.other),
                        _ptr(self.dtobs), _ptr(self.w), self.gamma)


def tt_misfit_cr(ctx, cr, Tr, chi_cr, R):
    """Eqs. 4 and A4: R += gamma dchi_cr/dT (in place), chi_cr [n_src] the sources' shares."""
    f64 = _f64()
    _room(Tr=(Tr, cr.n_src * cr.n_rec, f64), chi_cr=(chi_cr, cr.n_src, f64),
          R=(R, cr.n_src * cr.n_rec, f64))
    _cuda_ok(Tr, chi_cr, R)
    D = cr.c_struct()
    _check(ctx, lib.tt_misfit_cr(ctx.handle, C.byref(D), _ptr(Tr), _ptr(chi_cr), _ptr(R)))


def tt_field_at_points(ctx, G, pts, val, grad):
    """Values val [n_pts, M] and physical gradients grad [n_pts, M, 3] (float64) at the points
    pts [n_pts, 3] (float64: depth km, lat deg, lon deg) of the M batched fields G [..., M]
    (for relocation: tt_forward's T with the receivers as the sources)."""
    M, n_pts = G.shape[-1], pts.shape[0]
    f64 = _f64()
    _dtype_code(G)
    _room(G=(G, _nodes(ctx) * M), pts=(pts, 3 * n_pts, f64), val=(val, n_pts * M, f64),
          grad=(grad, 3 * n_pts * M, f64))
    _cuda_ok(G, pts, val, grad)
    _check(ctx, lib.tt_field_at_points(ctx.handle, _ptr(G), _dtype_code(G), G.shape[-1],
                                       pts.shape[0], _ptr(pts), _ptr(val), _ptr(grad)))


def tt_misfit_table(ctx, val, otime, data, Tr=None, chi=None, R=None):
    """tt_misfit on given arrivals Tr = val + otime[:, None] (otime may be None)."""
    nb = data.n_src * data.n_rec
    f64 = _f64()
    _room(val=(val, nb, f64), otime=(otime, data.n_src, f64), Tr=(Tr, nb, f64),
          chi=(chi, 2 * data.n_src, f64), R=(R, nb, f64))
    _cuda_ok(val, otime, Tr, chi, R)
    D = data.c_struct()
    _check(ctx, lib.tt_misfit_table(ctx.handle, _ptr(val), _ptr(otime), C.byref(D), _ptr(Tr),
                                    _ptr(chi), _ptr(R)))


def tt_reloc_kernels(ctx, R, grad, Kx, Ktau):
    """Kx [n_src, 3] = sum_m R grad, Ktau [n_src] = sum_m R (Eqs. B5-B11)."""
    n, m = R.shape[0], R.shape[1]
    f64 = _f64()
    _room(R=(R, n * m, f64), grad=(grad, 3 * n * m, f64), Kx=(Kx, 3 * n, f64),
          Ktau=(Ktau, n, f64))
    _cuda_ok(R, grad, Kx, Ktau)
    _check(ctx, lib.tt_reloc_kernels(ctx.handle, R.shape[0], R.shape[1], _ptr(R), _ptr(grad),
                                     _ptr(Kx), _ptr(Ktau)))


def tt_reloc_update(ctx, pts, otime, Kx, Ktau, step_km, step_s):
    """One normalised gradient step of the event positions pts [n, 3] and origin times
    otime [n] (may be None), in place."""
    n = pts.shape[0]
    f64 = _f64()
    _room(pts=(pts, 3 * n, f64), otime=(otime, n, f64), Kx=(Kx, 3 * n, f64),
          Ktau=(Ktau, n, f64))
    _cuda_ok(pts, otime, Kx, Ktau)
    _check(ctx, lib.tt_reloc_update(ctx.handle, pts.shape[0], _ptr(pts), _ptr(otime), _ptr(Kx),
                                    _ptr(Ktau), step_km, step_s))


def tt_tele2d(ctx, s_r, r_min, r_max, d_max_deg, r_src, T, tol=1e-8, max_iter=500,
              allow_unconverged=False):
    """2-D traveltimes of teleseismic events in a 1-D model: s_r [n_r] (CUDA, float32 or
    float64) slowness at the radii r_min..r_max (km); r_src [n_ev] the events' radii (host);
    T [n_ev, n_r, n_d] output (CUDA, same dtype) on Delta = 0..d_max_deg. Returns the
    iterations per event."""
    n_ev, n_r, n_d = T.shape
    _dtype_code(T)
    _room(s_r=(s_r, n_r, T.dtype))
    if len(np.atleast_1d(r_src)) < n_ev:
        raise ValueError("r_src holds %d radii for %d events" % (len(np.atleast_1d(r_src)), n_ev))
    _cuda_ok(s_r, T)
    rs = np.ascontiguousarray(r_src, dtype=np.float64)
    it = (C.c_int * n_ev)()
    st = lib.tt_tele2d(ctx.handle, _dtype_code(T), n_r, n_d, r_min, r_max, d_max_deg, _ptr(s_r),
                       n_ev, rs.ctypes.data_as(C.POINTER(C.c_double)), tol, max_iter, _ptr(T), it)
    _check(ctx, st, (TT_ENOTCONVERGED,) if allow_unconverged else ())
    return np.frombuffer(it, dtype=np.int32).copy()


def tt_tele_region_times(ctx, T2, r_min, r_max, d_max_deg, events, T):
    """The 2-D times T2 [n_ev, n_r, n_d] interpolated at every node of the context's grid
    for events at (depth, lat, lon) points (only lat and lon are read): T [..., n_ev]."""
    n_ev, n_r, n_d = T2.shape
    pts, n = _points(events)
    if n < n_ev:
        raise ValueError("%d event positions for %d events" % (n, n_ev))
    _dtype_code(T2)
    _room(T=(T, _nodes(ctx) * n_ev, T2.dtype))
    _cuda_ok(T2, T)
    _check(ctx, lib.tt_tele_region_times(ctx.handle, _dtype_code(T2), n_r, n_d, r_min, r_max,
                                         d_max_deg, _ptr(T2), n_ev, pts, _ptr(T)))


def tt_forward_tele(ctx, model, T, opts=None, allow_unconverged=False):
    """The region's solve for teleseismic events with the faces of T [..., n_ev] held fixed
    (T holds the faces' data and the interior's start on entry, the solution on return).
    Returns the iterations per event."""
    n_ev = T.shape[-1]
    ft = _model_room(ctx, model)
    _room(T=(T, _nodes(ctx) * n_ev, ft))
    M = _model(model)
    _cuda_ok(T)
    if opts is None:
        opts = default_opts(M.dtype)
    it = (C.c_int * n_ev)()
    st = lib.tt_forward_tele(ctx.handle, C.byref(M), n_ev, _ptr(T), C.byref(opts), it)
    _check(ctx, st, (TT_ENOTCONVERGED,) if allow_unconverged else ())
    return np.frombuffer(it, dtype=np.int32).copy()


def tt_kernel_density(ctx, P_hat, Kd):
    """Kd += sum over sources of P_hat (Eq. 19); P_hat [..., n_src] from tt_adjoint with R = 1."""
    _dtype_code(P_hat)
    _room(P_hat=(P_hat, _nodes(ctx) * P_hat.shape[-1]), Kd=(Kd, _nodes(ctx), _f64()))
    _cuda_ok(P_hat, Kd)
    _check(ctx, lib.tt_kernel_density(ctx.handle, _ptr(P_hat), P_hat.shape[-1],
                                      _dtype_code(P_hat), _ptr(Kd)))


def tt_kernel_normalize(ctx, Ks, Kxi, Keta, Kd, eps, zeta):
    """Eq. 18 in place: K <- K / (Kd + eps)^zeta."""
    N = _nodes(ctx)
    f64 = _f64()
    _room(Ks=(Ks, N, f64), Kxi=(Kxi, N, f64), Keta=(Keta, N, f64), Kd=(Kd, N, f64))
    _cuda_ok(Ks, Kxi, Keta, Kd)
    _check(ctx, lib.tt_kernel_normalize(ctx.handle, _ptr(Ks), _ptr(Kxi), _ptr(Keta), _ptr(Kd),
                                        float(eps), float(zeta)))


def tt_kernel_normalize_rel(ctx, Ks, Kxi, Keta, Kd, eps_rel, zeta):
    """Eq. 18 in place with eps = eps_rel max(Kd), the maximum taken on the device."""
    N = _nodes(ctx)
    f64 = _f64()
    _room(Ks=(Ks, N, f64), Kxi=(Kxi, N, f64), Keta=(Keta, N, f64), Kd=(Kd, N, f64))
    _cuda_ok(Ks, Kxi, Keta, Kd)
    _check(ctx, lib.tt_kernel_normalize_rel(ctx.handle, _ptr(Ks), _ptr(Kxi), _ptr(Keta),
                                            _ptr(Kd), float(eps_rel), float(zeta)))


def tt_misfit_total(ctx, chi, alpha=1.0, beta=1.0, chi_cr=None, gamma=1.0):
    """alpha sum chi[:, 0] + beta sum chi[:, 1] (+ gamma sum chi_cr) of a batch, an FP64 sum
    on the device; chi [n_src, 2] and chi_cr [n_src] float64 CUDA tensors."""
    n = chi.shape[0]
    f64 = _f64()
    _room(chi=(chi, 2 * n, f64), chi_cr=(chi_cr, n, f64))
    _cuda_ok(chi, chi_cr)
    out = C.c_double()
    _check(ctx, lib.tt_misfit_total(ctx.handle, n, _ptr(chi), float(alpha), float(beta),
                                    _ptr(chi_cr), float(gamma), C.byref(out)))
    return out.value


def mgrid(n_r, n_t, n_p, n_grids):
    """Description of n_grids offset inversion grids of n_r x n_t x n_p nodes."""
    return TTMgrid(n_r, n_t, n_p, n_grids)


def tt_mgrid_project(ctx, mg, K, G):
    """Eq. 17: G [n_grids, n_r, n_t, n_p] (float64) from the kernel K (float64, grid shape)."""
    _room(K=(K, _nodes(ctx), _f64()), G=(G, mg.n_grids * mg.n_r * mg.n_t * mg.n_p, _f64()))
    _cuda_ok(K, G)
    _check(ctx, lib.tt_mgrid_project(ctx.handle, C.byref(mg), _ptr(K), _ptr(G)))


def tt_mgrid_expand(ctx, mg, G, D):
    """Eq. 15: D (float64, grid shape) from the coefficients G."""
    _room(G=(G, mg.n_grids * mg.n_r * mg.n_t * mg.n_p, _f64()), D=(D, _nodes(ctx), _f64()))
    _cuda_ok(G, D)
    _check(ctx, lib.tt_mgrid_expand(ctx.handle, C.byref(mg), _ptr(G), _ptr(D)))


def tt_model_update(ctx, model, Ds, Dxi, Deta, step):
    """One gradient-descent step on the model's arrays, in place (see tt.h)."""
    N = _nodes(ctx)
    _model_room(ctx, model)
    f64 = _f64()
    _room(Ds=(Ds, N, f64), Dxi=(Dxi, N, f64), Deta=(Deta, N, f64))
    M = _model(model)
    _cuda_ok(Ds, Dxi, Deta)
    _check(ctx, lib.tt_model_update(ctx.handle, C.byref(M), _ptr(Ds), _ptr(Dxi), _ptr(Deta),
                                    float(step)))


def tt_get_stats(ctx, which=TT_STATS_FORWARD):
    """Measurements of the last forward or adjoint sweep, as a dict."""
    s = TTStats()
    _check(ctx, lib.tt_get_stats(ctx.handle, which, C.byref(s)))
    return {k: getattr(s, k) for k, _ in TTStats._fields_}


def tt_misfit_noalloc(grid, T, data, Tr=None, chi=None, R=None, stream=None):
    """tt_misfit without a context and without device allocation (static scratch; at most
    TT_NOALLOC_MAX_REC receivers). Same outputs as tt_misfit."""
    import torch
    G = make_grid(grid)
    nb = data.n_src * data.n_rec
    f64 = _f64()
    _dtype_code(T)
    _room(T=(T, int(G.n_r) * int(G.n_t) * int(G.n_p) * data.n_src), Tr=(Tr, nb, f64),
          chi=(chi, 2 * data.n_src, f64), R=(R, nb, f64))
    _cuda_ok(T, Tr, chi, R)
    if stream is None:
        stream = torch.cuda.current_stream()
    D = data.c_struct()
    err = C.create_string_buffer(256)
    st = lib.tt_misfit_noalloc(C.byref(G), _ptr(T), _dtype_code(T), C.byref(D), _ptr(Tr),
                               _ptr(chi), _ptr(R), C.c_void_p(stream.cuda_stream), err, 256)
    if st != TT_OK:
        raise TTError(st, err.value.decode())


class Plan:
    """A whole step over one batch captured into a CUDA graph (tt_plan). Keeps references to
    every buffer it binds."""

    def __init__(self, ctx, handle, n_src, refs):
        self.ctx, self.handle, self.n_src, self._refs = ctx, handle, n_src, refs

    def close(self):
        if self.handle:
            lib.tt_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tt_plan_create(ctx, model, src, data, tau, T, P, chi, R, Ks, Kxi, Keta, opts=None,
                   cr=None, Tr=None, chi_cr=None):
    """A captured step (see tt.h). With cr (the batch's CrData), Tr [n_src, n_rec] and
    chi_cr [n_src] (float64 CUDA tensors) the step includes the common-receiver terms
    (tt_plan_create_cr)."""
    pts, n = _points(src)
    N = _nodes(ctx)
    ft, f64 = _model_room(ctx, model), _f64()
    _room(tau=(tau, N * n, ft), T=(T, N * n, ft), P=(P, N * n, ft), chi=(chi, 2 * n, f64),
          R=(R, n * data.n_rec, f64), Ks=(Ks, N, f64), Kxi=(Kxi, N, f64), Keta=(Keta, N, f64))
    if cr is not None:
        if Tr is None or chi_cr is None:
            raise ValueError("cr needs the Tr and chi_cr buffers")
        _room(Tr=(Tr, n * data.n_rec, f64), chi_cr=(chi_cr, n, f64))
    M = _model(model)
    _cuda_ok(tau, T, P, chi, R, Ks, Kxi, Keta, Tr, chi_cr)
    if opts is None:
        opts = default_opts(M.dtype)
    D = data.c_struct()
    h = C.c_void_p()
    if cr is None:
        st = lib.tt_plan_create(C.byref(h), ctx.handle, C.byref(M), pts, n, C.byref(D),
                                C.byref(opts), _ptr(tau), _ptr(T), _ptr(P), _ptr(chi), _ptr(R),
                                _ptr(Ks), _ptr(Kxi), _ptr(Keta))
        crs = None
    else:
        crs = cr.c_struct()
        st = lib.tt_plan_create_cr(C.byref(h), ctx.handle, C.byref(M), pts, n, C.byref(D),
                                   C.byref(crs), C.byref(opts), _ptr(tau), _ptr(T), _ptr(P),
                                   _ptr(chi), _ptr(Tr), _ptr(chi_cr), _ptr(R), _ptr(Ks),
                                   _ptr(Kxi), _ptr(Keta))
    _check(ctx, st)
    return Plan(ctx, h, n, (model, data, tau, T, P, chi, R, Ks, Kxi, Keta, pts, D, opts, cr,
                            crs, Tr, chi_cr))


def tt_plan_run(plan, allow_unconverged=False):
    """Replays the step; returns (forward iterations, adjoint iterations)."""
    itf = (C.c_int * plan.n_src)()
    ita = (C.c_int * plan.n_src)()
    st = lib.tt_plan_run(plan.handle, itf, ita)
    _check(plan.ctx, st, (TT_ENOTCONVERGED,) if allow_unconverged else ())
    return (np.frombuffer(itf, dtype=np.int32).copy(), np.frombuffer(ita, dtype=np.int32).copy())


# ----------------------------------------------------------------------- warm-start network

def tt_net_param_count():
    return int(lib.tt_net_param_count())


def _f32(*tensors):
    import torch
    for x in tensors:
        if x.dtype != torch.float32 or not x.is_contiguous():
            raise TypeError("network buffers must be contiguous float32 CUDA tensors")


# input channels of the network per node: s / s_ref - 1, xi, eta and the source offset
NET_FEATURES = 6


def tt_net_nodes(ctx):
    """Node count of the network's grid (the context's grid, or every other node along each
    axis after tt_net_set_stride(ctx, 2)): the sizes the library's tt_net_nodes reports, from
    the grid and the stride this binding set."""
    c = getattr(ctx, "net_stride", 1)
    g = ctx.grid
    axis = lambda n: int(n) if c == 1 else (int(n) + c - 2) // c + 1
    return axis(g.n_r) * axis(g.n_t) * axis(g.n_p)


def tt_net_set_stride(ctx, stride):
    """The network's grid: 1 = the context's grid, 2 = every other node along each axis (the
    warm start interpolates the prediction to the other nodes). Goes with the weights."""
    _check(ctx, lib.tt_net_set_stride(ctx.handle, int(stride)))
    ctx.net_stride = int(stride)


def _net_room(ctx, n_grids, **named):
    """Sizes of the network's buffers: parameter-sized (theta, grad, m, v), inputs
    n_grids x Nn x NET_FEATURES (x), per-node outputs n_grids x Nn (y, target, mask), Nn the
    network grid's nodes."""
    N = tt_net_nodes(ctx)
    per = {"theta": tt_net_param_count(), "grad": tt_net_param_count(),
           "m": tt_net_param_count(), "v": tt_net_param_count(),
           "x": n_grids * N * NET_FEATURES, "y": n_grids * N, "target": n_grids * N,
           "mask": n_grids * N}
    _room(**{k: (v, per[k]) for k, v in named.items()})


def tt_net_features(ctx, model, src, x):
    """x: float32 [n_src, Nn, 6] at the network grid's nodes (for stride 1 any contiguous
    shape of that size, e.g. [n_src, N_r, N_t, N_p, 6])."""
    _model_room(ctx, model)
    pts, n = _points(src)
    _f32(x)
    _room(x=(x, n * tt_net_nodes(ctx) * NET_FEATURES))
    M = _model(model)
    _cuda_ok(x)
    _check(ctx, lib.tt_net_features(ctx.handle, C.byref(M), pts, n, _ptr(x)))


def tt_net_forward(ctx, theta, x, y):
    """y[n] = network(x[n]) for the n = x.shape[0] grids of the context."""
    _f32(theta, x, y)
    _net_room(ctx, x.shape[0], theta=theta, x=x, y=y)
    _cuda_ok(theta, x, y)
    _check(ctx, lib.tt_net_forward(ctx.handle, _ptr(theta), _ptr(x), x.shape[0], _ptr(y)))


def tt_net_loss_grad(ctx, theta, x, target, mask, grad):
    """Masked MSE of the network output against target; writes grad, returns the loss."""
    _f32(theta, x, target, mask, grad)
    _net_room(ctx, x.shape[0], theta=theta, x=x, target=target, mask=mask, grad=grad)
    _cuda_ok(theta, x, target, mask, grad)
    loss = C.c_double()
    _check(ctx, lib.tt_net_loss_grad(ctx.handle, _ptr(theta), _ptr(x), _ptr(target), _ptr(mask),
                                     x.shape[0], _ptr(grad), C.byref(loss)))
    return loss.value


def tt_net_loss_grad_tc(ctx, theta, x, target, mask, grad):
    """tt_net_loss_grad with the convolutions on the tensor cores (BF16 operands)."""
    _f32(theta, x, target, mask, grad)
    _net_room(ctx, x.shape[0], theta=theta, x=x, target=target, mask=mask, grad=grad)
    _cuda_ok(theta, x, target, mask, grad)
    loss = C.c_double()
    _check(ctx, lib.tt_net_loss_grad_tc(ctx.handle, _ptr(theta), _ptr(x), _ptr(target),
                                        _ptr(mask), x.shape[0], _ptr(grad), C.byref(loss)))
    return loss.value


def tt_net_adam(ctx, theta, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    _f32(theta, grad, m, v)
    _net_room(ctx, 0, theta=theta, grad=grad, m=m, v=v)
    _cuda_ok(theta, grad, m, v)
    _check(ctx, lib.tt_net_adam(ctx.handle, _ptr(theta), _ptr(grad), _ptr(m), _ptr(v), int(step),
                                lr, beta1, beta2, eps))


def tt_net_set_weights(ctx, theta):
    _f32(theta)
    _net_room(ctx, 0, theta=theta)
    _cuda_ok(theta)
    _check(ctx, lib.tt_net_set_weights(ctx.handle, _ptr(theta)))


AUTOTUNE_CANDIDATES = ("nodes/1 group", "nodes/2 groups", "nodes/4 groups", "nodes/8 groups",
                       "tiles 2x4x8", "tiles 4x4x4", "tiles 2x8x8")


def tt_autotune(ctx, model, src, opts):
    """Times the forward sweep's launch configurations on this workload and writes the
    fastest into opts; returns {candidate: ms per iteration} (0 = skipped or cached)."""
    _model_room(ctx, model)
    M = _model(model)
    pts, n = _points(src)
    ms = (C.c_double * len(AUTOTUNE_CANDIDATES))()
    _check(ctx, lib.tt_autotune(ctx.handle, C.byref(M), pts, n, C.byref(opts), ms))
    return dict(zip(AUTOTUNE_CANDIDATES, list(ms)))


ADJ_AUTOTUNE_CANDIDATES = ("all sources/1 group", "all sources/2 groups",
                           "all sources/4 groups", "all sources/8 groups", "chunks of 128",
                           "chunks of 64/1 group")


def tt_autotune_adjoint(ctx, model, src, T, rec, R, opts):
    """Times the adjoint sweep's launch configurations on this batch (T, R as for tt_adjoint)
    and writes the fastest into opts; returns {candidate: ms per solve} (0 = skipped or
    cached)."""
    pts, n = _points(src)
    rpts, nr = _points(rec)
    ft = _model_room(ctx, model)
    _room(T=(T, _nodes(ctx) * n, ft), R=(R, n * nr, _f64()))
    M = _model(model)
    _cuda_ok(T, R)
    ms = (C.c_double * len(ADJ_AUTOTUNE_CANDIDATES))()
    _check(ctx, lib.tt_autotune_adjoint(ctx.handle, C.byref(M), pts, n, _ptr(T), nr, rpts,
                                        _ptr(R), C.byref(opts), ms))
    return dict(zip(ADJ_AUTOTUNE_CANDIDATES, list(ms)))


def tt_net_start(ctx, model, src, tau):
    """The warm start's tau (opts.init = 2) without the sweep: tau [N_r, N_t, N_p, n_src] of
    the model's dtype = 1 + the clamped prediction, 1 on the fixed sets."""
    pts, n = _points(src)
    ft = _model_room(ctx, model)
    _room(tau=(tau, _nodes(ctx) * n, ft))
    M = _model(model)
    _cuda_ok(tau)
    _check(ctx, lib.tt_net_start(ctx.handle, C.byref(M), pts, n, _ptr(tau)))


def tt_net_infer(ctx, x, y):
    """Warm-start inference with the weights of tt_net_set_weights (tensor cores)."""
    _f32(x, y)
    _net_room(ctx, x.shape[0], x=x, y=y)
    _cuda_ok(x, y)
    _check(ctx, lib.tt_net_infer(ctx.handle, _ptr(x), x.shape[0], _ptr(y)))
