"""Helpers for the GPU tests: run a workload through the C ABI, run it through the oracle."""
import numpy as np


def to_dev(a, dtype, device="cuda"):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=device)


def gpu_solve(w, dtype_name="f32", opts=None, adj_opts=None, steps=("fwd", "misfit", "adj", "kernel"),
              ctx=None, tau_init=None):
    """Runs the batched path on the GPU; returns numpy arrays in (n_r, n_t, n_p, B) layout."""
    import torch
    import paper_2412_00031_gb300 as tt
    dt = torch.float32 if dtype_name == "f32" else torch.float64
    code = tt.TT_F32 if dtype_name == "f32" else tt.TT_F64
    g = w.grid
    B = w.n_src
    model = tuple(to_dev(a, dt) for a in (w.s, w.xi, w.eta))
    own = ctx is None
    if own:
        ctx = tt.tt_ctx_create(g.as_dict())
    shape = g.shape + (B,)
    out = {}
    tau = torch.empty(shape, dtype=dt, device="cuda")
    if tau_init is not None:
        tau.copy_(to_dev(tau_init, dt))
    T = torch.empty_like(tau)
    o = opts if opts is not None else tt.default_opts(code)
    out["iters_fwd"] = tt.tt_forward(ctx, model, w.src, tau, T, o)
    out["tau"], out["T"] = tau.cpu().numpy(), T.cpu().numpy()
    if "misfit" in steps:
        data = tt.DeviceData.from_workload(w)
        R = torch.empty((B, data.n_rec), dtype=torch.float64, device="cuda")
        chi = torch.empty((B, 2), dtype=torch.float64, device="cuda")
        Tr = torch.empty((B, data.n_rec), dtype=torch.float64, device="cuda")
        tt.tt_misfit(ctx, T, data, Tr, chi, R)
        out["R"], out["chi"], out["Tr"] = R.cpu().numpy(), chi.cpu().numpy(), Tr.cpu().numpy()
    if "adj" in steps:
        P = torch.empty_like(tau)
        ao = adj_opts if adj_opts is not None else o
        out["iters_adj"] = tt.tt_adjoint(ctx, model, w.src, T, w.rec, R, P, ao)
        out["P"] = P.cpu().numpy()
    if "kernel" in steps:
        K = [torch.zeros(g.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
        tt.tt_kernel(ctx, model, T, P, *K)
        out["K"] = [k.cpu().numpy() for k in K]
    torch.cuda.synchronize()
    if own:
        ctx.close()
    return out


def rounded_model(w, dtype_name):
    """The model as the GPU sees it (float32-rounded for the f32 path), in float64."""
    if dtype_name == "f64":
        return w.s, w.xi, w.eta
    return tuple(np.asarray(a, dtype=np.float32).astype(np.float64) for a in (w.s, w.xi, w.eta))


def oracle_solve(w, model=None, tol=1e-10, with_kernel=True):
    import oracle as O
    g = w.grid.as_dict()
    s, xi, eta = model if model is not None else (w.s, w.xi, w.eta)
    res = []
    K = [np.zeros(w.grid.shape) for _ in range(3)]
    for b in range(w.n_src):
        r = O.solve_source(g, s, xi, eta, w.src[b], w.rec, w.source_data(b), tol_fwd=tol,
                           tol_adj=tol, max_iter=2000)
        if with_kernel:
            O.kernel_add(g, s, r["T"], r["P"], *K)
        res.append(r)
    return res, K


def rel_linf(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)
