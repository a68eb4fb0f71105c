"""Benchmark: forward + adjoint source-solves per second on one GB300.

One step is one pass of the whole hot path over one batch of sources: the factored
fast-sweeping forward solve of every source to convergence, receiver misfits and adjoint
sources, the adjoint solve of every source to convergence and the FP64 accumulation of the
sensitivity kernels. The default workload is the anisotropic batch: a 121 x 161 x 161
spherical grid (depth 0-100 km, 3 x 4 deg), Vp 5 -> 8 km/s with a +-4 % checkerboard, xi
and eta checkerboards of amplitude 0.04, 256 sources with 20-200 receivers each; FP32 sweeps
with FP64 reductions; synthetic inputs (tt_inputs.anisotropic_batch).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank solves its own batch (sources are independent); timing
is the maximum over ranks. Prints one JSON line on rank 0.

--impl reference times the FP64 CPU oracle on the host cores instead (bounded samples of the
same workload, scaled to the same metric).

The JSON line also carries legs measured in the same run: the unbatched step, the
retire-and-refill forward, the warm-started step, and the step with the anisotropic Godunov
forward solver (`godunov`; the headline value is the Lax-Friedrichs step). Other modes:
--infer-only N (the warm start's tensor-core inference alone) and --inversion K (K step
attempts of the inversion loop on the 201 x 201 x 101 workload).
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import tt_inputs as I  # noqa: E402

METRIC = "forward+adjoint source-solves/s on 1 GB300 at 121×161×161; % HBM roofline"
UNIT = "source-solves/s"
FWD_BYTES_PER_UPDATE = 8      # FP32 tau read + write per (node, source) update
FWD_BYTES_PER_NODE_SWEEP = 12  # s, xi, eta once per node per sweep (shared by the batch)
ADJ_BYTES_PER_UPDATE = 12     # FP32 P read + write and T read per (node, source) update
ADJ_BYTES_PER_NODE_SWEEP = 8  # xi, eta once per node per sweep
KACC_BYTES_PER_PAIR = 8       # FP32 T and P read per (node, source) of the kernel accumulation
KACC_BYTES_PER_NODE = 52      # s read + FP64 read-modify-write of K_s, K_xi, K_eta per node


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def bf16_peak():
    """Dense BF16 tensor peak (burst, for a kernel timed alone) in TFLOP/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (burst)"
    except Exception:
        return 1900.0, "fallback"


def hbm_kernel(ms, pairs, nodes, per_pair, per_node, hbm):
    """HBM roofline entry of one launch: algorithmic bytes / CUDA-event time."""
    b = pairs * per_pair + nodes * per_node
    gbs = b / (ms * 1e-3) / 1e9
    return {"ms": ms, "algorithmic_bytes": b, "GBps": gbs, "frac_hbm": gbs / hbm}


def workload_config(w, n_gpus):
    g = w.grid
    return {"workload": "anisotropic batch %dx%dx%d (r x lat x lon), depth %g-%g km, "
                        "%gx%g deg, %d sources, 20-200 receivers each"
                        % (g.n_r, g.n_t, g.n_p, g.depth_min_km, g.depth_max_km,
                           g.lat_max_deg - g.lat_min_deg, g.lon_max_deg - g.lon_min_deg, w.n_src),
            "grid": [g.n_r, g.n_t, g.n_p], "n_src_per_gpu": w.n_src,
            "receivers": int(len(w.rec)), "abs_records": int(len(w.abs_rec)),
            "cs_pairs": int(len(w.cs_m)), "precision": "fp32 sweeps, fp64 misfit and kernels",
            "tol_fwd": 1e-6, "tol_adj": 1e-6,
            "l2": "inputs larger than L2 (tau, T and P are 3.2 GB each)",
            "parallelism": "sources sharded across %d GPU(s)" % n_gpus}


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU arm

class GpuPath:
    """Device buffers and one step of the hot path through the C ABI."""

    def __init__(self, w, device):
        import torch
        import paper_2412_00031_gb300 as tt
        self.tt, self.torch, self.w, self.dev = tt, torch, w, device
        g = w.grid
        B = w.n_src
        f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=device)
        self.model = (f32(w.s), f32(w.xi), f32(w.eta))
        self.ctx = tt.tt_ctx_create(g.as_dict())
        shape = g.shape + (B,)
        self.tau = torch.empty(shape, dtype=torch.float32, device=device)
        self.T = torch.empty_like(self.tau)
        self.P = torch.empty_like(self.tau)
        self.data = tt.DeviceData.from_workload(w, device=device)
        nr = self.data.n_rec
        self.R = torch.empty((B, nr), dtype=torch.float64, device=device)
        self.chi = torch.empty((B, 2), dtype=torch.float64, device=device)
        self.K = [torch.zeros(g.shape, dtype=torch.float64, device=device) for _ in range(3)]
        self.opts = tt.default_opts(tt.TT_F32)
        self.allow_unconverged = False
        self.iters = []
        self.plan = None

    def use_plan(self):
        """Captures the whole step into a CUDA graph (tt_plan) and replays it from then on."""
        tt = self.tt
        self.plan = tt.tt_plan_create(self.ctx, self.model, self.w.src, self.data, self.tau,
                                      self.T, self.P, self.chi, self.R, *self.K, opts=self.opts)

    def step(self):
        tt = self.tt
        if self.plan is not None:
            itf, ita = tt.tt_plan_run(self.plan, allow_unconverged=self.allow_unconverged)
            fs = tt.tt_get_stats(self.ctx, tt.TT_STATS_FORWARD)
            as_ = tt.tt_get_stats(self.ctx, tt.TT_STATS_ADJOINT)
            self.iters.append((itf, ita, fs, as_, self.kernel_stats()))
            return
        for k in self.K:
            k.zero_()
        au = self.allow_unconverged
        itf = tt.tt_forward(self.ctx, self.model, self.w.src, self.tau, self.T, self.opts,
                            allow_unconverged=au)
        tt.tt_misfit(self.ctx, self.T, self.data, None, self.chi, self.R)
        ita = tt.tt_adjoint(self.ctx, self.model, self.w.src, self.T, self.w.rec, self.R,
                            self.P, self.opts, allow_unconverged=au)
        tt.tt_kernel(self.ctx, self.model, self.T, self.P, *self.K)
        fs = tt.tt_get_stats(self.ctx, tt.TT_STATS_FORWARD)
        as_ = tt.tt_get_stats(self.ctx, tt.TT_STATS_ADJOINT)
        self.iters.append((itf, ita, fs, as_, self.kernel_stats()))

    def launches(self):
        return self.tt.tt_get_stats(self.ctx, self.tt.TT_STATS_FORWARD)["launches"]

    def kernel_stats(self):
        return self.tt.tt_get_stats(self.ctx, self.tt.TT_STATS_KERNEL)


def run_e2e(gp, w, steps):
    """Same metric through the public API with host inputs: every step copies the model and
    the observations from pinned host memory and reads back the misfits and the kernels."""
    torch = gp.torch
    host = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()
            for a in (w.s, w.xi, w.eta)]
    d = gp.data
    dev_data = [d.abs_off, d.abs_rec, d.abs_tobs, d.abs_w, d.cs_off, d.cs_m, d.cs_i, d.cs_dtobs,
                d.cs_w]
    host_data = [t.cpu().pin_memory() for t in dev_data]
    out_chi = torch.empty(gp.chi.shape, dtype=torch.float64).pin_memory()
    out_K = [torch.empty(k.shape, dtype=torch.float64).pin_memory() for k in gp.K]
    h2d = sum(t.numel() * t.element_size() for t in host + host_data)
    d2h = out_chi.numel() * 8 + sum(k.numel() * 8 for k in out_K)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        for dst, src in zip(gp.model, host):
            dst.copy_(src, non_blocking=True)
        for dst, src in zip(dev_data, host_data):
            dst.copy_(src, non_blocking=True)
        gp.step()
        out_chi.copy_(gp.chi, non_blocking=True)
        for dst, src in zip(out_K, gp.K):
            dst.copy_(src, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return ms, h2d, d2h


def kernel_source_digest():
    h = hashlib.sha256()
    for name in ("tt_sweep.cu", "tt_common.cuh", "tt_internal.h"):
        with open(os.path.join(ROOT, "paper_2412_00031_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(digest, updates_per_launch):
    """DRAM bytes per launch of the forward sweep from the committed ncu summary, scaled by
    node updates; None if the summary is missing or was taken on different kernel source."""
    path = os.path.join(ROOT, "profiles", "fwd_sweep_kernel_anisotropic.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m_d = re.search(r"kernel source digest:\s*`?([0-9a-f]{16})", text)
    m_b = re.search(r"dram bytes per node update:\s*([0-9.eE+-]+)", text)
    if not m_d or not m_b or m_d.group(1) != digest:
        return None
    return float(m_b.group(1)) * updates_per_launch


def gpu_arm(args, rank, world):
    import torch
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = I.anisotropic_batch(seed=rank_seed(rank), n_src=args.n_src)
    gp = GpuPath(w, dev)
    gp.opts.sweep_schedule = args.schedule
    gp.opts.adj_chunk = args.adj_chunk
    gp.opts.launch_blocks = args.launch_blocks
    gp.opts.scheme = args.scheme
    if args.max_iter_fwd or args.max_iter_adj:  # profiling runs only: bounded iterations
        gp.opts.max_iter_fwd = args.max_iter_fwd or gp.opts.max_iter_fwd
        gp.opts.max_iter_adj = args.max_iter_adj or gp.opts.max_iter_adj
        gp.allow_unconverged = True
    tuned = None
    if args.autotune and args.schedule == 0:
        ms = gp.tt.tt_autotune(gp.ctx, gp.model, w.src, gp.opts)
        tuned = {"ms_per_iteration": {k: round(v, 3) for k, v in ms.items()},
                 "chosen": {"sweep_schedule": gp.opts.sweep_schedule,
                            "fwd_groups": gp.opts.fwd_groups}}
    if args.autotune and args.adj_chunk == 0:
        gp.step()                 # T and R of this batch for the adjoint tuner
        ms = gp.tt.tt_autotune_adjoint(gp.ctx, gp.model, w.src, gp.T, w.rec, gp.R, gp.opts)
        tuned = dict(tuned or {}, adjoint={
            "ms_per_solve": {k: round(v, 3) for k, v in ms.items()},
            "chosen": {"adj_chunk": gp.opts.adj_chunk, "adj_groups": gp.opts.adj_groups}})
    if args.plan:
        gp.use_plan()
    for _ in range(args.warmup):
        gp.step()
    gp.iters.clear()
    dist_barrier(world)
    torch.cuda.synchronize()
    launches0 = gp.launches()
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        gp.step()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = gp.launches() - launches0
    ms = e0.elapsed_time(e1) / args.steps
    ms = dist_max(ms, world)
    dist_barrier(world)

    if args.no_e2e:
        e2e_ms, h2d, d2h = float("nan"), 0, 0
    else:
        e2e_ms, h2d, d2h = run_e2e(gp, w, max(1, args.steps))
        e2e_ms = dist_max(e2e_ms, world)

    # roofline of the dominant kernel (forward sweep) and the adjoint sweep
    hbm, peak_kind = peaks()
    fwd = [s[2] for s in gp.iters]
    adj = [s[3] for s in gp.iters]
    f_ms = float(np.mean([s["sweep_ms"] for s in fwd]))
    a_ms = float(np.mean([s["sweep_ms"] for s in adj]))
    f_upd = float(np.mean([s["node_updates"] for s in fwd]))
    f_sw = float(np.mean([s["node_sweeps"] for s in fwd]))
    a_upd = float(np.mean([s["node_updates"] for s in adj]))
    a_sw = float(np.mean([s["node_sweeps"] for s in adj]))
    f_bytes = f_upd * FWD_BYTES_PER_UPDATE + f_sw * FWD_BYTES_PER_NODE_SWEEP
    a_bytes = a_upd * ADJ_BYTES_PER_UPDATE + a_sw * ADJ_BYTES_PER_NODE_SWEEP
    f_gbs = f_bytes / (f_ms * 1e-3) / 1e9
    a_gbs = a_bytes / (a_ms * 1e-3) / 1e9
    digest = kernel_source_digest()
    traffic = profiled_traffic(digest, f_upd)
    itf = np.concatenate([s[0] for s in gp.iters])
    ita = np.concatenate([s[1] for s in gp.iters])
    kacc = [s[4] for s in gp.iters]
    k_ms = float(np.mean([s["sweep_ms"] for s in kacc]))
    kernel_accum = hbm_kernel(k_ms, float(np.mean([s["node_updates"] for s in kacc])),
                              float(np.mean([s["node_sweeps"] for s in kacc])),
                              KACC_BYTES_PER_PAIR, KACC_BYTES_PER_NODE, hbm)
    kernel_accum["bytes_per_unit"] = "%d B per (node, source) + %d B per node" % (
        KACC_BYTES_PER_PAIR, KACC_BYTES_PER_NODE)
    value = world * w.n_src / (ms * 1e-3)
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(w, world),
        "step_form": ("one captured CUDA graph per step (tt_plan)" if args.plan
                      else "four C-ABI calls per step"),
        "roofline": {"bound": "hbm", "kernel": "fwd_sweep_kernel<float>", "achieved": f_gbs,
                     "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s", "frac": f_gbs / hbm,
                     "traffic": traffic, "algorithmic_bytes_per_launch": f_bytes,
                     "launch_ms": f_ms, "kernel_source_digest": digest},
        "kernels": {
            "fwd_sweep": {"ms": f_ms, "node_updates": f_upd, "GBps": f_gbs,
                          "frac_hbm": f_gbs / hbm, "iters_mean": float(itf.mean()),
                          "iters_max": int(itf.max())},
            "adj_sweep": {"ms": a_ms, "node_updates": a_upd, "GBps": a_gbs,
                          "frac_hbm": a_gbs / hbm, "iters_mean": float(ita.mean()),
                          "iters_max": int(ita.max())},
            "kernel_accum": kernel_accum,
            "rest_ms": ms - f_ms - a_ms - k_ms},
        "e2e": {"value": world * w.n_src / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": e2e_ms},
        "autotune": tuned,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if args.unbatched > 0:
        result["unbatched"] = unbatched_leg(args, w, dev, world)
    if args.refill_sources > w.n_src:
        result["refill"] = refill_leg(args, dev, world, w.n_src, gp)
    if args.warm_start and os.path.exists(args.warm_start):
        result["warm_start"] = warm_leg(args, gp, world)
    if args.godunov:
        result["godunov"] = godunov_leg(args, gp, world)
    if args.train_timing:
        result["warm_start_training"] = training_leg(dev)
    return result, w, (float(itf.mean()), float(ita.mean()))


def training_leg(dev, steps=10, warmup=3):
    """One training step of the warm-start network (masked MSE and its gradient over a batch of
    8 grids of 81^3, the trainer's batch) with the FP32 convolutions and with the convolutions
    on the tensor cores (tt_net_loss_grad_tc), timed with CUDA events after a warm-up."""
    import torch
    import paper_2412_00031_gb300 as tt
    from paper_2412_00031_gb300 import warmstart as WS
    g, models = I.random_field_models(seed=I.SEED_BASE + 40, n_models=1, shape=(81, 81, 81),
                                      n_src=8)
    s, xi, eta, src = models[0]
    ctx = tt.tt_ctx_create(g.as_dict())
    model = tuple(torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)
                  for a in (s, xi, eta))
    x = torch.empty((len(src),) + g.shape + (6,), dtype=torch.float32, device=dev)
    tt.tt_net_features(ctx, model, src, x)
    gen = torch.Generator(device=dev).manual_seed(7)
    target = 1.0 + 0.05 * torch.randn(x.shape[:-1], generator=gen, device=dev)
    mask = torch.ones_like(target)
    theta = torch.as_tensor(WS.init_params(3), device=dev)
    grad = torch.empty_like(theta)
    out = {}
    for name, fn in (("fp32", tt.tt_net_loss_grad), ("tensor_cores", tt.tt_net_loss_grad_tc)):
        for _ in range(warmup):
            fn(ctx, theta, x, target, mask, grad)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn(ctx, theta, x, target, mask, grad)
        e1.record()
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) / steps
    ctx.close()
    return {"batch": "%d grids of 81^3" % len(src), "fp32_ms_per_step": out["fp32"],
            "tensor_core_ms_per_step": out["tensor_cores"],
            "speedup": out["fp32"] / out["tensor_cores"],
            "note": "loss and gradient of the warm-start network; tensor cores: the forward, "
                    "input-gradient and weight-gradient convolutions on tcgen05 (BF16 operands, "
                    "FP32 accumulation)"}


def godunov_leg(args, gp, world):
    """The same step with the Godunov local solver for anisotropic models (opts.scheme = 2)
    in the forward sweep instead of Lax-Friedrichs: a different first-order discretisation of
    the same equation (its fixed point differs at O(h); parity is against the oracle's
    solver of the same scheme). Launch configuration autotuned for the scheme."""
    torch, tt = gp.torch, gp.tt
    if gp.plan is not None:
        gp.plan.close()
        gp.plan = None
    gp.opts.init = tt.TT_INIT_ABOVE
    gp.opts.scheme = 2
    tuned = None
    if args.autotune and args.schedule == 0:
        ms = tt.tt_autotune(gp.ctx, gp.model, gp.w.src, gp.opts)
        tuned = {"ms_per_iteration": {k: round(v, 3) for k, v in ms.items()},
                 "chosen": {"fwd_groups": gp.opts.fwd_groups}}
    if args.plan:
        gp.use_plan()
    for _ in range(args.warmup):
        gp.step()
    gp.iters.clear()
    dist_barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        gp.step()
    e1.record()
    torch.cuda.synchronize()
    ms = dist_max(e0.elapsed_time(e1) / args.steps, world)
    itf = np.concatenate([s[0] for s in gp.iters])
    ita = np.concatenate([s[1] for s in gp.iters])
    fwd = [s[2] for s in gp.iters]
    adj = [s[3] for s in gp.iters]
    hbm, _ = peaks()
    f_ms = float(np.mean([s["sweep_ms"] for s in fwd]))
    fwd_kernel = hbm_kernel(f_ms, float(np.mean([s["node_updates"] for s in fwd])),
                            float(np.mean([s["node_sweeps"] for s in fwd])),
                            FWD_BYTES_PER_UPDATE, FWD_BYTES_PER_NODE_SWEEP, hbm)
    fwd_kernel["kernel"] = "fwd_sweep_kernel<float, unsigned, 0, 2>"
    # The same forward from tau = 1 (opts.init = 0), for comparison with the start from above.
    o1 = tt.default_opts(tt.TT_F32, scheme=2, fwd_groups=gp.opts.fwd_groups)
    it1 = tt.tt_forward(gp.ctx, gp.model, gp.w.src, gp.tau, None, o1)
    ms1 = tt.tt_get_stats(gp.ctx, tt.TT_STATS_FORWARD)["sweep_ms"]
    return {"value": world * gp.w.n_src / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "forward_kernel": fwd_kernel,
            "scheme": "Godunov upwind for anisotropic models (opts.scheme = 2)",
            "start": "from above (opts.init = 3)",
            "iters_fwd_mean": float(itf.mean()), "iters_fwd_max": int(itf.max()),
            "iters_adj_mean": float(ita.mean()),
            "forward_ms": float(np.mean([s["sweep_ms"] for s in fwd])),
            "adjoint_ms": float(np.mean([s["sweep_ms"] for s in adj])),
            "start_from_one": {"iters_fwd_mean": float(it1.mean()),
                               "iters_fwd_max": int(it1.max()), "forward_ms": ms1},
            "ideal_start_bound": start_bound(gp, scheme=2, cold_init=tt.TT_INIT_ABOVE,
                                             above=True),
            "autotune": tuned}


def refill_leg(args, dev, world, slots, gp):
    """Forward sweeps of a workload larger than one batch (args.refill_sources sources on
    the same grid) with `slots` sources in flight: one retire-and-refill launch against
    consecutive resident batches of `slots` sources (what a caller does without refill)."""
    torch, tt = gp.torch, gp.tt
    big = I.anisotropic_batch(seed=I.SEED_BASE + 2 + 100, n_src=args.refill_sources)
    f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)
    model = (f32(big.s), f32(big.xi), f32(big.eta))
    ctx = tt.tt_ctx_create(big.grid.as_dict())
    tau = torch.empty(big.grid.shape + (big.n_src,), dtype=torch.float32, device=dev)
    o_refill = tt.default_opts(tt.TT_F32, fwd_slots=slots, fwd_groups=gp.opts.fwd_groups)
    o_batch = tt.default_opts(tt.TT_F32, fwd_groups=gp.opts.fwd_groups)
    starts = list(range(0, big.n_src, slots))
    taus = [torch.empty(big.grid.shape + (min(slots, big.n_src - s0),), dtype=torch.float32,
                        device=dev) for s0 in starts]

    def refill():
        return tt.tt_forward(ctx, model, big.src, tau, None, o_refill)

    def batches():
        return np.concatenate([tt.tt_forward(ctx, model, big.src[s0:s0 + slots], tb, None,
                                             o_batch) for s0, tb in zip(starts, taus)])

    out = {}
    for name, fn in (("refill", refill), ("batches", batches)):
        fn()                                  # warm-up: allocation
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        it = fn()
        e1.record()
        torch.cuda.synchronize()
        out[name] = (dist_max(e0.elapsed_time(e1), world), it)
    ctx.close()
    return {"sources": big.n_src, "slots": slots, "forward_ms_refill": out["refill"][0],
            "forward_ms_batches": out["batches"][0],
            "speedup": out["batches"][0] / out["refill"][0],
            "iters_fwd_mean": float(out["refill"][1].mean()),
            "iters_fwd_max": int(out["refill"][1].max()),
            "same_iterations": bool(np.array_equal(out["refill"][1], out["batches"][1])),
            "note": "forward only; refill = one launch with %d slots; batches = %d resident "
                    "launches of up to %d sources" % (slots, len(starts), slots)}


def unbatched_leg(args, w, dev, world):
    """The plain FP32 path one source at a time (the same step on a one-source batch) for
    the first args.unbatched sources of the workload."""
    torch = __import__("torch")
    ms = []
    for b in range(min(args.unbatched, w.n_src)):
        one = GpuPath(w.subset([b]), dev)
        one.use_plan()
        one.step()                     # warm-up (allocation, graph upload)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        one.step()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        one.plan.close()
        one.ctx.close()
    ms_mean = dist_max(float(np.mean(ms)), world)
    return {"value": world / (ms_mean * 1e-3), "unit": UNIT, "ms_per_solve": ms_mean,
            "sources": len(ms), "note": "one source per step, same kernels and graph"}


def start_bound(gp, rel=3e-3, scheme=0, cold_init=0, above=False):
    """How many sweeps an ideal warm start could save: the forward solve started from the
    converged tau of a solve from opts.init = cold_init times (1 + rel * f), f a smooth field
    of unit amplitude (one sinusoid per axis with a phase per source; |f| when above, so that
    the start lies above the solution), the same tolerance, against that solve.
    LF sweeping contracts the error at a roughly fixed rate and its slow last phase sits
    next to the downstream faces, so the count depends little on the starting error. The
    Godunov update converges fast from any start above the solution (opts.init = 3), which
    leaves an ideal predictor little to save."""
    torch, tt = gp.torch, gp.tt
    g = gp.w.grid
    B = gp.w.n_src
    o = tt.default_opts(tt.TT_F32, fwd_groups=gp.opts.fwd_groups, scheme=scheme, init=cold_init)
    tau = torch.empty(g.shape + (B,), dtype=torch.float32, device=gp.dev)
    it_cold = tt.tt_forward(gp.ctx, gp.model, gp.w.src, tau, None, o)
    ms_cold = tt.tt_get_stats(gp.ctx, tt.TT_STATS_FORWARD)["sweep_ms"]
    ax = [torch.linspace(0, np.pi, n, device=gp.dev) for n in g.shape]
    ph = torch.linspace(0, 2 * np.pi, B, device=gp.dev)
    f = (torch.sin(ax[0][:, None, None, None] + ph) * torch.sin(2 * ax[1][None, :, None, None] + ph)
         * torch.sin(3 * ax[2][None, None, :, None] + ph))
    tau.mul_(1.0 + rel * (f.abs() if above else f))
    del f
    o.init = tt.TT_INIT_GIVEN
    it_warm = tt.tt_forward(gp.ctx, gp.model, gp.w.src, tau, None, o)
    ms_warm = tt.tt_get_stats(gp.ctx, tt.TT_STATS_FORWARD)["sweep_ms"]
    return {"relative_start_error": rel, "iters_fwd_mean_cold": float(it_cold.mean()),
            "iters_fwd_max_cold": int(it_cold.max()), "iters_fwd_mean": float(it_warm.mean()),
            "iters_fwd_max": int(it_warm.max()), "forward_ms_cold": ms_cold,
            "forward_ms": ms_warm,
            "note": "forward solve started from the converged tau with a smooth relative error "
                    "of %g%s (an ideal predictor's bound), against the start opts.init = %d"
                    % (rel, " above the solution" if above else "", cold_init)}


def warm_leg(args, gp, world):
    """The same step with the learned warm start (opts.init = 2): the forward sweep starts
    from the network's tau and still runs to the same tolerance."""
    import json as _json
    torch, tt = gp.torch, gp.tt
    z = np.load(args.warm_start)
    meta = _json.loads(str(z["summary"]))
    stride = int(meta.get("stride", 1))
    theta = torch.as_tensor(z["theta"], device=gp.dev)
    tt.tt_net_set_stride(gp.ctx, stride)
    tt.tt_net_set_weights(gp.ctx, theta)
    if gp.plan is not None:
        gp.plan.close()
    gp.opts.init = 2
    if args.plan:
        gp.use_plan()
    for _ in range(args.warmup):
        gp.step()
    gp.iters.clear()
    dist_barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        gp.step()
    e1.record()
    torch.cuda.synchronize()
    ms = dist_max(e0.elapsed_time(e1) / args.steps, world)
    itf = np.concatenate([s[0] for s in gp.iters])
    fwd = [s[2] for s in gp.iters]
    inf_ms = float(np.mean([s["warm_ms"] for s in fwd]))
    from paper_2412_00031_gb300.warmstart import net_shape
    fwd_it_ms = float(np.mean([s["sweep_ms"] / max(1, s["iters_max"]) for s in fwd]))
    sweep_ms = float(np.mean([s["sweep_ms"] for s in fwd]))
    hbm, _ = peaks()
    sweep = hbm_kernel(sweep_ms, float(np.mean([s["node_updates"] for s in fwd])),
                       float(np.mean([s["node_sweeps"] for s in fwd])), FWD_BYTES_PER_UPDATE,
                       FWD_BYTES_PER_NODE_SWEEP, hbm)
    return {"value": world * gp.w.n_src / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "iters_fwd_mean": float(itf.mean()), "iters_fwd_max": int(itf.max()),
            "inference_ms": inf_ms, "sweep_ms": sweep_ms,
            "network_grid": list(net_shape(gp.w.grid.shape, stride)),
            "inference_in_forward_iterations": inf_ms / fwd_it_ms,
            "inference_roofline": net_roofline(net_shape(gp.w.grid.shape, stride), gp.w.n_src,
                                               inf_ms),
            "ideal_start_bound": start_bound(gp),
            "forward_kernel": sweep,
            "inference": "3x3x3 convolutions, all four layers on the tensor cores (tcgen05, BF16 "
                         "operands, FP32 accumulation in tensor memory)%s"
                         % ("" if stride == 1 else ", on every other node along each axis, "
                            "the prediction interpolated trilinearly to the others"),
            "weights": "%s: trained on %d forward solves on %s random-field models, held-out "
                       "sweeps %.1f -> %.1f" % (os.path.basename(args.warm_start),
                                                meta["solves_train"], "x".join(map(str, meta["grid"])),
                                                meta["held_out_sweeps_cold"],
                                                meta["held_out_sweeps_warm"])}


# Executed tensor-core FLOPs per 128-row tile of the four layers (M = 128, N = 3 x output
# channels, K = 16 per MMA): layer 1 one K step per (di, dj), layers 2-3 two, layer 4 two
# with N = 48), and the useful FLOPs of the network per node (unpadded channels).
NET_TILE_FLOP = 9 * 2 * 128 * 16 * (96 * 1 + 96 * 2 + 96 * 2 + 48 * 2)
NET_TILE_ROWS = 126
NET_USEFUL_FLOP_PER_NODE = 2 * 27 * (6 * 32 + 32 * 32 + 32 * 32 + 32 * 1)


def net_roofline(shape, n_grids, ms):
    """Tensor roofline of the warm start's inference over n_grids grids in ms (the whole
    inference: features, packing, four tcgen05 convolution layers, the start of tau):
    executed MMA FLOPs and useful network FLOPs against the dense BF16 peak."""
    nodes = int(np.prod(shape))
    rows = shape[0] * (shape[1] + 1) * (shape[2] + 1)
    tiles = -(-rows // NET_TILE_ROWS) * n_grids
    executed = NET_TILE_FLOP * tiles / (ms * 1e-3) / 1e12
    useful = NET_USEFUL_FLOP_PER_NODE * nodes * n_grids / (ms * 1e-3) / 1e12
    peak, src = bf16_peak()
    return {"bound": "tensor", "kernel": "conv3d_tc_kernel (4 layers)", "achieved": executed,
            "useful_tflops": useful, "peak": peak, "unit": "TFLOP/s", "frac": executed / peak,
            "frac_useful": useful / peak, "peak_source": src}


def infer_only(args):
    """Times the warm start's inference alone (tt_net_infer) on args.infer_only sources of the
    benchmark grid, features computed beforehand; one JSON line."""
    import torch
    import paper_2412_00031_gb300 as tt
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    nb = args.infer_only
    w = I.anisotropic_batch(seed=rank_seed(0), n_src=nb)
    g = w.grid
    ctx = tt.tt_ctx_create(g.as_dict())
    z = np.load(args.warm_start)
    stride = int(json.loads(str(z["summary"])).get("stride", 1))
    from paper_2412_00031_gb300.warmstart import net_shape
    shape = net_shape(g.shape, stride)
    tt.tt_net_set_stride(ctx, stride)
    tt.tt_net_set_weights(ctx, torch.as_tensor(z["theta"], device=dev))
    f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)
    x = torch.empty((nb,) + shape + (6,), dtype=torch.float32, device=dev)
    tt.tt_net_features(ctx, (f32(w.s), f32(w.xi), f32(w.eta)), w.src, x)
    y = torch.empty(x.shape[:-1], dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        tt.tt_net_infer(ctx, x, y)
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        tt.tt_net_infer(ctx, x, y)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ctx.close()
    ms = float(np.median(times))
    roof = net_roofline(shape, nb, ms)
    roof["note"] = "executed MMA FLOPs (padded channels, 126 of 128 rows per tile)"
    return {"metric": "warm-start inference throughput", "value": nb / (ms * 1e-3),
            "unit": "source-grids/s", "ms": ms, "grids": nb, "grid": list(g.shape),
            "network_grid": list(shape),
            "useful_tflops": roof["useful_tflops"], "roofline": roof,
            "gpu_launches_per_call": 5}


def inversion_batches(tt, ctx, w, batch, dev):
    """Observations of the 201 x 201 x 101 inversion workload from FP32 solves in its true
    model (tt_forward + tt_misfit's receiver times) plus seeded Gaussian noise, per-batch
    data (absolute times, common-source pairs as differences of the noisy picks), and the
    common-receiver pairs of all sources closer than meta["cr_deg"], across batches (a
    CrData over all sources, or None)."""
    import torch
    g = w.grid
    true = tuple(torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)
                 for a in w.meta["true"])
    rng = np.random.default_rng(w.meta["noise_seed"])
    out = []
    picks, seen_all = [], []
    for b0 in range(0, w.n_src, batch):
        idx = list(range(b0, min(b0 + batch, w.n_src)))
        sub = w.subset(idx)
        B, nr = len(idx), len(w.rec)
        d0 = tt.DeviceData.from_workload(sub, device=dev)
        tau = torch.empty(g.shape + (B,), dtype=torch.float32, device=dev)
        T = torch.empty_like(tau)
        tt.tt_forward(ctx, true, sub.src, tau, T)
        Tr = torch.empty((B, nr), dtype=torch.float64, device=dev)
        R = torch.empty_like(Tr)
        tt.tt_misfit(ctx, T, d0, Tr, None, R)
        del tau, T
        pick = Tr.cpu().numpy() + w.meta["noise_s"] * rng.standard_normal((B, nr))
        abs_tobs = np.concatenate([pick[n, sub.abs_rec[sub.abs_off[n]:sub.abs_off[n + 1]]]
                                   for n in range(B)])
        cs_n = np.repeat(np.arange(B), np.diff(sub.cs_off))
        cs_dtobs = pick[cs_n, sub.cs_m] - pick[cs_n, sub.cs_i]
        data = tt.DeviceData(w.rec, sub.abs_off, sub.abs_rec, abs_tobs, sub.abs_w, sub.cs_off,
                             sub.cs_m, sub.cs_i, cs_dtobs, sub.cs_w, device=dev)
        seen = np.zeros((B, nr), dtype=bool)
        for n in range(B):
            seen[n, sub.abs_rec[sub.abs_off[n]:sub.abs_off[n + 1]]] = True
        picks.append(pick)
        seen_all.append(seen)
        out.append((sub.src, data, None))
    pick, seen = np.concatenate(picks), np.concatenate(seen_all)
    pairs = []
    ep = w.src[:, 1:]
    for a in range(w.n_src):
        close = np.nonzero(np.hypot(*(ep[a + 1:] - ep[a]).T) < w.meta["cr_deg"])[0] + a + 1
        for j in close:
            for m in np.nonzero(seen[a] & seen[j])[0]:
                pairs.append((a, j, m, pick[a, m] - pick[j, m], 1.0))
    cr_all = tt.CrData(w.n_src, len(w.rec), pairs, gamma=1.0, device=dev) if pairs else None
    return out, cr_all


def inversion_leg(args):
    """Times the inversion loop (step 4 of Sec. 2 with Eqs. 11-19, absolute, common-source and
    common-receiver data) on the 201 x 201 x 101 workload, args.n_src sources in batches of
    args.inv_batch, 5 offset 11^3 inversion grids, args.inversion step attempts. One JSON
    line: wall time per step attempt (each attempt is one evaluation: forward, misfit and two
    adjoints of every source, kernels, kernel density, then the direction)."""
    import torch
    import paper_2412_00031_gb300 as tt
    from paper_2412_00031_gb300.invert import Inversion
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = I.inversion_201(n_src=args.inv_sources)
    g = w.grid
    ctx = tt.tt_ctx_create(g.as_dict())
    t0 = time.perf_counter()
    batches, cr_all = inversion_batches(tt, ctx, w, args.inv_batch, dev)
    t_obs = time.perf_counter() - t0
    model = tuple(torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)
                  for a in (w.s, w.xi, w.eta))
    opts = tt.default_opts(tt.TT_F32, scheme=args.inv_scheme)
    inv = Inversion(ctx, model, None, None, g.shape, tt.mgrid(11, 11, 11, 5), opts=opts,
                    batches=batches, cr_all=cr_all)
    times, hist = [], []
    step, chi = 0.02, None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    chi = inv.evaluate()
    inv.direction()
    torch.cuda.synchronize()
    times.append(time.perf_counter() - t0)
    hist.append((chi, step, True))
    its = [float(np.mean(np.concatenate([b.iters_fwd for b in inv.batches])))]
    for _ in range(args.inversion):
        t0 = time.perf_counter()
        saved = [a.clone() for a in model]
        tt.tt_model_update(ctx, model, *inv.D, step)
        new = inv.evaluate()
        if new < chi:
            chi = new
            inv.direction()
            hist.append((new, step, True))
        else:
            for a, b in zip(model, saved):
                a.copy_(b)
            hist.append((new, step, False))
            step *= 0.5
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        its.append(float(np.mean(np.concatenate([b.iters_fwd for b in inv.batches]))))
    ctx.close()
    n_cr = cr_all.n_entries if cr_all is not None else 0
    return {"metric": "inversion step time at 201x201x101 (depth x lat x lon), %d sources"
                      % w.n_src, "value": float(np.mean(times[1:])) if len(times) > 1 else times[0],
            "unit": "s per step attempt", "higher_is_better": False,
            "first_evaluation_s": times[0], "step_s": times[1:], "observations_s": t_obs,
            "chi": [h[0] for h in hist], "step": [h[1] for h in hist],
            "accepted": [h[2] for h in hist], "iters_fwd_mean": its,
            "config": {"workload": "inversion 201x201x101, %d sources in batches of %d, "
                                   "400 stations, 5 offset 11^3 inversion grids" % (w.n_src, args.inv_batch),
                       "forward_scheme": ["Lax-Friedrichs", "Godunov (isotropic)",
                                          "Godunov (anisotropic)"][args.inv_scheme],
                       "abs_records": int(len(w.abs_rec)), "cs_pairs": int(len(w.cs_m)),
                       "cr_entries": int(n_cr), "cr_pairs": "across all sources (joined tables)",
                       "precision": "fp32 sweeps, fp64 misfit and kernels"},
            "data": "synthetic: observations from FP32 solves in the true checkerboard model + "
                    "N(0, 0.05 s)"}


def tele_leg(args):
    """Times teleseismic events on the benchmark's 121 x 161 x 161 region: args.tele events
    8-20 deg away at 30-300 km depth in a 1-D model (Vp 5.8 -> 8.8 km/s over 400 km), the
    region's model the benchmark's anisotropic one. One JSON line: the 2-D solves, the
    region's face data and the region's solve (Lax-Friedrichs with fixed faces), each timed
    with CUDA events after a warm-up run."""
    import torch
    import paper_2412_00031_gb300 as tt
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = I.anisotropic_batch(n_src=1)
    g = w.grid
    rng = np.random.default_rng(20241205)
    n_ev = args.tele
    dist = rng.uniform(8.0, 20.0, n_ev)
    az = rng.uniform(0.0, 2 * np.pi, n_ev)
    lat0, lon0 = 0.5 * (g.lat_min_deg + g.lat_max_deg), 0.5 * (g.lon_min_deg + g.lon_max_deg)
    events = np.stack([rng.uniform(30.0, 300.0, n_ev), lat0 + dist * np.cos(az),
                       lon0 + dist * np.sin(az)], 1)
    RE, n_r, n_d, dmax = g.earth_radius_km, 201, 401, 25.0
    r = np.linspace(RE - 400.0, RE, n_r)
    s_r = torch.as_tensor(1.0 / (5.8 + 3.0 * (RE - r) / 400.0), device=dev)
    ctx = tt.tt_ctx_create(g.as_dict())
    f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)
    model = (f32(w.s), f32(w.xi), f32(w.eta))
    T2 = torch.empty((n_ev, n_r, n_d), dtype=torch.float64, device=dev)
    T = torch.empty(g.shape + (n_ev,), dtype=torch.float32, device=dev)
    T2f = torch.empty((n_ev, n_r, n_d), dtype=torch.float32, device=dev)

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    tele_opts = tt.default_opts(tt.TT_F32, tol_fwd=3e-5)
    res = {}
    for rep in range(2):                         # the first run is the warm-up
        ms2, it2 = timed(lambda: tt.tt_tele2d(ctx, s_r, RE - 400.0, RE, dmax, RE - events[:, 0],
                                              T2, tol=1e-10))
        T2f.copy_(T2)
        msf, _ = timed(lambda: tt.tt_tele_region_times(ctx, T2f, RE - 400.0, RE, dmax, events, T))
        # FP32 resolves T ~ 100-250 s to ~1.5e-5 s: the tolerance is a few of those units
        ms3, it3 = timed(lambda: tt.tt_forward_tele(ctx, model, T, tele_opts))
        res = {"tele2d_ms": ms2, "region_times_ms": msf, "region_solve_ms": ms3,
               "iters_2d_mean": float(np.mean(it2)), "iters_3d_mean": float(np.mean(it3)),
               "iters_3d_max": int(np.max(it3))}
    ctx.close()
    total = res["tele2d_ms"] + res["region_times_ms"] + res["region_solve_ms"]
    return {"metric": "teleseismic events per second on 1 GB300 at 121x161x161",
            "value": n_ev / (total * 1e-3), "unit": "events/s", "events": n_ev, **res,
            "config": {"workload": "%d teleseismic events, 8-20 deg, 30-300 km deep; 2-D grid "
                                   "%dx%d over 400 km x %g deg (FP64); region 121x161x161 "
                                   "anisotropic (FP32)" % (n_ev, n_r, n_d, dmax)},
            "tol_fwd_region_s": 3e-5,
            "note": "region solve: one persistent launch of the node-hyperplane sweep (Lax-"
                    "Friedrichs on T, faces fixed, FP32 arithmetic, convergence on the device)"}


# ----------------------------------------------------------------------------- CPU oracle

def oracle_sample(w, n_threads, n_src_sample, sweeps=1):
    """Times the FP64 oracle on the host cores: each thread runs `sweeps` forward sweeps and
    `sweeps` adjoint sweeps of one source of the workload. Returns seconds per forward and
    adjoint (node, source) update, per thread, and the threads used."""
    import oracle as O
    g = w.grid.as_dict()
    O.lib()
    srcs = list(range(min(n_src_sample, w.n_src)))
    n_int = (w.grid.n_r - 2) * (w.grid.n_t - 2) * (w.grid.n_p - 2)
    n_all = w.grid.n_nodes
    T0 = O.T0(g, w.s, w.xi, w.eta, w.src[0])[0]
    R = np.zeros(len(w.rec))
    d = w.source_data(0)
    R[d["abs_rec"]] = 0.1
    times = {}

    def run(kind):
        def work(b):
            if kind == "fwd":
                O.forward_sweeps(g, w.s, w.xi, w.eta, w.src[b], sweeps)
            else:
                O.adjoint_sweeps(g, T0, w.xi, w.eta, w.src[b], w.rec, R, sweeps)
        ths = [threading.Thread(target=work, args=(b,)) for b in srcs[:n_threads]]
        t0 = time.perf_counter()
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        times[kind] = time.perf_counter() - t0

    run("fwd")
    run("adj")
    nth = min(n_threads, len(srcs))
    t_fu = times["fwd"] / (sweeps * n_int)   # wall per update per thread (threads in parallel)
    t_au = times["adj"] / (sweeps * n_all)
    return t_fu, t_au, nth, times


def cpu_baseline(w, iters_f, iters_a, cores, source="the GPU run's means"):
    t_fu, t_au, nth, times = oracle_sample(w, cores, cores)
    n_int = (w.grid.n_r - 2) * (w.grid.n_t - 2) * (w.grid.n_p - 2)
    per_solve = 8 * n_int * iters_f * t_fu + 8 * w.grid.n_nodes * iters_a * t_au
    value = nth / per_solve
    return {"value": value, "unit": UNIT, "cores": nth, "kind": "oracle",
            "sample": "FP64 oracle, %d threads each running 1 forward and 1 adjoint sweep of "
                      "one source on the 121x161x161 grid (%.1f s + %.1f s wall); scaled to a "
                      "solve with %.1f forward and %.1f adjoint iterations (%s)"
                      % (nth, times["fwd"], times["adj"], iters_f, iters_a, source)}


def reference_arm(args):
    """The oracle as the reference implementation: each step is a bounded sample."""
    w = I.anisotropic_batch(n_src=args.n_src)
    cores = os.cpu_count() or 1
    # iteration counts: the FP32 Lax-Friedrichs sweeps of this workload converge in these
    # mean counts (measured by the GPU arm); the oracle needs at least as many at its FP64
    # tolerance
    iters_f, iters_a = args.ref_iters_fwd, args.ref_iters_adj
    vals, walls = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(w, iters_f, iters_a, cores,
                          "the mean counts the GPU arm measures on this workload")
        walls.append(time.perf_counter() - t0)
        vals.append(cb["value"])
    value = float(np.mean(vals))
    cb["value"] = value
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * np.mean(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, 1), "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ----------------------------------------------------------------------------- distributed

# One process per GPU. Sources are independent, so each rank solves its own batch (seeded by
# its rank) and nothing crosses ranks on the data path; the only collectives are the
# barriers around the timed region and the max of the per-rank times (weak scaling).

def dist_init():
    """Joins the process group under torchrun (NCCL with GPUs, gloo without)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def dist_max(x, world):
    """The maximum of x over the ranks (every rank gets it)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(rank):
    """Seed of a rank's batch: every rank solves different sources of the same workload."""
    return I.SEED_BASE + 2 + rank


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-src", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="profiling runs: skip the e2e leg")
    ap.add_argument("--max-iter-fwd", type=int, default=0, help="profiling runs only")
    ap.add_argument("--max-iter-adj", type=int, default=0, help="profiling runs only")
    ap.add_argument("--plan", type=int, default=1,
                    help="1: replay the step as one captured CUDA graph (tt_plan); 0: the four "
                         "individual calls")
    ap.add_argument("--warm-start", default=os.path.join(ROOT, "paper_2412_00031_gb300",
                                                      "warmstart_81_s2.npz"),
                    help="weights of the warm-start network; '' skips the warm-started leg")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1: pick the forward launch configuration with tt_autotune first")
    ap.add_argument("--refill-sources", type=int, default=768,
                    help="sources of the retire-and-refill line (forward only; 0 skips it)")
    ap.add_argument("--unbatched", type=int, default=2,
                    help="sources timed one per step for the unbatched line (0 skips it)")
    ap.add_argument("--launch-blocks", type=int, default=0,
                    help="profiling runs: cap on the blocks of a persistent launch")
    ap.add_argument("--adj-chunk", type=int, default=0,
                    help="adjoint sources per launch (tt_opts.adj_chunk; 0 = automatic)")
    ap.add_argument("--schedule", type=int, default=0,
                    help="forward sweep schedule (tt_opts.sweep_schedule; 0 = automatic)")
    ap.add_argument("--ref-iters-fwd", type=float, default=63.7,
                    help="reference arm: forward iterations per solve (the GPU arm's mean)")
    ap.add_argument("--ref-iters-adj", type=float, default=5.1,
                    help="reference arm: adjoint iterations per solve (the GPU arm's mean)")
    ap.add_argument("--infer-only", type=int, default=0,
                    help="time only the warm start's inference on this many sources")
    ap.add_argument("--scheme", type=int, default=0,
                    help="profiling runs: forward local solver of the main step (tt_opts.scheme)")
    ap.add_argument("--train-timing", type=int, default=1,
                    help="time a training step of the warm-start network (FP32 and tensor cores)")
    ap.add_argument("--godunov", type=int, default=1,
                    help="also time the step with the anisotropic Godunov solver (a leg)")
    ap.add_argument("--inversion", type=int, default=0,
                    help="time this many step attempts of the inversion loop on the "
                         "201x201x101 workload instead of the benchmark step")
    ap.add_argument("--inv-sources", type=int, default=1024)
    ap.add_argument("--inv-batch", type=int, default=256)
    ap.add_argument("--tele", type=int, default=0,
                    help="time this many teleseismic events on the benchmark region instead")
    ap.add_argument("--inv-scheme", type=int, default=0,
                    help="forward local solver of the inversion loop (tt_opts.scheme)")
    args = ap.parse_args()
    if args.infer_only > 0:
        print(json.dumps(infer_only(args)))
        return
    if args.inversion > 0:
        print(json.dumps(inversion_leg(args)))
        return
    if args.tele > 0:
        print(json.dumps(tele_leg(args)))
        return
    rank, world = dist_init()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(reference_arm(args)))
        return
    result, w, (itf, ita) = gpu_arm(args, rank, world)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline(w, itf, ita, os.cpu_count() or 1)
        print(json.dumps(result))


if __name__ == "__main__":
    main()
