"""Host logic of bench.py that needs no GPU: the DRAM traffic taken from the committed ncu
summary (bytes per update scaled to a launch, and null once the kernel source differs from
the one profiled), the kernel source digest, and the workload description."""
import os
import re

import bench
import tt_inputs as I


def _profile():
    path = os.path.join(bench.ROOT, "profiles", "fwd_sweep_kernel_anisotropic.md")
    text = open(path).read()
    digest = re.search(r"kernel source digest:\s*`?([0-9a-f]{16})", text).group(1)
    per_update = float(re.search(r"dram bytes per node update:\s*([0-9.]+)", text).group(1))
    return digest, per_update


def test_traffic_scales_the_profiled_bytes_per_update():
    digest, per_update = _profile()
    assert bench.profiled_traffic(digest, 1e9) == per_update * 1e9


def test_traffic_is_null_for_other_kernel_source():
    digest, _ = _profile()
    other = "0" * 16 if digest != "0" * 16 else "1" * 16
    assert bench.profiled_traffic(other, 1e9) is None


def test_kernel_source_digest_is_stable_hex():
    d = bench.kernel_source_digest()
    assert re.fullmatch(r"[0-9a-f]{16}", d)
    assert d == bench.kernel_source_digest()


def test_workload_config_names_the_benchmark_workload():
    w = I.anisotropic_batch(n_src=4, shape=(9, 11, 11))
    c = bench.workload_config(w, 2)
    assert c["workload"].startswith("anisotropic batch 9x11x11")
    assert c["grid"] == [9, 11, 11] and c["n_src_per_gpu"] == 4
    assert c["abs_records"] == len(w.abs_rec) and c["cs_pairs"] == len(w.cs_m)
    assert "2 GPU" in c["parallelism"]
