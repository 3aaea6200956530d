"""Host logic of bench.py on CPU: the roofline arithmetic of the local solve and the memory-bound passes, and the
clock sampler's parsing of nvidia-smi output (a stand-in nvidia-smi on PATH prints fixed samples)."""
import os
import stat
import time
import types

import pytest


def test_local_solve_roofline_counts_the_methods_148_bytes_per_voxel():
    import bench
    n = 128
    N3 = n ** 3
    wl = types.SimpleNamespace(n=n)
    ms, launches = 10.0, 100                       # 100 launches of 0.1 ms
    out = bench.roofline("newton", {"newton": (ms, launches)}, wl, N3, iters=100, solves=N3 * 100,
                         evals=N3 * 100, pk={"hbm_gbs": 6000.0}, pk_kind="measured", precision="mixed",
                         facs=0, reuse=True)
    hbm = out["resources"]["hbm"]
    # eps 6, eps_p 6, tau_c 12, sigma warm start 6 in, sigma 6 out; g0: the method's operands, no factor cache
    assert hbm["bytes_per_launch"] == 148 * N3
    assert hbm["minimal_operand_bytes_per_launch"] == 80 * N3          # eps_tr 6, sigma 6, tau_c 1, sigma 6; g0
    assert hbm["bytes_per_launch_with_factor_cache"] == 164 * N3       # + 21 stored factor words
    assert hbm["achieved"] == pytest.approx(148 * N3 / 1e-4 / 1e9)
    assert hbm["frac"] == pytest.approx(hbm["achieved"] / 6000.0)
    assert out["bound"] == "hbm" and out["frac"] == pytest.approx(hbm["frac"])
    # FP32 pipe: residual-only evaluations with tangent reuse, FP32 triangular solves
    alu = out["resources"]["alu"]
    assert alu["pipe"] == "fp32"
    assert alu["flops_fp32"] == bench.NEWTON_FLOPS_RESID * N3 * 100 + bench.NEWTON_FLOPS_SOLVE * N3 * 100
    # the exact Newton has the same algorithmic operands
    ex = bench.roofline("newton", {"newton": (ms, launches)}, wl, N3, 100, N3 * 100, N3 * 100, {"hbm_gbs": 6000.0},
                        "measured", "mixed", reuse=False)
    assert ex["resources"]["hbm"]["bytes_per_launch"] == 148 * N3


def test_stored_traffic_is_dropped_once_its_sources_change(tmp_path, monkeypatch):
    import bench
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.sources_sha(["k.cu"])
    table = {(1, "mixed", True): (123.0, sha)}
    assert bench.measured_traffic(table, (1, "mixed", True), ["k.cu"]) == 123.0
    src.write_text("kernel v2")
    assert bench.measured_traffic(table, (1, "mixed", True), ["k.cu"]) is None
    assert bench.measured_traffic(table, (2, "mixed", True), ["k.cu"]) is None


def test_iteration_classes_are_averaged_over_the_iterations_that_ran():
    """Iterations queued after convergence return at once: an iteration class is averaged over the iterations that
    ran (its brackets' total time over them), a per-increment class over its launches."""
    import bench
    assert bench.per_unit("fft_z_gamma", 128.0, 128, 113) == pytest.approx(128.0 / 1e3 / 113)
    assert bench.per_unit("newton", 10.0, 128, 113) == pytest.approx(10.0 / 1e3 / 113)
    assert bench.per_unit("state_update", 0.15, 1, 113) == pytest.approx(0.15 / 1e3)
    assert bench.per_unit("fft_z_gamma", 1.0, 16, None) == pytest.approx(1.0 / 1e3 / 16)
    m = bench.memory_kernels({"fft_y_fwd": (2.0, 128)}, types.SimpleNamespace(n=128), 128 ** 3, "mixed",
                             {"hbm_gbs": 5000.0}, iterations=100)
    assert m["fft_y_fwd"]["avg_us"] == 20.0


def test_fft_pass_bytes_follow_the_half_spectrum():
    import bench
    n, T = 128, 4
    H = (n // 2 + 1) / n
    assert bench.hbm_bytes_per_voxel("fft_xy_r2c", n, T) == pytest.approx((6 + 12 * H) * T)
    for k in ("fft_y_fwd", "fft_z_gamma", "fft_y_inv"):
        assert bench.hbm_bytes_per_voxel(k, n, T) == pytest.approx(24 * H * T)
    assert bench.hbm_bytes_per_voxel("fft_xy_c2r_update", n, T) == pytest.approx((12 * H + 12) * T)
    m = bench.memory_kernels({"fft_y_fwd": (2.0, 100)}, types.SimpleNamespace(n=n), n ** 3, "mixed",
                             {"hbm_gbs": 5000.0})
    gbs = 24 * H * T * n ** 3 / 20e-6 / 1e9
    assert m["fft_y_fwd"]["avg_us"] == 20.0 and m["fft_y_fwd"]["GB/s"] == pytest.approx(gbs, abs=0.05)


def test_clock_sampler_reads_median_clock_and_throttle_reasons(tmp_path, monkeypatch):
    import bench
    fake = tmp_path / "nvidia-smi"
    lines = ["0, 2070, 2070, 350.5, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 410.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage line"]
    fake.write_text("#!/bin/sh\n" + "".join(f"echo '{ln}'\n" for ln in lines) + "exec sleep 30\n")
    fake.chmod(fake.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    cs = bench.ClockSampler(0)
    cs.start()
    time.sleep(0.5)
    out = cs.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["power_w_max"] == 900.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))
    cs = bench.ClockSampler(0)
    cs.start()
    assert cs.stop()["reasons"] == ["nvidia-smi unavailable"]
