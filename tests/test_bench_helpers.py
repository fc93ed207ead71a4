"""Host logic of bench.py's measurement helpers (no GPU needed)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_ncu_traffic_gated_by_kernel_source(tmp_path, monkeypatch):
    """Traffic counters are used only while the kernel source they were taken
    on is unchanged."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.kernel_source_hash()
    (prof / "ncu_traffic.txt").write_text(f"# comment\nsweep_fp64 {h} 123\nsweep_fp32_acc 0000000000000000 456\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.ncu_traffic("sweep_fp64") == 123
    assert bench.ncu_traffic("sweep_fp32_acc") is None  # taken on another source
    assert bench.ncu_traffic("sweep_fp32") is None  # not captured


def test_clock_summary(tmp_path):
    c = bench.Clocks(0)
    c.proc = object()  # as if the sampler had run
    c.path = str(tmp_path / "clocks.csv")
    rows = ["0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    open(c.path, "w").write("\n".join(rows) + "\n")
    s = c.summary()
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_unitarity_helper():
    rng = np.random.default_rng(0)
    Z = rng.normal(size=(500, 3, 3)) + 1j * rng.normal(size=(500, 3, 3))
    Q, R = np.linalg.qr(Z)
    Q = Q * (np.diagonal(R, axis1=1, axis2=2) / np.abs(np.diagonal(R, axis1=1, axis2=2)))[:, None, :]
    Q = Q / np.linalg.det(Q)[:, None, None] ** (1 / 3)
    umax, umean, dmax = bench.unitarity(Q)
    assert umax < 1e-14 and dmax < 1e-14
    Q[7, 1, 2] += 1e-6
    umax, umean, dmax = bench.unitarity(Q)
    assert 5e-7 < umax < 3e-6 and umean < umax


def test_serving_stream_is_rate_independent():
    """The Poisson stream's jobs (lattice, gauge, seed) do not depend on the
    rate; only the arrival times scale with 1/rate."""
    from paper_1212_5221_gb300 import inputs

    a = inputs.poisson_jobs(50, 1.0, 4)
    b = inputs.poisson_jobs(50, 0.25, 4)
    assert [(j["dims"], j["gauge"], j["seed"]) for j in a] == [(j["dims"], j["gauge"], j["seed"]) for j in b]
    assert np.allclose([4 * j["arrival"] for j in a], [j["arrival"] for j in b])
    lat = {j["dims"] for j in inputs.poisson_jobs(400, 1.0, 4)}
    assert lat == {(16, 16, 16, 16), (48, 24, 24, 24), (32, 32, 32, 32), (96, 48, 48, 48)}


def test_bench_help_without_gpu():
    """The command line parses without a GPU (--help)."""
    import subprocess

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and "--serving" in r.stdout and "--study" in r.stdout and "--slab" in r.stdout
