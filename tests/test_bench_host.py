"""Host logic of bench.py on the CPU: the clock sampler's parsing (against a fake nvidia-smi),
the reference arm under two ranks, and the roofline arithmetic."""
import json
import os
import stat
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

FAKE_SMI = """#!/bin/sh
printf '0, 1965, 2070, 910.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\\n'
printf '0, 1980, 2070, 1200.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active\\n'
printf '0, 1950, 2070, 1005.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\\n'
printf 'garbage line\\n'
exec sleep 30
"""


def test_clock_sampler_parses_nvidia_smi(tmp_path, monkeypatch):
    smi = tmp_path / "nvidia-smi"
    smi.write_text(FAKE_SMI)
    smi.chmod(smi.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    c = bench.ClockSampler(0)
    c.start()
    import time
    time.sleep(0.5)
    clk = c.stop()
    assert clk["sm_mhz"] == 1965.0 and clk["sm_max_mhz"] == 2070.0
    assert clk["reasons"] == ["sw_power_cap"] and clk["samples"] == 3
    assert clk["power_w_max"] == 1200.5


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))           # nothing to run
    c = bench.ClockSampler(0)
    c.start()
    clk = c.stop()
    assert clk["sm_mhz"] is None and clk["reasons"] == ["nvidia-smi unavailable"]


def _reference(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                           "--steps", "1", "--warmup", "3", "--cpu-sample", "128"],
                          capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)


def test_reference_arm_under_two_ranks():
    # only rank 0 runs the oracle and prints; the other rank exits 0 without work or output
    r1 = _reference({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert r1.returncode == 0 and not [ln for ln in r1.stdout.splitlines() if ln.startswith("{")]
    r0 = _reference({"WORLD_SIZE": "2", "RANK": "0", "LOCAL_RANK": "0"})
    assert r0.returncode == 0, r0.stderr[-2000:]
    lines = [ln for ln in r0.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["config"]["sample_n"] == 128


def test_emulated_update_roofline_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: ({"bf16_tflops": 1900.0}, "measured"))
    # 1e12 FP64 flops of update work in 100 ms: 10 TF/s algorithmic, 1050 TF/s executed on E4M3
    r = bench.zgemm_roofline(1e12, 100.0, 0.5)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s" and r["peak"] == pytest.approx(3800.0)
    assert r["algorithmic_fp64_tflops"] == pytest.approx(10.0)
    assert r["achieved"] == pytest.approx(1050.0) and r["frac"] == pytest.approx(1050.0 / 3800.0)
    assert r["update_share_of_step"] == pytest.approx(0.2)


def test_dfma_roofline_is_an_alu_peak(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: ({"sm_max_mhz": 2070.0}, "measured"))
    r = bench.fp64_roofline(1.2e12, 1000.0, 2.0)
    peak = 152 * 4 * 2070e6 / 1e12                       # 152 SMs x 2 DFMA per clock x 2.07 GHz
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(peak, rel=1e-4)
    assert r["achieved"] == pytest.approx(1.2) and r["frac"] == pytest.approx(1.2 / peak)


def test_accuracy_probe_products_against_dense():
    # bench.py's harness-side products with packed tiles (used by the factor backward-error
    # probe of the four-precision line), on the CPU against dense numpy, ragged n
    import numpy as np
    import torch

    import oracle
    n, b = 300, 128
    rng = np.random.default_rng(0)
    M = rng.standard_normal((n, n))
    S = M @ M.T + n * np.eye(n)
    nt = -(-n // b)
    N = nt * b
    Sp = np.eye(N)
    Sp[:n, :n] = S
    P = torch.from_numpy(oracle.pack_tiles(Sp, b).reshape(-1).copy())
    Lo = np.linalg.cholesky(Sp)
    Lp = torch.from_numpy(oracle.pack_tiles(np.tril(Lo) + np.triu(rng.standard_normal((N, N)), 1), b)
                          .reshape(-1).copy())              # garbage above the diagonal is ignored
    x = rng.standard_normal(n)
    xt = torch.from_numpy(x)
    assert np.allclose(bench.tiles_matvec(P, n, b, xt, "cpu", "sym").numpy(), S @ x, rtol=1e-12, atol=1e-10)
    L = Lo[:n, :n]
    assert np.allclose(bench.tiles_matvec(Lp, n, b, xt, "cpu", "L").numpy(), L @ x, rtol=1e-12, atol=1e-10)
    assert np.allclose(bench.tiles_matvec(Lp, n, b, xt, "cpu", "Lt").numpy(), L.T @ x, rtol=1e-12, atol=1e-10)
    # the probe: an exact factor gives FP64 rounding, a perturbed one its perturbation
    assert bench.factor_probe_berr(P, Lp, n, b, "cpu") < 1e-14
    Lq = Lo.copy()
    Lq[:n, :n] *= 1.0 + 1e-6
    Lqp = torch.from_numpy(oracle.pack_tiles(np.tril(Lq), b).reshape(-1).copy())
    assert 1e-6 < bench.factor_probe_berr(P, Lqp, n, b, "cpu") < 4e-6
