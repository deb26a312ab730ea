"""Host side of the benchmark: the CPU-baseline leg's chunked oracle pass and the accuracy measure
it reports for the timed run's output (CPU only; the device output is stood in for by a CPU tensor)."""
import numpy as np
import pytest
import torch

import bench
import oracle
import workloads
from workloads import designs


@pytest.fixture(scope="module")
def case():
    sos = designs.butter_lowpass(4, 0.2)
    x = workloads.normal_f32(5, 5000)
    y_ref = oracle.sosfilt(sos, x)
    return sos, x, y_ref


def test_chunked_pass_reports_float32_rounding_only(case):
    sos, x, y_ref = case
    y = torch.from_numpy(y_ref.astype(np.float32))
    base, acc = bench.cpu_baseline_leg(sos, x, y, chunk=1024)
    # the state carried between chunks makes the chunked oracle equal the one-pass one: the only
    # difference left is the float32 rounding of the stand-in output
    assert acc["max_rel_error"] < 1e-7
    assert acc["bound"] == 1e-4
    # against the oracle on float32-rounded coefficients the stand-in differs by that rounding
    y32 = oracle.sosfilt(np.asarray(sos, np.float32).astype(np.float64), x)
    assert acc["max_rel_error_vs_f32_coefficients"] == pytest.approx(oracle.rel_err(y.numpy(), y32), rel=1e-9)
    assert base["cores"] == 1 and base["kind"] == "oracle" and base["value"] > 0


@pytest.mark.parametrize("where", [0, 1023, 1024, 4999])
def test_planted_error_is_found_anywhere(case, where):
    sos, x, y_ref = case
    y = torch.from_numpy(y_ref.astype(np.float32))
    peak = float(np.abs(y_ref).max())
    y[where] += np.float32(0.01 * peak)
    _, acc = bench.cpu_baseline_leg(sos, x, y, chunk=1024)
    assert acc["max_rel_error"] == pytest.approx(0.01, rel=1e-3)


def test_without_output_only_times(case):
    sos, x, _ = case
    base, acc = bench.cpu_baseline_leg(sos, x)
    assert acc is None and base["value"] > 0


def test_bound_follows_the_pole_radius():
    x = workloads.normal_f32(6, 2048)
    sos = designs.resonator_bank()
    y = torch.from_numpy(oracle.sosfilt(sos, x).astype(np.float32))
    _, acc = bench.cpu_baseline_leg(sos, x, y, chunk=512)
    assert acc["bound"] == 2e-3 and acc["max_rel_error"] < 1e-6


def _run_bench(args, env_extra=None):
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **(env_extra or {}))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), *args], capture_output=True, text=True,
                         env=env, timeout=300, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_prints_one_contract_line():
    (line,) = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert line["impl"] == "reference" and line["unit"] == "GS/s" and line["value"] > 0
    assert line["steps"] == 1 and line["warmup"] == 3 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "GS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "2^28" in line["config"]["workload"]


def test_reference_arm_other_ranks_exit_quietly():
    assert _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "3"],
                      {"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"}) == []


def test_batched_sample_leg_counts_signals_within_their_bound():
    specs = [(sos, min(n, 20000), seed) for sos, n, seed in (workloads.batched_signal(i) for i in range(10))]
    xs = [workloads.normal_f32(seed, n) for _, n, seed in specs]
    ys = [torch.from_numpy(oracle.sosfilt(sos, x).astype(np.float32)) for (sos, _, _), x in zip(specs, xs)]
    ys[3][len(ys[3]) // 2] += 1.0  # one signal's output off by far more than its bound
    base, acc = bench.batch_sample_leg(specs, xs, ys, n_sample=8)
    assert acc["signals"] == 8 and acc["within_bound"] == 7
    assert acc["max_rel_error"] > 1e-3 and acc["median_rel_error"] < 1e-6
    assert base["kind"] == "oracle" and base["cores"] == 1 and base["value"] > 0
