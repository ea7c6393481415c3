"""bench.py's command-line contract on the CPU: the reference arm (the FP64 oracle timed on
the host cores) prints one JSON line with the contract's keys, and the native arm refuses
to run without a GPU instead of falling back to anything on the host."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, timeout=300):
    return subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True,
                          text=True, timeout=timeout)


def test_reference_arm_prints_the_contract_line():
    p = run_bench("--impl", "reference", "--workload", "validate", "--steps", "3", "--warmup",
                  "3")
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1
    assert d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["vs_baseline"] is None
    assert isinstance(d["config"].get("workload"), str)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["unit"] == d["unit"] and isinstance(cb["sample"], str)
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_native_arm_fails_loudly_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the native arm would run")
    p = run_bench("--steps", "1", "--warmup", "3", "--legs", "none")
    assert p.returncode != 0
    assert not [l for l in p.stdout.splitlines() if l.startswith("{")]


def test_roofline_accounting():
    """The per-unit work bench.py divides by kernel time: one Alg. 1 waypoint update at
    dof 7 = 558 FLOP (chain 48, roll-pitch task 8 and damped step 9 and update 10 per joint,
    plus the fixed parts), sphere FK 18, 11 / 34 / 25 per sphere / box / capsule pair, the
    warm-start network's 2 x (7x256 + 2x256x256 + 256x7) per row, and the nominal FP32 peak
    152 SMs x 128 lanes x 2 x 2070 MHz."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench

    assert bench.flops_waypoint_iter(7) == 558
    assert bench.flops_cc_waypoint(1, 1, 0, 0) == 18 + 11
    assert bench.flops_cc_waypoint(59, 100, 60, 40) == 59 * (18 + 100 * 11 + 60 * 34 + 40 * 25)
    # outcomes: valid, projection failed, first collision at waypoint 3
    f, cc = bench.algorithmic_flops(7, 32, 59, (16, 0, 0), [0, 1, 2], [-1, 5, 3], [2, 20, 1])
    assert cc == 32 + 0 + 4
    assert f == (2 + 20 + 1) * 31 * 558 + cc * bench.flops_cc_waypoint(59, 16, 0, 0)
    ex = bench.executed_flops(7, [10, 3, 100, 7, 5, 2])
    assert ex == 10 * 558 + 3 * 7 * 48 + 100 * 18 + 7 * 11 + 5 * 34 + 2 * 25
    assert bench.mlp_flops_per_row(7) == 269312
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 80.548) < 1e-3
    work = np.array([[100, 40], [0, 8]])
    from paper_2505_06791_gb300 import synth as S
    scenes = [S.make_scene(1, 16), S.make_scene(2, 4, 2, 1)]
    want = 100 * 558 + 40 * bench.flops_cc_waypoint(59, 16, 0, 0) + \
        8 * bench.flops_cc_waypoint(59, 4, 2, 1)
    assert bench.plan_flops(7, scenes, 59, work) == want


def test_reference_arm_under_torchrun_prints_once():
    """Launched as the scaling run launches it (torchrun, 2 ranks; gloo here), only rank 0
    runs the oracle and prints; the other rank exits 0 without work."""
    env = dict(os.environ, CPRRTC_BENCH_GLOO="1")
    p = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", "29563", "bench.py", "--impl", "reference",
                        "--gpus", "2", "--workload", "validate", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True,
                       timeout=300, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
