"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps
the JSON contract of the benchmark line, on CPU."""
import json
import os
import subprocess
import sys

from conftest import ROOT


def run_bench(*args):
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                         capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_prints_one_contract_line():
    d = run_bench("--impl", "reference", "--workload", "vortex_square_small", "--steps", "2",
                  "--warmup", "1")
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert "unavailable" not in d
    assert d["metric"] == "cell updates/s" and d["unit"] == "cell-updates/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1
    assert d["config"]["workload"] == "vortex_square_small"
    assert d["config"]["cells"] == 4096
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_on_the_batch_samples_its_largest_mesh():
    d = run_bench("--impl", "reference", "--workload", "batch_256", "--steps", "1",
                  "--warmup", "0")
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["config"]["workload"] == "batch_256"
    assert d["config"]["cells"] > 100_000


def test_reference_arm_other_ranks_exit_without_work():
    # under torchrun only rank 0 prints the line; the other ranks exit 0
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "vortex_square_small", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
