"""GPU check of bench.py's own line on the small single-cylinder configuration: one JSON
line with the contract's keys (roofline with the measured peak, the CPU baseline from the
oracle, clocks, the end-to-end figure with its copy bytes, the kernel-launch count, the
parity block), for the Q4 mesh and the mixed-cell mesh."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("mesh", ["q4", "cut"])
def test_bench_prints_one_contract_line(mesh):
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, "bench.py", "--config", "c1", "--steps", "2", "--warmup", "3",
                        "--mesh", mesh, "--cpu-units", "2e6", "--cpu-procs", "2", "--fp64-steps", "1",
                        "--mg-steps", "1"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "clocks", "e2e",
              "gpu_launches", "parity", "plain_fp64", "mg_pcg"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["all_converged"] and d["gpu_launches"] > 0
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["peak"] > 0
    assert rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"])
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 2
    e2e = d["e2e"]
    assert e2e["unit"] == d["unit"] and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]
    assert d["parity"]["variants"][0]["rel_residual_by_oracle"] <= 1e-8
    assert ("cutmesh" in d["config"]["workload"]) == (mesh == "cut")
