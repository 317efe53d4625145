"""bench.py's reference arm (the FP64 oracle timed on the host cores) keeps
the benchmark's JSON contract: one line with the GPU arm's metric, unit and
direction, `impl: "reference"`, a `cpu_baseline` describing the sample and an
`e2e` object with no host-device traffic.  Ranks other than 0 exit 0 without
work.  Run at refinement 3 (the profiling option) so that it takes seconds."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, env=None):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_json_line():
    out = _bench("--impl", "reference", "--steps", "2", "--warmup", "1", "--refinement", "3")
    assert out.returncode == 0, out.stderr
    lines = [line for line in out.stdout.splitlines() if line.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("phase-averaged RHS evals/sec")
    assert d["unit"] == "evals/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    # ms_per_step is the measured wall time of one sample step; value extrapolates to an evaluation
    assert d["value"] > 0 and d["ms_per_step"] > 0 and abs(d["est_eval_s"] * d["value"] - 1.0) <= 1e-12
    assert d["config"]["workload"].startswith("averaged_rhs r3 M64 T1h")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == min(16, os.cpu_count()) and cb["value"] == d["value"]
    assert "refinement 3" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = _bench("--impl", "reference", "--steps", "1", "--warmup", "0", "--refinement", "3", env=env)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""
