"""The reference arm of bench.py (the FP64 CPU oracle, timed on the host
cores) keeps the one-line JSON contract: run here on a 33^3 grid, where the
oracle finishes in about a second.  No GPU is involved on this arm."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, steps=1, extra_args=()):
    env = dict(os.environ)
    env.update(extra_env or {})
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "33", "--steps", str(steps),
                        "--warmup", "1", *extra_args], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    return [ln for ln in p.stdout.splitlines() if ln.strip()]


def test_reference_arm_prints_one_json_line_with_the_contract_keys():
    lines = _run()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["unit"] == "unknowns/s" and d["higher_is_better"] is True
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (1, 1, 1)
    assert "33^3" in d["config"]["workload"] and d["config"]["n"] == 33
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    # every step is a complete, measured solve to the tolerance
    assert len(d["solve_s"]) == d["steps"] and d["residual"] <= d["config"]["tol"] and d["cycles_per_solve"] > 0
    assert abs(1e3 * sum(d["solve_s"]) / d["steps"] - d["ms_per_step"]) <= 1e-6 * d["ms_per_step"]
    assert "measured" in cb["sample"] and "extrapolat" not in cb["sample"]


def test_reference_arm_times_every_requested_step_that_fits_and_one_thread_on_request():
    d = json.loads(_run(steps=3, extra_args=("--cpu-threads", "1"))[0])
    assert d["steps"] == d["steps_requested"] == 3 and len(d["solve_s"]) == 3
    assert d["cpu_baseline"]["cores"] == 1


def test_reference_arm_runs_on_rank_zero_only():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []
