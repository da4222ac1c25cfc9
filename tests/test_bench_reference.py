"""The bench's reference arm on the host (no GPU): for every operation it
prints one JSON line with the contract's keys, timed on the oracle."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


@pytest.mark.parametrize("op,extra", [("knn", ["--ref-queries", "8"]),
                                      ("knn", ["--workload", "latent3", "--ref-queries", "8"]),
                                      ("knn", ["--workload", "gmm16"]),
                                      ("knn", ["--workload", "batched", "--ref-queries", "16"]),
                                      ("kfn", []), ("range", []), ("emst", [])])
def test_reference_arm_prints_one_line(op, extra):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--op", op,
           "--n-ref", "3000", "--n-query", "200", "--steps", "1", "--warmup", "1", *extra]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    j = json.loads(lines[0])
    assert KEYS <= set(j), KEYS - set(j)
    assert j["impl"] == "reference" and j["value"] > 0 and j["higher_is_better"] is True
    assert j["e2e"]["value"] == j["value"] and j["cpu_baseline"]["kind"] == "oracle"
