"""CPU test of bench.py's reference arm (the oracle timed on the host cores):
one JSON line with the contract's keys, an e2e entry with zero transfers, a
cpu_baseline describing the sample, ms_per_step the measured time of one
sampled step (a full step of the bench workload is far beyond what the oracle
can run in a bench step; its extrapolated time is a separate, labelled key),
and the same config as the GPU arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "block_20x20x10",
           "--steps", "2", "--warmup", "1", "--cpu-stations", "4", "--cpu-cells", "8"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT,
                         env={**os.environ, "WORLD_SIZE": "1", "RANK": "0"})
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
              "cpu_baseline", "e2e", "impl"):
        assert k in rec, k
    assert rec["impl"] == "reference" and rec["steps"] == 2 and rec["warmup"] == 1
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["e2e"]["d2h_bytes_per_step"] == 0
    assert rec["e2e"]["value"] == rec["value"] and rec["cpu_baseline"]["value"] == rec["value"]
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["cores"] >= 1
    # 20 x 20 x 10 cells, 441 stations: a step is 2 N M pairs, the sample 4 M + 8 N
    assert rec["sample_pairs_per_step"] == 4 * 4000 + 8 * 441
    assert rec["ms_per_step_basis"].startswith("measured")
    # the value is the sample's rate; the extrapolated full step follows from it
    full = 2 * 441 * 4000
    assert abs(rec["full_step_ms_extrapolated"] - full / rec["value"] * 1e3) < 1e-9 * rec["full_step_ms_extrapolated"]
    # ms_per_step is a measured sample step: within a factor of the sample at the median rate
    est = rec["sample_pairs_per_step"] / rec["value"] * 1e3
    assert 0.2 * est < rec["ms_per_step"] < 5 * est
    assert rec["config"]["workload"] == "block_20x20x10" and rec["config"]["cells"] == 4000
    assert set(rec["config"]) == {"workload", "cells", "stations", "precision", "near_cells", "l2", "parallelism"}
