"""The bench's reference arm (the FP64 oracle timed on the host cores) runs
without a GPU and prints one JSON line with the bench contract's keys; a rank
other than 0 prints nothing and exits 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, *args):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    p = _run({}, "--steps", "1", "--warmup", "0")
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, p.stdout
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference"
    assert rec["unit"] == "particle-steps/s" and rec["higher_is_better"] is True
    assert rec["value"] > 0 and rec["steps"] == 1 and rec["warmup"] == 0 and rec["n_gpus"] == 1
    assert rec["dtype"] == "f64" and rec["data"] == "synthetic" and rec["scaling"] == "weak"
    assert rec["vs_baseline"] is None
    assert rec["config"]["workload"] and rec["config"]["particles"] > 0
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == rec["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = rec["e2e"]
    assert e2e["value"] == rec["value"] and e2e["unit"] == rec["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_print_nothing():
    p = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--steps", "1", "--warmup", "0")
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
