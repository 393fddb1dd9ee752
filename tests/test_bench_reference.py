"""The benchmark's reference arm (the CPU oracle, no GPU): its JSON line keeps
the keys of the benchmark contract, and the forms the oracle does not have
print an `unavailable` line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_line_has_the_contract_keys():
    d = _run("--workload", "hp2d-coef", "--steps", "1", "--warmup", "0")
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert "coefficient" in d["config"]["workload"] and d["config"]["n_dofs"] == 98127
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_reference_unavailable_for_batched_form():
    d = _run("--workload", "batched")
    assert d["impl"] == "reference" and "unavailable" in d


def test_reference_amr_sequence():
    d = _run("--workload", "amr-layer", "--amr-steps", "3")
    assert d["impl"] == "reference" and d["value"] > 0 and len(d["table"]) == 4
    assert d["table"][-1]["n_dofs"] > d["table"][0]["n_dofs"]
