"""bench.py's JSON contract on the host: the reference arm (the oracle) of the
blockwise-SVD workload runs without a GPU and prints one line with every key
the contract names; the workload list and step defaults parse."""
import json
import os
import subprocess
import sys

from tests.conftest import ROOT

KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e")


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--workload", "u1_two_site_svd", "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in KEYS:
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert "workload" in d["config"]


def test_every_workload_parses_with_its_defaults():
    sys.path.insert(0, ROOT)
    import bench
    for w in ("u1_mps_heff", "su2_recouple", "u1_two_site_batch", "u1_mera_grad", "z2f_mps_heff", "su2u1_mps_heff",
              "u1_two_site_svd", "su2_micro"):
        old = sys.argv
        sys.argv = ["bench.py", "--workload", w]
        try:
            a = bench.parse()
        finally:
            sys.argv = old
        assert a.workload == w and a.steps >= 1 and a.warmup >= 1
