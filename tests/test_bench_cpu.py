"""CPU tests of the benchmark's contract pieces that need no GPU: the
reference arm's JSON line (the FP64 oracle on the host cores), the git blob
hash that gates the recorded DRAM traffic, and the roofline arithmetic."""
import io
import json
import os
import subprocess
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.main(["--impl", "reference", "--workload", "conjugate_gaussian_M8_N16_K16", "--steps", "2",
                         "--warmup", "1", "--ref-seconds", "1"])
    assert rc == 0
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "conjugate_gaussian_M8_N16_K16"


def test_blob_hash_matches_git(tmp_path):
    rel = os.path.relpath(os.path.join(ROOT, "include", "qem.h"), ROOT)
    try:
        want = subprocess.check_output(["git", "hash-object", rel], cwd=ROOT, text=True).strip()
    except Exception:
        import pytest
        pytest.skip("git unavailable")
    assert bench.git_blob_hash(rel) == want


def test_roofline_arithmetic():
    r = bench.roofline_for("forward", "bf16x3", 18, pairs=1e12, ms=100.0, sm_max_mhz=2000.0)
    assert abs(r["peak"] - 152 * 32 * 2e9 / 1e9) < 1e-6          # Gpair/s
    assert abs(r["achieved"] - 1e4) < 1e-6                         # 1e12 pairs in 0.1 s
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    f = bench.roofline_for("forward", "fp32", 18, pairs=1e12, ms=100.0, sm_max_mhz=2000.0)
    assert abs(f["peak"] - 152 * 128 * 2e9 / (3 * 18 + 4) / 1e9) < 1e-6


def _reference_line(argv):
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.main(["--impl", "reference", "--steps", "1", "--warmup", "1", "--ref-seconds", "1"] + argv)
    assert rc == 0
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_of_the_other_paths():
    """The split root, the parent-conditioned proposal and the chain plate time
    their own oracles (their pairs per step and proposal labelled in config)."""
    d = _reference_line(["--workload", "hier_logistic_M300_N5_K128", "--root", "split"])
    assert d["config"]["root"].startswith("split") and d["value"] > 0
    d = _reference_line(["--workload", "hier_logistic_M300_N5_K128", "--qcond"])
    assert d["config"]["proposal"].startswith("parent-conditioned") and d["value"] > 0
    d = _reference_line(["--workload", "chain_poisson_R92_T109_K128"])
    assert "regions" in d["cpu_baseline"]["sample"] and d["cpu_baseline"]["cores"] == 1


def test_traffic_gate_follows_the_source_hash():
    e = bench.NCU_TRAFFIC[("forward", "hier_logistic_M5000_N10_K1024", "bf16x3")]
    same = bench.git_blob_hash(e["source"]) == e["blob"]
    assert (bench.ncu_traffic("forward", "hier_logistic_M5000_N10_K1024", "bf16x3") is not None) == same
    assert bench.ncu_traffic("forward", "hier_logistic_M300_N5_K128", "fp32") is None


def test_profile_summaries_name_committed_commands():
    """Every summary under profiles/ gives the command that made it, through
    committed files (bench.py or a committed probe), never scratch paths, and
    every traffic figure the bench reports names an existing summary."""
    prof = os.path.join(ROOT, "profiles")
    names = sorted(f for f in os.listdir(prof) if f.endswith((".md", ".txt")))
    assert names
    for f in names:
        text = open(os.path.join(prof, f)).read()
        assert "bench.py" in text, f
        assert "_work" not in text and "/root/" not in text, f
        # commands continue over lines ending in a backslash
        for cmd in text.replace("\\\n", " ").splitlines():
            if cmd.lstrip().startswith("ncu "):
                assert "--clock-control none" in cmd, (f, cmd)
    for e in bench.NCU_TRAFFIC.values():
        assert os.path.exists(os.path.join(ROOT, e["profile"])), e["profile"]
        assert os.path.exists(os.path.join(ROOT, e["source"])), e["source"]
