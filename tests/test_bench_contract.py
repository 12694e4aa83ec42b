"""The benchmark's command-line contract on the CPU: the reference arm (the oracle timed on the
host cores) prints one JSON line with the keys the harness reads, and the argument parser
takes the documented flags."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("tube")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_parser_defaults_and_flags():
    sys.path.insert(0, ROOT)
    import bench
    a = bench.parse([])
    assert (a.gpus, a.steps, a.warmup, a.impl, a.solver) == (1, 5, 3, "ours", "chfsi")
    b = bench.parse(["--gpus", "2", "--steps", "4", "--warmup", "3", "--solver", "lobpcg", "--precond", "tpa"])
    assert (b.gpus, b.steps, b.warmup, b.solver, b.precond) == (2, 4, 3, "lobpcg", "tpa")
