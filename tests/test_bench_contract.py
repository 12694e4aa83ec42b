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


def test_roofline_traffic_only_for_the_captured_kernel_source(tmp_path, monkeypatch):
    """The bench reports a kernel's DRAM traffic from the committed counter record
    (profiles/dram_traffic.json) only while the recorded source hash matches the kernel's
    current source text; otherwise null.  Every record names its summary, which quotes the same
    byte count and hash."""
    sys.path.insert(0, ROOT)
    import bench
    rec = json.load(open(bench.TRAFFIC_JSON))["kernels"]
    assert rec
    for phase, r in rec.items():
        txt = open(os.path.join(ROOT, "profiles", r["summary"])).read()
        assert str(r["dram_bytes_per_launch"]) in txt and r["source_sha16"] in txt, phase
        current = bench.kernel_source_sha(r["source"], r.get("markers")) == r["source_sha16"]
        assert (bench._traffic(phase) == r["dram_bytes_per_launch"]) if current else bench._traffic(phase) is None
    # a record whose hash no longer matches the source is not reported
    stale = {"kernels": {p: dict(r, source_sha16="0" * 16) for p, r in rec.items()}}
    path = tmp_path / "dram_traffic.json"
    path.write_text(json.dumps(stale))
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(path))
    for phase in rec:
        assert bench._traffic(phase) is None, phase


def test_profile_commands_run_committed_files_only():
    """Each profile summary gives the command that made it, and that command runs committed
    files (no scratch scripts)."""
    pdir = os.path.join(ROOT, "profiles")
    for name in os.listdir(pdir):
        if not name.endswith((".md", ".txt")):
            continue
        txt = open(os.path.join(pdir, name)).read()
        assert "_work/" not in txt, name
        assert "--clock-control none" in txt or "nvidia-smi" in txt, name


def test_chosen_block_and_degree():
    """The tube's chosen form runs at the swept block and degree unless the flags override them;
    LOBPCG keeps the library's block rule; every start block is drawn at least as wide as the
    block it feeds."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.chosen_block_degree(bench.parse([]), 64) == (80, 28)
    assert bench.chosen_block_degree(bench.parse(["--block", "84", "--degree", "26"]), 64) == (84, 26)
    assert bench.chosen_block_degree(bench.parse(["--solver", "lobpcg"]), 64) == (bench.solver_blocks(64)["lobpcg"], None)
    nb = bench.chosen_block_degree(bench.parse([]), 64)[0]
    assert max(max(bench.solver_blocks(64).values()), nb) >= nb > bench.solver_blocks(64)["chfsi"]
