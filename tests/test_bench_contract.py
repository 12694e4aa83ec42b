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
    """The bench reports a kernel's DRAM traffic from its committed ncu summary only while the
    summary's source hash matches the kernel's current source text; otherwise null."""
    sys.path.insert(0, ROOT)
    import bench
    for phase, (summary, source, markers) in bench._TRAFFIC_SRC.items():
        txt = open(os.path.join(ROOT, "profiles", summary)).read()
        assert bench.kernel_source_sha(source, markers) in txt, phase   # captured on this source
        assert bench._traffic(phase) > 0, phase
        stale = tmp_path / "profiles"
        stale.mkdir(exist_ok=True)
        (stale / summary).write_text(txt.replace(bench.kernel_source_sha(source, markers), "0" * 16))
        real_root = bench.ROOT
        monkeypatch.setattr(bench, "ROOT", str(tmp_path))
        (tmp_path / "paper_2210_12252_gb300").mkdir(exist_ok=True)
        src = tmp_path / "paper_2210_12252_gb300" / "csrc"
        src.mkdir(exist_ok=True)
        (src / source).write_bytes(open(os.path.join(real_root, "paper_2210_12252_gb300", "csrc", source), "rb").read())
        assert bench._traffic(phase) is None, phase
        monkeypatch.setattr(bench, "ROOT", real_root)


def test_profile_commands_run_committed_files_only():
    """Each profile summary gives the command that made it, and that command runs committed
    files (no scratch scripts)."""
    pdir = os.path.join(ROOT, "profiles")
    for name in os.listdir(pdir):
        txt = open(os.path.join(pdir, name)).read()
        assert "_work/" not in txt, name
        assert "--clock-control none" in txt or "nvidia-smi" in txt, name
