"""bench.py's reference arm, which times the CPU oracle and needs no GPU: one JSON line on stdout
with the keys of the benchmark line and the oracle's rate as its value (the rate itself, a
timing, is not checked)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line(oracle):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "cell-updates/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"] and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["nproc"] >= 1 and d["cpu_baseline"]["lscpu_model"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("euler1d_batch4096")


def test_reference_arm_uses_the_benchmark_config():
    """The two arms describe the same workload: the reference line's config is the one the GPU
    line prints."""
    sys.path.insert(0, ROOT)
    import bench

    assert bench.config_dict(1)["problems"] == 4096 and bench.config_dict(2)["problems"] == 8192
    assert bench.RK_STEPS == 20 * bench.RK_PER_STEP  # 20 benchmark steps are the whole run


def test_kernel_hash_sees_code_not_comments(tmp_path, monkeypatch):
    """The hash that ties the committed ncu counters to the kernels: a changed comment or blank
    line keeps it, a changed line of code retires it; every committed counter file matches the
    current sources."""
    sys.path.insert(0, ROOT)
    import shutil

    import bench

    csrc = tmp_path / "paper_1504_00731_gb300" / "csrc"
    shutil.copytree(os.path.join(ROOT, "paper_1504_00731_gb300", "csrc"), csrc)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_hash()
    f = csrc / "wt_kernels.cuh"
    text = f.read_text()
    f.write_text("// a new comment\n\n" + text.replace("// ", "//  ", 3) + "\n/* and a block comment */\n")
    assert bench.kernel_hash() == h0
    f.write_text(text.replace("constexpr int kBar = 0;", "constexpr int kBar = 1;", 1))
    assert bench.kernel_hash() != h0
    monkeypatch.setattr(bench, "ROOT", ROOT)
    for kind in bench.COUNTERS:
        assert bench.counters(kind) is not None, kind
