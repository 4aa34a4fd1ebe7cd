"""bench.py's reference arm prints the contract's JSON line (CPU only: the arm
times the FP64 oracle on a bounded sample of the benchmark workload)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

REQUIRED = ["metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
            "scaling", "vs_baseline", "dtype", "data", "config"]


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--ref-sample", "400"], capture_output=True, text=True, cwd=ROOT, env=env,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in REQUIRED:
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["warmup"] >= 3 and d["steps"] == 1
    assert d["value"] > 0 and d["unit"] == "Gpts/s" and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("precision_N1000000")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "400" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_is_silent_off_rank_zero():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--ref-sample", "400"], capture_output=True, text=True, cwd=ROOT, env=env,
                       timeout=600)
    assert r.returncode == 0
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_traffic_figure_only_for_the_kernel_source_it_was_taken_on(tmp_path):
    """roofline.traffic comes from the committed ncu table and is dropped as soon as
    the sources the kernel is built from differ from those the counters were taken on."""
    sys.path.insert(0, ROOT)
    import bench
    sha = bench.source_sha(["dense3.cu", "common.cuh"])
    f = tmp_path / "t.md"
    f.write_text("| kernel | workload | bytes | sources | sha |\n|---|---|---|---|---|\n"
                 f"| `k_x<14>` | wl | 1,234,567 | dense3.cu + common.cuh | {sha} |\n"
                 "| `k_y<14>` | wl | 999 | dense3.cu | 0000000000000000 |\n")
    assert bench.traffic_per_launch("k_x<14>", "wl", path=str(f)) == 1234567
    assert bench.traffic_per_launch("k_x<14>", "other", path=str(f)) is None
    assert bench.traffic_per_launch("k_y<14>", "wl", path=str(f)) is None     # stale: sources changed
    assert bench.traffic_per_launch("k_z<14>", "wl", path=str(f)) is None
