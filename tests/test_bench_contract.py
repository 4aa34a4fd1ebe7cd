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


def test_other_forms_report_a_failing_form_and_keep_the_rest(monkeypatch):
    """The default run's window-construction, serving and batching entries: a
    form that raises is reported in its own entry (the headline line is still
    printed), the others keep their records and say how they were reduced."""
    sys.path.insert(0, ROOT)
    import argparse
    import bench

    seen = {}

    def ok(name):
        def fn(a):
            seen[name] = a
            return {"ran": name}
        return fn

    def broken(a):
        raise RuntimeError("no device")

    monkeypatch.setattr(bench, "features_result", ok("features"))
    monkeypatch.setattr(bench, "serve_result", broken)
    monkeypatch.setattr(bench, "batch_result", ok("batch"))
    args = argparse.Namespace(steps=50, warmup=5, features_cpu_rows=20000, serve_seconds=10.0, batch_problems=64,
                              batch_rhs=16, batch_sample=8, batch_lambda_min=1e-4)
    out = bench.other_forms(args)
    assert set(out) == {"window_construction", "serving", "batching"}
    assert out["serving"]["error"] == "RuntimeError: no device" and out["serving"]["reduced"] is None
    assert out["window_construction"]["ran"] == "features" and "10 timed calls" in out["window_construction"]["reduced"]
    assert out["batching"]["ran"] == "batch" and "16 problems" in out["batching"]["reduced"]
    # the reduced copies do not touch the caller's arguments
    assert seen["features"].steps == 10 and args.steps == 50
    assert seen["batch"].batch_problems == 16 and args.batch_problems == 64
