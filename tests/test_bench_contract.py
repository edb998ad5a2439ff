"""The reference arm of bench.py (the oracle timed on the host cores) keeps the
JSON-line contract: one line from rank 0 with the metric, unit and config of
the GPU arm, `impl: reference`, a `cpu_baseline` describing the run and an
`e2e` entry without host-device copies; other ranks exit 0 without work.
Runs without a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)


def test_reference_arm_prints_one_contract_line():
    r = _run({}, "--steps", "1", "--warmup", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1
    assert d["ms_per_step"] > 0 and d["n_gpus"] == 1 and d["data"] == "synthetic"
    assert d["config"]["workload"] == bench.WORKLOAD and d["config"]["gaussians"] == 2_000_000
    from paper_2606_21791_gb300 import synth as S
    _, cams, flips = S.scale_workload(n=1000)
    assert d["config"] == bench.workload_config(2_000_000, cams, len(flips))   # the GPU arm's config
    assert "oracle" in d["engine"] and "not extrapolated in pixels" in d["cpu_baseline"]["sample"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    r = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}, "--gpus", "2", "--steps", "1", "--warmup", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_default_steps_per_arm(monkeypatch):
    """Without --steps/--warmup the GPU arm times 2,000 steps after 5 warm-up
    steps, the reference arm (seconds of CPU work a step) 4 after 1, so a run
    with no flags ends within minutes in both arms; given flags win."""
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.steps, a.warmup) == (2000, 5)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference"])
    a = bench.parse()
    assert (a.steps, a.warmup) == (4, 1)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "20", "--warmup", "5"])
    a = bench.parse()
    assert (a.steps, a.warmup) == (20, 5)
