"""The reference arm of bench.py (the oracle timed on the host cores), on the small real workload:
one JSON line with the keys the bench line carries, the same metric and workload naming as the
GPU arm, e2e equal to the line's value with no host-device bytes, and no output on ranks other
than 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ, **(extra_env or {}))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                           "--warmup", "1", "--workload", "1"], capture_output=True, text=True, env=env,
                          timeout=300, cwd=ROOT)


def test_reference_line_contract():
    p = _run()
    assert p.returncode == 0, p.stderr
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "moves/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    assert abs(d["ms_per_step"] - 1e3 / d["value"]) < 1e-9 * d["ms_per_step"]
    assert d["config"]["workload"] == bench.workload_name(1)
    assert "D=2 chi=16 (q=4: 3 even/1 odd)" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and "D=2" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "moves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    p = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_workload_name_of_the_headline():
    import bench
    assert bench.workload_name(3) == ("real C4v iPEPS d=2 D=6 chi=144 (q=36: 21 even/15 odd), seeded N(0,1), "
                                      "D4-symmetrised, max|A|=1")
