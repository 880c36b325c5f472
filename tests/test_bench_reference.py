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


def test_clock_summary_reads_the_samples(tmp_path):
    """The clock record of the timed region: median SM clock, the maximum, and every throttle reason
    seen active in any sample (nvidia-smi csv, noheader, nounits); malformed lines are skipped."""
    import bench
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active\n"
                "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                "garbage line\n"
                "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    c.proc = object()          # as if the sampler had run
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    with open(c.path, "a") as f:
        f.write("0, 1500, 2070, 1000.0, 0x0, Not Active, Active, Not Active, Not Active\n"
                "0, 1500, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    s = c.summary()
    assert s["sm_mhz"] == 1980.0 and s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    c.proc = None              # no sampler (no nvidia-smi): no record
    assert c.summary() is None
