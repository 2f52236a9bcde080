"""Host logic of bench.py on CPU: the reference arm (the oracle, timed on host cores) prints one JSON line with
the fields of the benchmark contract, the oracle described in cpu_baseline and no host-device traffic; the
clock sampler reduces nvidia-smi rows to the clocks record (median SM clock, maximum, active throttle reasons)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--workload", "heat2d-32-radau2"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["unit"] == "time-steps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1000.0 / d["value"]) <= 0.05 * d["ms_per_step"] + 0.01
    assert d["config"]["workload"] == "heat2d-32-radau2"
    # the same config object the GPU arm prints for these arguments (the driver compares the two)
    sys.path.insert(0, ROOT)
    import argparse

    import bench

    wl = bench.W.WORKLOADS["heat2d-32-radau2"]
    args = argparse.Namespace(orth="cgs", restart=50, tab_override=None)
    assert d["config"] == bench.workload_config(wl, args, "fp64", "lower", "ia", 1)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_clock_sampler_parses_nvidia_smi_rows(tmp_path):
    """The clocks record of the JSON line: median SM clock under load, the maximum, and the throttle reasons
    seen active in any sample (nvidia-smi csv,noheader,nounits rows; 'Not Active' is not a reason)."""
    sys.path.insert(0, ROOT)
    import bench

    c = bench.Clocks(None)
    rows = ["0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("\n".join(rows) + "\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c.proc = Done()
    c.fh = open(os.devnull, "w")
    rec = c.stop()
    assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not os.path.exists(c.path)
