"""The benchmark's reference arm (the oracle timed on the host) prints one JSON
line with the contract's keys; runs on CPU in a few seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-cores", "2"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["cpu_baseline"]["cores"] == 2 and line["config"]["streams"] == 2


def test_clock_summary_parses_nvidia_smi_lines():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.lines = ["2070, 2070, 800.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
               "2055, 2070, 812.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "[N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    s = c.summary()
    assert s == {"sm_mhz": 2062.5, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 2}
    assert bench.ClockSampler(0).summary()["samples"] == 0


def test_gpus_flag_must_match_the_launched_ranks():
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--impl", "reference"],
                       capture_output=True, text=True, timeout=120, cwd=ROOT, env=env)
    assert r.returncode != 0 and "--gpus 2 but the launcher started 1 ranks" in r.stderr


def test_gpus_flag_without_a_launcher_starts_one_rank_per_gpu(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    seen = {}
    monkeypatch.setattr(bench.subprocess, "call", lambda cmd: seen.setdefault("cmd", cmd) and 0)
    monkeypatch.setattr(bench.sys, "argv", ["bench.py", "--gpus", "4", "--steps", "3"])
    assert bench.launch_ranks(4) == 0
    cmd = seen["cmd"]
    assert cmd[1:3] == ["-m", "torch.distributed.run"]
    assert cmd[cmd.index("--nproc-per-node") + 1] == "4" and cmd[cmd.index("--master-addr") + 1] == "127.0.0.1"
    assert cmd[-4:] == ["--gpus", "4", "--steps", "3"]
    assert bench.host_cores() >= 1


def test_launch_count_per_frame_follows_the_schedule():
    # splat, fill, window, row scan, census, cost, sweep(s), update
    sys.path.insert(0, ROOT)
    import bench
    assert bench.launches_per_frame(0) == 9          # row sweep beside the line sweep
    for rows in (8, 16, 32):
        assert bench.launches_per_frame(rows) == 8   # one line sweep for every direction
