"""Host logic of the library that needs no GPU: the batch planner.

tests/host/plan_batch_check.cpp is compiled against the library's headers
and linked with the built shared library (xg::plan_batch is exported); it
plans 400 seeded random batches and checks every invariant the batch kernel
relies on: each unit reachable once from the chain heads, one stream per
chain in submission order, heads costliest first, pieces only for calls
alone on their stream and at least two pieces long, contiguous pieces with
the right skips, output offsets and last-piece flag, exact coverage of every
call."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plan_batch_invariants(tmp_path):
    from paper_1108_0486_gb300 import build as B
    try:
        lib = B.build()
    except RuntimeError as e:  # pragma: no cover
        pytest.skip(str(e))
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("g++ unavailable")
    cuda_inc = "/usr/local/cuda/include"
    exe = str(tmp_path / "plan_batch_check")
    cmd = [cxx, "-O1", "-std=c++17", f"-I{ROOT}/include", f"-I{B.CSRC}", f"-I{cuda_inc}",
           os.path.join(ROOT, "tests", "host", "plan_batch_check.cpp"), "-o", exe,
           f"-L{os.path.dirname(lib)}", "-lxorgens_gb300", f"-Wl,-rpath,{os.path.dirname(lib)}"]
    for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/x86_64-linux/lib",
              "/usr/local/cuda/targets/sbsa-linux/lib"):
        if os.path.isdir(d):
            cmd += [f"-L{d}", f"-Wl,-rpath,{d}"]
    cmd += ["-lcudart"]
    subprocess.run(cmd, check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok 400"), out.stdout


def test_bench_clock_record_rules():
    """bench.py measures its timed region again when the clock record shows a
    slowdown reason, or SM clocks well below their maximum with no reason (a
    leftover clock lock); a power cap alone is kept."""
    import bench
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert not bench._throttled(ok)
    assert not bench._throttled(dict(ok, reasons=["sw_power_cap"]))
    assert bench._throttled(dict(ok, reasons=["hw_thermal_slowdown"]))
    assert bench._throttled(dict(ok, sm_mhz=1500.0))
    assert not bench._throttled({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]})


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference times the CPU oracle (the reference arm) and
    prints one JSON line with the contract's keys, its metric and config
    those of the GPU arm, a cpu_baseline describing the run and an e2e
    object with no bytes crossing."""
    import json
    import sys
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["warmup"] >= 3
    assert line["value"] > 0 and line["higher_is_better"] is True and line["unit"] == "RN/s"
    assert "workload" in line["config"]
    base = line["cpu_baseline"]
    assert base["kind"] == "oracle" and base["cores"] >= 1 and base["value"] == line["value"] and base["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
