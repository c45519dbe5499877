"""Host side of the benchmark (no GPU): the committed ncu summaries describe
the kernel sources as they are (a kernel edit without a new capture fails
here), the stored DRAM traffic is the one read of Y the roofline assumes,
and the reference arm prints its JSON line on rank 0 only."""

import importlib.util
import json
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORKLOAD = "seg256s_bank1024_pn35"


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_profiles_describe_the_current_kernel_sources(bench):
    dig = bench.source_digest()
    for kernel in ("pass1", "pass2"):
        text = open(os.path.join(ROOT, "profiles", f"{kernel}_{WORKLOAD}.md")).read()
        assert re.search(r"source_digest:\s*([0-9a-f]+)", text).group(1) == dig, kernel
    text = open(os.path.join(ROOT, "profiles", f"launches_{WORKLOAD}.md")).read()
    assert re.search(r"Source digest of the fused kernels: ([0-9a-f]+)", text).group(1) == dig


def test_stored_traffic_is_one_read_of_y(bench):
    n = 1 << 20
    algorithmic = n * 8  # complex64 Y, read once per template
    t = bench.stored_traffic("pass2", WORKLOAD)
    assert t is not None and 0.99 * algorithmic <= t <= 1.02 * algorithmic
    assert bench.stored_traffic("pass2", "no_such_workload") is None


def _run_reference(env_extra):
    env = dict(os.environ, **env_extra)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
           "seg16s_bank64_pn2", "--steps", "1", "--warmup", "0"]
    return subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)


def test_reference_arm_prints_one_oracle_line():
    r = _run_reference({})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "templates/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "seg16s_bank64_pn2"


def test_reference_arm_is_silent_off_rank_zero():
    r = _run_reference({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
