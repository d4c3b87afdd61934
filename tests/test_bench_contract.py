"""bench.py's host logic and the reference arm's JSON line, on the CPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_of_the_1m_atom_product():
    # 1,970,150 bonds x 100 FP64 entries + x and y (10M rows, 8 B) + species and potential per atom
    assert bench.alg_bytes_per_hx(1_970_150, 1_000_000, 10_000_000, 8, 8, False) == 1_745_120_000
    # matrix-free: no blocks, one 8-byte strain per bond instead
    assert bench.alg_bytes_per_hx(1_970_150, 1_000_000, 10_000_000, 4, 4, True) == \
        2 * 10_000_000 * 4 + 9_000_000 + 8 * 1_970_150
    assert bench.flops_per_hx(1_970_150, 1_000_000) == 2.0 * (200 * 1_970_150 + 10 * 1_000_000)


def test_job_throughput_counts_every_rank():
    assert bench.job_throughput(4, 1e9, 10, 2.0) == pytest.approx(20.0)


def test_clock_summary_reads_samples_and_reasons(tmp_path):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    s.proc = object()          # samples present, as if nvidia-smi had run
    with open(s.path, "w") as f:
        f.write("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("garbage line\n")
    out = s.summary()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, cwd=ROOT, timeout=600, check=True)
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    # the config names the slab the reference arm times (50 x 50 x 4 cells of the 1M-atom recipe)
    assert line["config"]["atoms"] == 80_000 and line["config"]["rows"] == 800_000
    assert "50x50x4" in line["config"]["workload"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
