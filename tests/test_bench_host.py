"""Host-side pieces of bench.py that need no GPU: the reference arm's JSON line
(the FP64 oracle on the host cores, small workload) and the parsing of the
nvidia-smi clock samples."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "0",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["unit"] == "evals/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "d=8" in d["config"]["workload"]


def test_clock_sampler_parses_samples_and_reasons():
    cs = bench.ClockSampler(0)
    cs.proc = None
    assert cs.stop()["reasons"] == ["nvidia-smi unavailable"]

    class _P:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs.proc = _P()
    cs.lines = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
                "0, 2040, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
                "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
                "garbage line"]
    r = cs.stop()
    assert r["sm_mhz"] == 2055.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] == 3 and r["power_w_max"] == 1400.0
