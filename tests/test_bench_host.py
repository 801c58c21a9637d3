"""Host logic of bench.py that needs no GPU: the clock sampler keeps only the
samples time-stamped inside the timed region, and the step defaults."""
import os
import sys
import time
from datetime import datetime

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Done:
    """Stands in for the nvidia-smi process once it has written its samples."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _line(t, sm, power_cap="Not Active"):
    stamp = datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ("%s, 0, %d, 2070, 900.00, 0x0000000000000000, Not Active, Not Active, "
            "Not Active, %s\n" % (stamp, sm, power_cap))


def _sampled(tmp_path, lines, t0, t1):
    c = bench.Clocks(None)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.writelines(lines)
    c.f = open(c.path)
    c.proc = _Done()
    return c.stop(t0, t1)


def test_only_samples_inside_the_timed_region_count(tmp_path):
    now = time.time()
    lines = [_line(now - 1.0, 1000), _line(now + 0.10, 2070), _line(now + 0.12, 2055),
             _line(now + 0.14, 2070, power_cap="Active"), _line(now + 2.0, 600)]
    out = _sampled(tmp_path, lines, now, now + 0.2)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["window"] == "timed region"
    assert not os.path.exists(tmp_path / "clocks.csv")


def test_no_sample_inside_falls_back_and_says_so(tmp_path):
    now = time.time()
    out = _sampled(tmp_path, [_line(now - 1.0, 1980), _line(now + 5.0, 2070)], now, now + 0.05)
    assert out["samples"] == 0
    assert out["window"].startswith("whole run")
    assert out["sm_mhz"] == (1980 + 2070) / 2


def test_malformed_lines_are_skipped(tmp_path):
    now = time.time()
    lines = ["garbage\n", "[Not Supported], 0, N/A, N/A, , , , , , \n", _line(now + 0.01, 2070)]
    out = _sampled(tmp_path, lines, now, now + 0.1)
    assert out["samples"] == 1 and out["sm_mhz"] == 2070.0


def test_missing_sampler_is_reported():
    c = bench.Clocks(None)
    c.proc = None
    assert c.stop(0.0, 1.0)["reasons"] == ["nvidia-smi unavailable"]


def test_step_defaults(monkeypatch):
    def steps(*argv):
        monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
        a = bench.default_steps(bench.parse())
        return a.steps, a.warmup
    assert steps() == (20, 5)                              # the suite's headline
    assert steps("--workload", "atm_two_spot") == (200, 10)
    assert steps("--impl", "reference") == (20, 5)
    assert steps("--workload", "batch") == (3, 3)
    assert steps("--workload", "grad_batch") == (3, 3)
    assert steps("--steps", "7", "--warmup", "4") == (7, 4)


def test_traffic_only_for_the_profiled_configuration(monkeypatch):
    def cfg(*argv):
        monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
        return bench.profiled_config(bench.default_steps(bench.parse()))
    assert cfg()
    assert cfg("--steps", "2", "--warmup", "3", "--no-cpu-baseline", "--graph")
    assert not cfg("--workload", "batch")
    assert not cfg("--workload", "healpix_map")
    assert not cfg("--interp", "a")
    assert not cfg("--phase-sub", "4")
    assert not cfg("--walk", "1")
    assert not cfg("--autotune")


def test_forward_kernel_names():
    import numpy as np
    from paper_2510_07764_gb300 import synth
    w = synth.bb_small(n_theta=4, n_phi=4, n_phase=4, n_E=4)
    assert bench.forward_kernel_name(w) == "k_shift_add<blackbody>"
    w.inst.emission = 1
    assert bench.forward_kernel_name(w) == "k_shift_add<atmosphere>"
    w.inst.logT_map = np.zeros((1, 12))
    assert bench.forward_kernel_name(w) == "k_shift_add_map<atmosphere>"


def test_reference_stride_keeps_the_run_within_budget():
    # 55 steps of 1.9 s fit 120 s only at a wider stride; 10 steps do not need one
    assert bench.reference_stride(1.9, 64, 10, budget_s=120.0) == 64
    s = bench.reference_stride(1.9, 64, 205, budget_s=120.0, max_stride=128)
    assert s == 128                       # capped at the rings of a spot
    s = bench.reference_stride(1.9, 64, 100, budget_s=120.0, max_stride=1000)
    assert s >= 64 and 100 * 1.9 * 64 / s <= 120.0 + 1e-9


def test_sample_factor_counts_the_rings_sampled():
    from paper_2510_07764_gb300 import synth
    w = synth.atm_two_spot(n_theta=128, n_phi=8, n_phase=4, n_E=4, n_chan=2)
    assert bench.sample_factor(w.inst, 16, 4) == 16.0
    assert bench.sample_factor(w.inst, 100, 4) == 64.0     # rings 0 and 100 of 128
    assert bench.sample_factor(w.inst, 1, 4) == 1.0
    h = synth.healpix_map(n_side=8, n_phase=4, n_E=4, n_chan=2)
    assert bench.sample_factor(h.inst, 16, 4) == 31 / 2     # 4 N - 1 = 31 rings, 2 sampled


def test_reference_arm_prints_its_json_line():
    """bench.py --impl reference runs the oracle on the host and prints one
    JSON line with the keys the reference arm's contract names."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "bb_small", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, check=True, cwd=ROOT)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["unit"] == "profile evals/s" and line["higher_is_better"] is True
    assert (line["steps"], line["warmup"], line["n_gpus"]) == (2, 1, 1)
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert "ring" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 \
        and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"] == "bb_small"
