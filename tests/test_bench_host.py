"""Host-side pieces of bench.py: the clock record keeps only samples inside the timed region."""
import datetime
import time

import bench


def _line(t, sm, power_cap="Not Active"):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return (f"{ts}, 0, {sm}, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, "
            f"Not Active, {power_cap}\n")


def test_clock_summary_keeps_the_timed_window():
    now = time.time()
    lines = [_line(now - 1.0, 345), _line(now + 0.1, 2070), _line(now + 0.3, 2055, "Active"),
             _line(now + 0.5, 2070), _line(now + 2.0, 400)]
    c = bench.summarise_clocks(lines, (now, now + 1.0))
    assert c["samples"] == 3 and c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["scope"] == "timed region"


def test_clock_summary_falls_back_and_rejects_garbage():
    now = time.time()
    lines = [_line(now, 2000), _line(now + 0.2, 2070)]
    c = bench.summarise_clocks(lines, (now + 10, now + 11))
    assert c["samples"] == 2 and c["scope"].startswith("whole run")
    assert bench.summarise_clocks(["garbage\n", ""], (now, now + 1)) is None


def test_reference_arm_line_keeps_the_contract(monkeypatch, capsys):
    """`bench.py --impl reference` (the FP64 oracle on the host cores) prints one JSON line with
    the contract's keys; a tiny time budget makes each step a prefix of the Gaussians."""
    import argparse
    import json

    monkeypatch.setattr(bench, "REF_BUDGET_S", 0.5)
    bench.run_reference(argparse.Namespace(steps=2, warmup=1), 1, 0)
    d = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert "the first" in d["cpu_baseline"]["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # rank > 0 prints nothing
    bench.run_reference(argparse.Namespace(steps=2, warmup=1), 2, 1)
    assert capsys.readouterr().out == ""


def test_power_law_fit_recovers_exponent():
    """The kernel sweep's time ~ a N^k fit: exact on a power law, and a sweep's grid sizes are
    whole bricks (the voxelizer's sides are multiples of 16)."""
    xs = [256 ** 2, 512 ** 2, 1024 ** 2, 2048 ** 2]
    k, a = bench.power_law(xs, [3e-4 * x ** 0.75 for x in xs])
    assert abs(k - 0.75) < 1e-9 and abs(a / 3e-4 - 1) < 1e-9
    assert all(s % 16 == 0 for s in bench.SWEEP_VOL_SIDES + (bench.SWEEP_VOX_SIDE,))
    assert bench.SWEEP_PX_SIDE ** 2 > 1e6 > 0.8 * bench.SWEEP_VOX_SIDE ** 3
