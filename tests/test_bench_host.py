"""Host-side helpers of bench.py (no GPU): the clock sampler's summary and the peak table."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _clocks_from(bench, tmp_path, lines):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    return c.summary()


def test_clock_summary_median_max_and_reasons(bench, tmp_path):
    lines = ["0, 2070, 2070, 910.5, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2055, 2070, 990.2, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1001.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = _clocks_from(bench, tmp_path, lines)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    assert s["power_w_max"] == 1001.0
    assert not os.path.exists(str(tmp_path / "clocks.csv"))   # the sample file is removed


def test_clock_summary_flags_thermal_slowdown(bench, tmp_path):
    lines = ["0, 1500, 2070, 800.0, 0x40, Not Active, Active, Not Active, Not Active"]
    s = _clocks_from(bench, tmp_path, lines)
    assert s["reasons"] == ["hw_thermal_slowdown"] and s["sm_mhz"] == 1500.0


def test_clock_summary_without_samples(bench, tmp_path):
    s = _clocks_from(bench, tmp_path, ["", "garbage"])
    assert s["sm_mhz"] is None and s["reasons"] == ["no samples"]
    c = bench.Clocks(0)
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_peaks_reads_the_measured_table_or_falls_back(bench, tmp_path, monkeypatch):
    gbs, kind = bench.peaks()
    assert gbs > 0 and kind in ("measured", "fallback")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6767.4}')
    assert bench.peaks() == (6767.4, "measured")


def test_cpu_oracle_step_pieces_add_up_to_one_solve(bench):
    """The reference arm splits one oracle time-to-solution over the timed steps: any
    split runs the same Jacobi sweeps to the same iterate as one uninterrupted run."""
    from paper_1210_6412_gb300 import synth
    c = synth.dense_random_chain(n=1500, density=0.1, goal_frac=0.02, seed=3)
    one = bench.CpuOracleStep(c, pieces=1).run()
    many = bench.CpuOracleStep(c, pieces=7, expect_sweeps=one.sweeps // 2).run()
    assert one.done and many.done
    assert one.sweeps == many.sweeps
    assert (one.x == many.x).all()
    rec = many.record()
    assert rec["kind"] == "oracle" and rec["cores"] >= 1 and rec["nproc"] >= 1
    assert rec["max_err"]["jacobi"] < 1e-8 and rec["max_err"]["bicgstab"] < 1e-8
    assert abs(rec["value"] - sum(rec["parts_ms"].values())) < 1e-6
    single = bench.cpu_single_core_estimate(many.m, many.b, many.sweeps, sweeps=2)
    assert single["kind"] == "extrapolated" and single["cores"] == 1
