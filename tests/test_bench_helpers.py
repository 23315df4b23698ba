"""Host-side helpers of bench.py: the per-pair-form byte count, the
pair-kernel traffic lookup keyed by the kernel's source, and the compact
headline summary at the end of the JSON line, and the clock sampler (samples read
once nvidia-smi is stopped, warm work run while it starts)."""
import os
import shutil

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_pair_bytes():
    # 64 agents, 100 samples: 2016 pairs x 100 = 201,600 pair-times of 24 B, plus the
    # coefficients (3 axes x 11 x 64 floats) per instance
    assert bench.algorithmic_pair_bytes(64, 100, 1) == 24 * 201600 + 3 * 11 * 64 * 4
    assert bench.algorithmic_pair_bytes(64, 100, 256) == 256 * bench.algorithmic_pair_bytes(64, 100, 1)
    assert bench.algorithmic_pair_bytes(2, 10, 1) == 24 * 10 + 3 * 11 * 2 * 4


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    """A copy of the files the source key covers, and a profile summary keyed to them."""
    src = os.path.join(ROOT, "paper_2011_04240_b300", "csrc")
    dst = tmp_path / "paper_2011_04240_b300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("iterate.cu", "amto_internal.cuh", "pair_math.cuh", "schedule.cuh"):
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    key = bench.source_hash()
    (tmp_path / "profiles" / "pair_kernel_shell64.md").write_text(
        f"source_hash: {key}\nagents: 64\n"
        "dram_bytes_per_instance_launch_aggregate: 8.0e3\n"
        "dram_bytes_per_instance_launch_pairs: 4.7e6\n")
    return tmp_path


def test_traffic_lookup_scales_by_batch(fake_root):
    assert bench.profile_traffic(64, 256, "aggregate") == pytest.approx(8.0e3 * 256)
    assert bench.profile_traffic(64, 10, "pairs") == pytest.approx(4.7e6 * 10)


def test_traffic_lookup_other_agent_count_is_none(fake_root):
    assert bench.profile_traffic(32, 256, "aggregate") is None


def test_traffic_lookup_after_a_pair_kernel_change_is_none(fake_root):
    f = fake_root / "paper_2011_04240_b300" / "csrc" / "iterate.cu"
    f.write_text("// changed\n" + f.read_text())
    assert bench.profile_traffic(64, 256, "aggregate") is None


def test_traffic_lookup_ignores_the_right_hand_side_section(fake_root):
    # kernels after the pair kernel's section do not change the key
    f = fake_root / "paper_2011_04240_b300" / "csrc" / "iterate.cu"
    f.write_text(f.read_text() + "\n// a later kernel\n")
    assert bench.profile_traffic(64, 256, "aggregate") == pytest.approx(8.0e3 * 256)


def test_headline_summary_rounds_and_orders():
    rec = {"p50_ms": 18.654, "p99_ms": 56.81, "inst_iter_per_s": 85726.4, "resid_max": 0.0099999}
    ex = {"serving": [{"rate_req_s": 200.0, "window_s": 5.0, "server": rec,
                       "plain_fp32_per_instance": rec}],
          "mixed": {k: {"value": 3.7654e6} for k in
                    ("mixed", "mixed_branches", "mixed_loops", "per_count_sequential",
                     "per_count_concurrent_streams")},
          "precision": {"k": [1, 2], "oracle_K_par": [3, 4],
                        "errors": {"fp32": {"1": 3.04e-6, "2": 6.01e-6}},
                        "final_resid_max": {"fp32": 0.29674}}}
    out = bench.headline_summary(ex)
    assert out["serving"][0]["srv_p50_ms"] == 18.7 and out["serving"][0]["srv_res"] == 0.01
    assert out["mixed_ii_s"]["mixed_loops"] == 3.77e6
    assert out["precision"]["K_par"] == 3
    assert out["precision"]["xi_err"]["fp32"] == [3.0e-6, 6.0e-6]
    assert out["precision"]["res200"]["fp32"] == 0.3
    assert bench.headline_summary({}) == {}


class _FakeSmi:
    """Stands in for the nvidia-smi process: its samples come back from
    communicate() once it is stopped."""
    OUT = ("0, 2032, 2032, 455.30, 100, Not Active, Not Active, Not Active, Active\n"
           "0, 1980, 2032, 300.00, 98, Not Active, Not Active, Not Active, Not Active\n"
           "0, 2032, 2032, 120.00, 0, Not Active, Not Active, Not Active, Not Active\n"
           "garbage line\n")

    def __init__(self, *a, **k):
        self.stopped = False

    def terminate(self):
        self.stopped = True

    def communicate(self, timeout=None):
        assert self.stopped  # read only after the process is told to stop
        return self.OUT, None

    def kill(self):
        self.stopped = True


def test_clock_sampler_reads_after_stopping_and_runs_the_warm_work(monkeypatch):
    monkeypatch.setattr(bench.subprocess, "Popen", _FakeSmi)
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    ran = []
    with bench.ClockSampler(0, warm=lambda: ran.append(1)) as clk:
        assert clk.rows == []  # nothing is read while the timed code runs
    assert ran == [1]
    assert len(clk.rows) == 3
    sm = clk.summary()
    # samples under load (utilisation > 0): median SM clock, max power, reasons seen
    assert sm["samples"] == 2 and sm["sm_max_mhz"] == 2032.0
    assert sm["sm_mhz"] in (1980.0, 2032.0) and sm["power_w_max"] == 455.3
    assert sm["reasons"] == ["sw_power_cap"]
