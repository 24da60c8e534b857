"""bench.py's clock record on the CPU: the summary of nvidia-smi samples
(median SM clock inside the timed window, the maximum clock, the throttle
reasons seen there) from synthetic sample lines, through ClockSampler.stop
with a stand-in for the nvidia-smi process."""

import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

T0 = datetime.datetime(2026, 1, 2, 3, 4, 5)


def line(dt_ms, sm, smax, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    ts = (T0 + datetime.timedelta(milliseconds=dt_ms)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{ts}, {sm}, {smax}, 650.00, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def window(a_ms, b_ms):
    base = T0.timestamp()
    return base + a_ms / 1000.0, base + b_ms / 1000.0


def test_median_and_reasons_inside_the_window_only():
    out = "\n".join([line(0, 1000, 2070, hw="Active"),            # before the window
                     line(100, 2070, 2070), line(150, 2000, 2070, cap="Active"), line(200, 2070, 2070),
                     line(400, 900, 2100, hwt="Active"),          # after the window
                     "garbage line", "2026/01/02 03:04:05.300, [N/A], 2070, 1, 0x0, a, b, c, d"])
    t0, t1 = window(90, 210)
    r = bench.ClockSampler.summarise(out, t0, t1)
    assert r["sm_mhz"] == 2070.0 and r["samples"] == 3
    assert r["sm_max_mhz"] == 2100.0
    assert r["reasons"] == ["sw_power_cap"]
    assert abs(r["window_s"] - 0.12) < 1e-6  # epoch seconds in FP64


def test_no_samples_in_the_window():
    r = bench.ClockSampler.summarise(line(0, 2070, 2070), *window(500, 600))
    assert r["sm_mhz"] is None and r["samples"] == 0 and r["reasons"] == []


class FakeProc:
    def __init__(self, out):
        self.out, self.terminated = out, False

    def terminate(self):
        self.terminated = True

    def communicate(self, timeout=None):
        return self.out, None


def test_stop_reads_the_sampler_process():
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc = FakeProc("\n".join(line(t, 2070, 2070, swt="Active" if t == 50 else "Not Active") for t in range(0, 200, 50)))
    r = s.stop(*window(0, 150))
    assert s.proc.terminated and r["samples"] == 4 and r["reasons"] == ["sw_thermal_slowdown"]


def test_stop_without_nvidia_smi():
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc = None
    assert s.stop(0.0, 1.0)["reasons"] == ["nvidia-smi unavailable"]


def test_paper_context_block():
    """The bench line quotes what the paper gives about its runs (grid, step
    counts; no timing) and this run's throughput on that grid."""
    ctx = bench.paper_context(None)
    assert "600x150" in ctx["grid"] and "not reported" in ctx["timing"] and "here_on_that_grid" not in ctx
    ctx = bench.paper_context({"simulations": 108, "steps_per_case": 40000, "s_curves": 13.5})
    assert abs(ctx["here_on_that_grid"]["glups"] - 108 * 40000 * 600 * 150 / 13.5 / 1e9) < 1e-9
