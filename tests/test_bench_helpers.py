"""Host-side helpers of bench.py, on the CPU: the ncu traffic figure is reported only while the
strip kernel's sources hash to the captured ones; the clock sampler's parse keeps only the
samples written after it settled; the default step count is the workload's run length."""
import bench


def test_traffic_is_reported_only_for_the_captured_kernel_sources(monkeypatch):
    value, why = bench.measured_traffic("nls_well")
    assert value is not None and value > 0, why
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: "0" * 16)
    value, why = bench.measured_traffic("nls_well")
    assert value is None and "changed" in why
    value, why = bench.measured_traffic("no_such_workload")
    assert value is None


def test_clock_samples_before_the_timed_region_are_dropped(tmp_path):
    c = bench.Clocks.__new__(bench.Clocks)
    c.path = str(tmp_path / "clocks.csv")
    c.skip = 1
    rows = ["0, 1200, 2070, 300.0, 0x1, Not Active, Not Active, Not Active, Not Active",
            "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2070, 2070, 950.0, 0x4, Not Active, Not Active, Not Active, Active"]
    with open(c.path, "w") as f:
        f.write("\n".join(rows) + "\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c.proc = Done()
    c.f = open(c.path, "a")
    out = c.stop()
    assert out["samples"] == 2 and out["sm_mhz"] == 2070.0     # the 1200 MHz start-up sample is dropped
    assert out["reasons"] == ["sw_power_cap"]


def test_default_steps_are_the_workloads_run_length():
    assert bench.parse([]).steps == 200                          # nls_well: 200 steps
    assert bench.parse(["--workload", "gpe_batch"]).steps == 3
    assert bench.parse(["--steps", "7"]).steps == 7
