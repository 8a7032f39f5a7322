"""The clock record of bench.py on CPU: nvidia-smi samples (csv, noheader,
nounits) become the median SM clock under load, the maximum clock and the
throttle reasons seen active, as the bench line's `clocks` key reports them."""
import os
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _clocks_from(lines):
    c = bench.Clocks(0)
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    f.write("\n".join(lines) + "\n")
    f.flush()
    c.f, c.proc = f, _Done()
    return c.stop()


def test_median_clock_and_no_reasons():
    rows = [f"0, {mhz}, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
            for mhz in (2070, 2055, 2070, 1980, 2070)]
    d = _clocks_from(rows)
    assert d == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}


def test_reasons_seen_in_any_sample():
    rows = ["0, 2070, 2070, 1300, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 1800, 2070, 1400, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
            "0, 1950, 2070, 1350, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"]
    d = _clocks_from(rows)
    assert d["sm_mhz"] == 1950.0 and d["samples"] == 3
    assert d["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_unreadable_samples_give_no_record():
    assert _clocks_from(["garbage", ""]) is None
    c = bench.Clocks(0)
    assert c.stop() is None  # never started


def test_samples_filtered_to_the_timed_region():
    import datetime
    base = datetime.datetime(2026, 12, 4, 8, 40, 0)

    def row(mhz, dt):
        ts = (base + datetime.timedelta(seconds=dt)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"0, {mhz}, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active, {ts}"

    rows = [row(1200, 0.0), row(2070, 1.0), row(2055, 1.1), row(2070, 1.2), row(1300, 3.0)]
    c = bench.Clocks(0)
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    f.write("\n".join(rows) + "\n")
    f.flush()
    c.f, c.proc = f, _Done()
    t0 = base.timestamp()
    d = c.stop(window=(t0 + 0.95, t0 + 1.25))
    assert d["samples"] == 3 and d["samples_in_timed_region"] == 3
    assert d["sm_mhz"] == 2070.0
