"""The benchmark's clock record: only the nvidia-smi samples taken inside the
timed region count (a throttle reason outside it does not reject the run);
a region shorter than the sampling interval keeps the sample nearest to its
middle; lines that do not parse are skipped."""
import datetime

import bench


class _FakeSmi:
    """Stands in for the nvidia-smi process: returns the given CSV lines."""

    def __init__(self, lines):
        self.lines = lines

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return "\n".join(self.lines), None


def _line(t, sm, reasons=("Not Active",) * 4):
    stamp = t.strftime("%Y/%m/%d %H:%M:%S.") + f"{t.microsecond // 1000:03d}"
    return ", ".join([stamp, str(sm), "2070", "0x0", *reasons])


def _clocks(monkeypatch, t0, t1, lines):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    c = bench.Clocks(0)
    c.t0, c.t1 = t0, t1
    c.proc = _FakeSmi(lines)
    return c.stop()


T = datetime.datetime(2026, 1, 1, 12, 0, 0)


def _at(ms):
    return T + datetime.timedelta(milliseconds=ms)


def test_only_samples_inside_the_region_count(monkeypatch):
    thermal = ("Not Active", "Active", "Not Active", "Not Active")
    lines = [_line(_at(10), 1200, thermal),            # before the region: ignored
             _line(_at(120), 2070), _line(_at(140), 2050),
             _line(_at(160), 2060, ("Not Active",) * 3 + ("Active",)),
             _line(_at(400), 900, thermal),            # after the region: ignored
             "garbage line"]
    out = _clocks(monkeypatch, _at(100), _at(200), lines)
    assert out["samples"] == 3 and out["samples_total"] == 5
    assert out["sm_mhz"] == 2060 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"]
    assert out["region_s"] == 0.1


def test_short_region_keeps_the_nearest_sample(monkeypatch):
    lines = [_line(_at(0), 1500), _line(_at(20), 2070), _line(_at(40), 1800)]
    out = _clocks(monkeypatch, _at(22), _at(26), lines)
    assert out["samples"] == 1 and out["sm_mhz"] == 2070


def test_no_samples_gives_no_record(monkeypatch):
    assert _clocks(monkeypatch, _at(0), _at(10), ["not,a,sample"]) is None
