"""Host logic of bench.py that needs no GPU: the clock record taken during
the timed region and the lookup of the committed DRAM figure, which must be
dropped once the kernel sources differ from the ones it was measured on."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


class _Thread:
    def join(self, timeout=None):
        pass


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc, s._t, s.lines = _Proc(), _Thread(), list(lines)
    return s


def _line(sm, smax=2070, power=900.0, hw="Not Active", hwt="Not Active", swt="Not Active",
          cap="Not Active"):
    return f"0, {sm}, {smax}, {power}, 0x0, {hw}, {hwt}, {swt}, {cap}"


def test_clock_record_median_under_load_and_reasons():
    # idle samples before the kernels start (below half the top clock) are
    # left out of the median; a power cap seen once is reported
    lines = [_line(345), _line(345)] + [_line(f) for f in (1965, 1980, 1950, 2010)]
    lines.append(_line(1935, cap="Active"))
    rec = _sampler(lines).stop()
    assert rec["sm_mhz"] == 1965.0
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
    assert rec["samples"] == 7
    assert rec["power_w_max"] == 900.0


def test_clock_record_thermal_reasons_and_bad_lines():
    lines = ["", "garbage", "0, [N/A], 2070, 1.0, 0x0, a, b, c, d",
             _line(1900, hwt="Active"), _line(1920, hw="Active", swt="Active")]
    rec = _sampler(lines).stop()
    assert rec["sm_mhz"] == 1910.0
    assert rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert rec["samples"] == 2


def test_clock_record_without_samples_or_tool():
    assert _sampler([]).stop()["reasons"] == ["no samples"]
    s = bench.ClockSampler(0)          # nvidia-smi never started
    assert s.stop() == {"sm_mhz": None, "sm_max_mhz": None,
                        "reasons": ["nvidia-smi unavailable"]}


def _record():
    p = os.path.join(ROOT, "profiles", "path_kernel_elliptic3d_4096x1e5_dram.md")
    fields = {}
    with open(p) as f:
        for line in f:
            if ":" in line and not line.startswith(("#", "|", " ")):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
    return fields


def test_dram_record_used_only_for_the_measured_sources(monkeypatch):
    rec = _record()
    sha = rec["kernel_source_sha1"]
    assert len(sha) == 16 and int(sha, 16) >= 0
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: sha)
    assert bench._ncu_traffic() == int(rec["dram_bytes_per_launch"])
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench._ncu_traffic() is None


def test_kernel_source_hash_covers_every_listed_file(tmp_path, monkeypatch):
    # the hash changes when any one of the hashed sources changes
    for f in bench.KERNEL_SOURCES:
        d = tmp_path / os.path.dirname(f)
        d.mkdir(parents=True, exist_ok=True)
        (tmp_path / f).write_bytes(open(os.path.join(ROOT, f), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    assert h0 == bench.kernel_source_hash()
    seen = {h0}
    for f in bench.KERNEL_SOURCES:
        p = tmp_path / f
        orig = p.read_bytes()
        p.write_bytes(orig + b"\n")
        seen.add(bench.kernel_source_hash())
        p.write_bytes(orig)
    assert len(seen) == 1 + len(bench.KERNEL_SOURCES)
    assert bench.kernel_source_hash() == h0
