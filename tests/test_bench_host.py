"""Host-side bookkeeping of the benchmark (no GPU): which source a kernel's
committed ncu traffic belongs to, when that traffic may be reported, the
clock record taken during the timed region, and the whole-job rates."""
import json
import os

import pytest

import bench


def test_kernel_families():
    assert bench.kernel_family("k_sweep") == "psa"
    assert bench.kernel_family("k_sample") == "psa"
    assert bench.kernel_family("k2_group") == "two_level"
    assert bench.kernel_family("k_os_level") == "os_nd"
    assert bench.kernel_family("k_pp_merge") == "psa_plus"
    for fam, files in bench.KERNEL_SOURCES.items():
        assert all(os.path.exists(os.path.join(bench.ROOT, f)) for f in files), fam
        assert len(bench.source_sha(fam)) == 16


def test_traffic_only_for_the_source_it_was_taken_on(monkeypatch):
    """A committed entry scales to the launch by its units while its source is
    unchanged, and is withheld (None) once the source differs."""
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        entries = json.load(f)["kernels"]
    current = {k: e for k, e in entries.items() if e["source_sha"] == bench.source_sha(bench.kernel_family(k))}
    if not current:
        pytest.skip("no entry taken on the current sources")
    name, e = next(iter(current.items()))
    assert bench.traffic_for(name, 10 ** 9) == pytest.approx(e["dram_bytes_per_unit"] * 10 ** 9)
    monkeypatch.setattr(bench, "source_sha", lambda family="psa": "0" * 16)
    assert bench.traffic_for(name, 10 ** 9) is None
    assert bench.traffic_for("no_such_kernel", 10) is None


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_record_median_and_reasons(tmp_path):
    """nvidia-smi lines (index, sm, max sm, power, active mask, the four
    reasons): median SM clock, highest max clock, every reason seen active."""
    c = bench.Clocks(0, enabled=False)
    c.path = str(tmp_path / "clocks.csv")
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage line",
             "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    with open(c.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    c.proc, c.fh = _Proc(), open(str(tmp_path / "unused"), "w")
    rec = c.stop()
    assert rec == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    with open(c.path, "w") as f:
        f.write("0, 1200, 2070, 700, 0x8, Active, Not Active, Not Active, Not Active\n")
    c.proc, c.fh = _Proc(), open(str(tmp_path / "unused2"), "w")
    assert c.stop()["reasons"] == ["hw_slowdown"]
    assert bench.Clocks(0, enabled=False).stop() is None


def test_job_rates_are_whole_job():
    # 4 replicas x 3 steps of 10^9 weights in 150 ms; 4 x 3 x 10^9 samples in 300 ms
    gw, gs = bench.job_rates(4, 3, 10 ** 9, 10 ** 9, 150.0, 300.0)
    assert gw == pytest.approx(80.0) and gs == pytest.approx(40.0)
