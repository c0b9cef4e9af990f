"""Host logic of the benchmark that decides what its JSON line reports: the
clock summary taken from nvidia-smi samples (median SM clock, maximum clock,
throttle reasons seen active) and the DRAM traffic read from a committed ncu
summary, which must be dropped once the kernel source no longer matches the
hash the summary records."""
import hashlib
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def sample(sm, smax=2070, hw="Not Active", hw_th="Not Active", sw_th="Not Active", cap="Not Active"):
    return f"0, {sm}, {smax}, 850.00, 0x0000000000000000, {hw}, {hw_th}, {sw_th}, {cap}"


def test_clock_summary_median_max_and_reasons():
    lines = [sample(2070), sample(2055, cap="Active"), sample(1980), sample(2070, smax=2070), sample(2040)]
    s = bench.ClockSampler.summarise(lines)
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 5
    assert s["reasons"] == ["sw_power_cap"]
    s = bench.ClockSampler.summarise([sample(1500, hw_th="Active"), sample(1600, hw="Active", sw_th="Active")])
    assert s["sm_mhz"] == 1550.0
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_skips_malformed_lines():
    lines = ["", "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active", "0, 2070, 2070",
             sample(2010)]
    s = bench.ClockSampler.summarise(lines)
    assert s["samples"] == 1 and s["sm_mhz"] == 2010.0 and s["reasons"] == []
    s = bench.ClockSampler.summarise([])
    assert s["sm_mhz"] is None and s["samples"] == 0 and s["reasons"] == ["no samples"]


def _fake_tree(tmp_path, src: bytes, sha_prefix: str, traffic="345.8e6"):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_2506_05558_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / "paper_2506_05558_gb300" / "csrc" / "render.cu").write_bytes(src)
    text = (f"# summary\n\nsource_sha256: {sha_prefix} (render.cu, first 16 hex digits)\n\n"
            f"| counter | value |\n|---|---|\n| traffic_bytes_per_view | {traffic} |\n")
    (tmp_path / "profiles" / bench.PROFILE_OF_STAGE["composite_bwd"]).write_text(text)


def test_profiled_traffic_scales_by_views_when_the_source_matches(tmp_path):
    src = b"__global__ void k() {}\n"
    _fake_tree(tmp_path, src, hashlib.sha256(src).hexdigest()[:16])
    assert bench.profiled_traffic("composite_bwd", 8, root=str(tmp_path)) == 8 * 345.8e6
    assert bench.profiled_traffic("sort", 8, root=str(tmp_path)) is None  # no summary for that stage
    assert bench.profiled_traffic("render_fwd", 8, root=str(tmp_path)) is None  # summary file absent


def test_profiled_traffic_is_dropped_after_a_source_change(tmp_path):
    src = b"__global__ void k() {}\n"
    _fake_tree(tmp_path, src + b"// edited\n", hashlib.sha256(src).hexdigest()[:16])
    assert bench.profiled_traffic("composite_bwd", 8, root=str(tmp_path)) is None


def test_committed_summaries_name_their_source_and_command():
    """Every committed kernel summary records the hash of the source it was
    taken on (16 hex digits of an existing file) and the ncu command, with the
    clocks left alone."""
    pdir = os.path.join(ROOT, "profiles")
    for name in sorted(os.listdir(pdir)):
        text = open(os.path.join(pdir, name)).read()
        assert "ncu" in text, name
        for cmd in re.findall(r"^\s*ncu .*$", text, flags=re.M):
            assert "--clock-control none" in cmd, (name, cmd)
        for sha, path in re.findall(r"source_sha256: ([0-9a-f]+) \(([^,]+),", text):
            assert len(sha) == 16, name
            assert os.path.exists(os.path.join(ROOT, path)), (name, path)
