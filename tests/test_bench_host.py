"""Host-side logic of the benchmark that needs no GPU: the provenance check
that decides whether the committed ncu traffic figure still describes the
kNN kernel, the clock-sample summary that accepts or rejects a timed run,
the GPU index a rank takes from CUDA_VISIBLE_DEVICES, and that every
command the profile summaries give is one this benchmark accepts."""
import json
import os
import re

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _local_includes(path, seen):
    """Every repository file `path` includes, followed transitively."""
    if path in seen:
        return seen
    seen.add(path)
    src = open(os.path.join(ROOT, path)).read()
    for name in re.findall(r'^\s*#include\s+"([^"]+)"', src, re.M):
        for d in (os.path.dirname(path), "include"):
            cand = os.path.normpath(os.path.join(d, name))
            if os.path.exists(os.path.join(ROOT, cand)):
                _local_includes(cand, seen)
                break
        else:
            raise AssertionError(f"{path} includes {name}, found nowhere in the repository")
    return seen


def test_traffic_record_names_every_file_the_kernel_is_compiled_from():
    rec = json.load(open(bench.TRAFFIC_RECORD))
    kernel_src = "paper_1001_3411_gb300/csrc/knn_cg.cu"
    needed = _local_includes(kernel_src, set())
    assert kernel_src in needed and "include/hop.h" in needed
    assert needed <= set(rec["sources"]), needed - set(rec["sources"])
    assert rec["particles"] > (129 << 20) // 16          # positions alone larger than L2
    assert rec["traffic_bytes_per_particle"] == pytest.approx(
        (rec["dram_read_bytes"] + rec["dram_write_bytes"]) / rec["particles"], abs=0.01)


def test_traffic_figure_is_dropped_once_a_source_changes(tmp_path, monkeypatch):
    rec = json.load(open(bench.TRAFFIC_RECORD))
    # a record whose hashes match the files as they are now is used
    good = dict(rec, sources=bench.source_hashes(rec["sources"].keys()))
    p = tmp_path / "good.json"
    p.write_text(json.dumps(good))
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(p))
    tpp, basis = bench.knn_traffic_per_particle()
    assert tpp == rec["traffic_bytes_per_particle"] and basis == rec["basis"]
    # one stale hash: no traffic figure
    stale = json.loads(json.dumps(good))
    first = sorted(stale["sources"])[0]
    stale["sources"][first] = "0" * 16
    p.write_text(json.dumps(stale))
    tpp, why = bench.knn_traffic_per_particle()
    assert tpp is None and "changed" in why
    # no record at all
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(tmp_path / "missing.json"))
    assert bench.knn_traffic_per_particle() == (None, "no capture")


def _summary(lines):
    s = bench.ClockSampler(0)
    try:
        s.f.write("".join(l + "\n" for l in lines))
        return s.summary()
    finally:
        s.f.close()
        os.unlink(s.f.name)


def test_clock_summary_median_and_reasons():
    ok = "0, {sm}, 2070, {w}, 0x0000000000000000, Not Active, Not Active, Not Active, {cap}"
    lines = [ok.format(sm=sm, w=w, cap="Not Active") for sm, w in ((2070, 500.5), (2055, 610.0), (1980, 700.25))]
    lines.append(ok.format(sm=2070, w=650.0, cap="Active"))
    s = _summary(lines)
    assert s["sm_mhz"] == pytest.approx((2070 + 2055) / 2)
    assert s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 4 and s["power_w_max"] == pytest.approx(700.25)
    # a thermal slowdown in any one sample is reported, which rejects the run
    hot = "0, 1500, 2070, 900, 0x0000000000000048, Not Active, Active, Not Active, Not Active"
    s = _summary(lines + [hot])
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    # a malformed or missing reading does not count as a sample value
    s = _summary(["0, [N/A], 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active"] + lines[:1])
    assert s["sm_mhz"] == 2070 and s["power_w_max"] == pytest.approx(500.5)


def test_clock_summary_without_samples():
    s = _summary([])
    assert s["samples"] == 0 and s["sm_mhz"] is None and s["reasons"] == ["no samples"]


def test_gpu_index_follows_visible_devices(monkeypatch):
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "5,2")
    assert bench.gpu_index(0) == 5 and bench.gpu_index(1) == 2
    assert bench.gpu_index(7) == 2                  # more ranks than listed: the last one
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "GPU-3f2a")
    assert bench.gpu_index(1) == 1                  # a UUID: the rank's ordinal
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES")
    assert bench.gpu_index(3) == 3


def test_profile_commands_are_accepted_by_the_benchmark(monkeypatch):
    """Each profile summary names the command that produced it; every
    `python bench.py ...` line there (also the one ncu wraps) must parse
    with the benchmark's own arguments."""
    import glob
    import shlex
    import sys
    prof = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert prof
    seen = 0
    for path in prof:
        text = open(path).read().replace("\\\n", " ")
        cmds = re.findall(r"python bench\.py[^\n`]*", text)
        assert cmds, f"{os.path.basename(path)} gives no bench.py command"
        for c in cmds:
            argv = shlex.split(c)[1:]
            monkeypatch.setattr(sys, "argv", argv)
            bench.parse()
            seen += 1
    assert seen >= len(prof)
