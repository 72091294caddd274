"""Host-side logic of bench.py: the clock-sample summary and the attribution
of an ncu per-launch list to kernel families (no GPU needed)."""
import datetime
import json

import pytest

import bench


def _line(t, sm, mx, *reasons):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    flags = ["Active" if r else "Not Active" for r in reasons]
    return f"{ts}, 0, {sm}, {mx}, 900.0, 0x0, " + ", ".join(flags)


def test_summarize_clocks_window_and_reasons():
    t0 = 1_700_000_000.0
    text = "\n".join([
        _line(t0 - 5.0, 1200, 2070, 0, 0, 0, 0),   # before the window: ignored
        _line(t0 + 0.1, 2070, 2070, 0, 0, 0, 0),
        _line(t0 + 0.2, 2040, 2070, 0, 0, 0, 1),   # sw_power_cap
        _line(t0 + 0.3, 2070, 2070, 0, 0, 0, 0),
        _line(t0 + 9.0, 900, 2070, 1, 0, 0, 0),    # after: ignored
        "garbage line",
    ])
    c = bench.summarize_clocks(text, t0, t0 + 0.35)
    assert c["samples"] == 3
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]


def test_summarize_clocks_short_window_takes_nearest_sample():
    t0 = 1_700_000_000.0
    text = "\n".join([_line(t0 - 3.0, 1000, 2070, 0, 0, 0, 0), _line(t0 + 2.0, 1980, 2070, 0, 0, 0, 0)])
    c = bench.summarize_clocks(text, t0 + 1.0, t0 + 1.01)
    assert c["samples"] == 1 and c["sm_mhz"] == 1980.0


def test_summarize_clocks_no_samples():
    c = bench.summarize_clocks("", 0.0, 1.0)
    assert c["sm_mhz"] is None and c["samples"] == 0


def _ncu_rows(launches):
    hdr = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
           "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]
    out = [",".join(f'"{h}"' for h in hdr)]
    for i, (name, t, rd, wr) in enumerate(launches):
        for metric, val in [("gpu__time_duration.sum", t), ("dram__bytes_read.sum", rd),
                            ("dram__bytes_write.sum", wr)]:
            row = [str(i), "1", "python", "h", name, "1", "7", "(256, 1, 1)", "(10, 1, 1)", "0", "10.3",
                   "Command line profiler metrics", metric, "", str(val)]
            out.append(",".join(f'"{x}"' for x in row))
    return "\n".join(out) + "\n"


def test_write_traffic_attributes_launches_to_families(tmp_path, monkeypatch, capsys):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: "d1")
    (tmp_path / "profiles").mkdir()
    launches = [
        ("void at::vectorized_elementwise_kernel<4>(int)", 5000, 1e6, 1e6),   # the L2 flush: not ours
        ("void cfc::k_rowop<float, 64, 1, cfc::<unnamed>::OpSpmvDot<float>, 1, 0>(cfc::LevelView)", 40000,
         3e7, 1e6),
        ("void cfc::k_rowop<float, 64, 1, cfc::<unnamed>::OpSpmvDot<float>, 1, 0>(cfc::LevelView)", 38000,
         3.2e7, 1e6),
        ("cfc::<unnamed>::k_merge(const int *)", 9000, 4e6, 2e6),
    ]
    csv_path = tmp_path / "l.csv"
    csv_path.write_text(_ncu_rows(launches))
    log_path = tmp_path / "log.json"
    log_path.write_text(json.dumps({"workload": "w", "steps": 1, "source_digest": "d1",
                                    "families": ["spmv_fine", "spmv_fine", "setup"]}))
    bench.write_traffic(str(csv_path), str(log_path))
    j = json.loads((tmp_path / "profiles" / "traffic.json").read_text())
    spmv = j["w"]["spmv_fine"]
    assert spmv["launches"] == 2 and spmv["source_digest"] == "d1"
    assert spmv["dram_bytes_per_launch"] == pytest.approx((3.1e7 + 3.3e7) / 2)
    assert "OpSpmvDot" in spmv["kernel"]
    assert j["w"]["setup"]["dram_bytes_per_launch"] == pytest.approx(6e6)
    assert "spmv_fine" in capsys.readouterr().out
    # a log from other kernel sources, or a launch count that does not match, is refused
    log_path.write_text(json.dumps({"workload": "w", "steps": 1, "source_digest": "old",
                                    "families": ["spmv_fine", "spmv_fine", "setup"]}))
    with pytest.raises(SystemExit):
        bench.write_traffic(str(csv_path), str(log_path))
    log_path.write_text(json.dumps({"workload": "w", "steps": 1, "source_digest": "d1", "families": ["setup"]}))
    with pytest.raises(SystemExit):
        bench.write_traffic(str(csv_path), str(log_path))


def test_read_traffic_checks_the_digest(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        {"w": {"smooth_fine": {"source_digest": "d1", "dram_bytes_per_launch": 5.0, "kernel": "k"}}}))
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: "d1")
    assert bench.read_traffic("w", "smooth_fine") == (5.0, "k", None)
    assert bench.read_traffic("w", "spmv_fine") == (None, None, None)
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: "d2")
    assert bench.read_traffic("w", "smooth_fine") == (None, None, None)
