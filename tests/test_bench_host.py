"""Host-side logic of bench.py and of the binding's error mapping (no GPU)."""
import json
import os
import shutil

import pytest

from tests.conftest import ROOT


@pytest.fixture(scope="module")
def bench():
    import importlib
    import sys
    sys.path.insert(0, ROOT)
    return importlib.import_module("bench")


def test_traffic_figures_follow_the_kernel_source(bench, tmp_path, monkeypatch):
    """roofline.traffic comes from the committed capture only while the
    kernel source is the one that was captured."""
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        t = json.load(f)
    for k in ("light", "medium", "heavy"):
        assert k in t["kernels"] and t["kernels"][k]["dram_bytes_per_wedge"] > 0
    # a private copy of the layout: same capture, same source
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(ROOT, "profiles", "traffic.json"), tmp_path / "profiles" / "traffic.json")
    src = tmp_path / t["source_file"]
    src.parent.mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, t["source_file"]), src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench.measured_traffic("medium", 1000.0)
    assert got == pytest.approx(1000.0 * t["kernels"]["medium"]["dram_bytes_per_wedge"])
    assert bench.measured_traffic("sort", 1000.0) is None        # no capture of that kernel
    src.write_text(src.read_text() + "\n// changed\n")           # the kernel changed since the capture
    assert bench.measured_traffic("medium", 1000.0) is None


def test_clock_summary_reads_samples_and_reasons(bench):
    c = bench.Clocks(0, enabled=False)
    c.lines = ["2070, 2070, 800.5, 0x0, Not Active, Not Active, Not Active, Not Active",
               "1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               "2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    s = c.summary()
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = []
    assert c.summary() is None


def test_model_bytes_per_wedge(bench):
    # 4 B second endpoint; + 4 B per-vertex traffic; + 8 B read and 8 B write of the edge counter
    assert bench.BYTES_PER_WEDGE == {"all": 20, "edge": 20, "global": 4, "vertex": 8}


def test_default_workload_is_the_largest_single_gpu_configuration(bench, monkeypatch):
    """With no options the bench counts the 20M x 60M graph, per-edge, with
    batch aggregation inside a 16 GiB scratch budget."""
    import sys
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.workload == "cl3" and a.agg == "batch" and a.outputs == "edge" and a.scratch == 16 << 30
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "cl2", "--agg", "hash", "--scratch-gib", "2"])
    a = bench.parse()
    assert a.agg == "hash" and a.outputs == "all" and a.scratch == 2 << 30


def test_cpu_baseline_times_the_oracle_on_a_bounded_sample(bench):
    r = bench.cpu_baseline("er1", nthreads=2)
    assert r["kind"] == "oracle" and r["cores"] == 2 and r["value"] > 0 and r["W"] > 0
    assert "er" in r["sample"] and f"W={r['W']}" in r["sample"]
    for wl, sp in bench.SAMPLES.items():   # every sample is the workload's recipe at a smaller scale
        assert sp["step"]["m"] <= sp["baseline"]["m"]


def test_status_codes_raise_with_the_library_message():
    import paper_1907_08607_gb300 as pb
    from paper_1907_08607_gb300 import build as b
    pb.load_library(b.build())
    pb._check(0)
    for code in (1, 2, 3, 4, 5, 6):
        with pytest.raises(pb.PBError) as ei:
            pb._check(code)
        assert ei.value.status == code
        assert pb.STATUS[code] in str(ei.value)
