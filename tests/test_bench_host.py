"""Host-side logic of bench.py and of the binding's error mapping (no GPU)."""
import json
import os

import pytest

from tests.conftest import ROOT


@pytest.fixture(scope="module")
def bench():
    import importlib
    import sys
    sys.path.insert(0, ROOT)
    return importlib.import_module("bench")


def test_traffic_figures_follow_the_kernel_source(bench, tmp_path, monkeypatch):
    """roofline.traffic comes from a committed capture of the same workload
    (or of its reduced-scale copy) only while the kernel source is the one
    that was captured."""
    import hashlib
    src = tmp_path / "k.cu"
    src.write_text("// kernel source at capture time\n")
    cap = {"captures": [{"workload": "cl3s", "scales_to": "cl3", "source_file": "k.cu",
                         "source_sha256": hashlib.sha256(src.read_bytes()).hexdigest(),
                         "kernels": {"heavy": {"kernel": "k_heavy1", "dram_bytes_per_wedge": 2.5}}}]}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(cap))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("cl3", "heavy", 1000.0) == pytest.approx(2500.0)   # scaled from the small copy
    assert bench.measured_traffic("cl3s", "heavy", 10.0) == pytest.approx(25.0)
    assert bench.measured_traffic("cl2", "heavy", 1000.0) is None      # no capture of that workload
    assert bench.measured_traffic("cl3", "medium", 1000.0) is None     # no capture of that kernel
    src.write_text(src.read_text() + "// changed\n")                  # the kernel changed since the capture
    assert bench.measured_traffic("cl3", "heavy", 1000.0) is None
    # the committed file parses and names existing sources
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        t = json.load(f)
    for c in t["captures"]:
        assert os.path.exists(os.path.join(ROOT, c["source_file"]))
        assert all(k["dram_bytes_per_wedge"] > 0 for k in c["kernels"].values())


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


def test_noalloc_mode_runs_a_graph_within_its_scratch(bench, monkeypatch):
    """--mode noalloc times pb_count_noalloc; the 20M x 60M default has a side
    beyond its fixed scratch, so the mode falls back to the 1M x 4M graph."""
    import sys
    monkeypatch.setattr(sys, "argv", ["bench.py", "--mode", "noalloc"])
    a = bench.parse()
    assert a.mode == "noalloc" and bench.noalloc_workload(a.workload) == "cl2"
    assert bench.noalloc_workload("cl3s") == "cl3s" and bench.noalloc_workload("er1") == "er1"
    assert "cl2" in bench.WORKLOADS
