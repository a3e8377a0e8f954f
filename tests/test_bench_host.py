"""Host-side pieces of bench.py (no GPU): the recorded DRAM traffic is only
reported for the kernel sources it was captured on, the committed records
point at existing summaries, and the workload line names what it measures."""
import json
import os

import bench
from paper_2406_16091_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_records_are_well_formed():
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert set(d) >= {"k_interact_direct", "binning"}
    for key, rec in d.items():
        assert len(rec["source_hash"]) == 16
        assert rec["dram_bytes_per_launch"] > 0
        assert os.path.exists(os.path.join(ROOT, rec["capture"])), key


def test_traffic_only_for_matching_sources(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    h1 = bench.source_hash([str(src)])
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({"k": {"source_hash": h1, "dram_bytes_per_launch": 123}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("k", h1)["dram_bytes_per_launch"] == 123
    src.write_text("kernel v2")
    h2 = bench.source_hash([str(src)])
    assert h2 != h1
    assert bench.recorded_traffic("k", h2) is None
    assert bench.recorded_traffic("other", h1) is None


def test_workload_line_names_the_layout():
    class Args:
        algo, precision, gpus, flush_mb = "tiled", "fp32", 1, 512

    for name in ("scale", "clustered"):
        w = W.WORKLOADS[name]
        cfg = bench.workload_config(w, Args)
        assert cfg["workload"].startswith(name + ":")
        assert w.layout in cfg["workload"]
        assert cfg["n_particles"] == w.n and cfg["r_c"] == w.rc


def test_binning_bytes_follow_the_algorithmic_formula():
    """48 bytes per particle and 12 per cell: 103.8 MB at 2,097,152
    particles in 64^3 cells; the figure with the P record is separate."""
    n, C = 2097152, 64 ** 3
    assert bench.binning_bytes(n, C) == 48 * n + 12 * C == 103_809_024
    assert bench.binning_bytes_with_p(n, C) > bench.binning_bytes(n, C)


def test_binning_paths_match_the_header_and_sources():
    """Each --binning choice sets the PI_OPT_BINNING value include/pi.h
    gives it, and names kernels and sources that exist."""
    import re

    header = open(os.path.join(ROOT, "include", "pi.h")).read()
    enum = re.search(r"enum \{ (PI_BIN_[^}]*)\};", header).group(1)
    values = {k.strip(): int(v) for k, v in (e.split("=") for e in enum.split(",") if e.strip())}
    names = {"per_particle": "PI_BIN_PER_PARTICLE", "bucketed": "PI_BIN_BUCKETED", "radix": "PI_BIN_RADIX"}
    assert set(bench.BINNING_PATHS) == set(names)
    csrc = os.path.join(ROOT, "paper_2406_16091_gb300", "csrc")
    for choice, path in bench.BINNING_PATHS.items():
        assert path["option"] == values[names[choice]]
        text = ""
        for f in path["files"]:
            text += open(os.path.join(csrc, f)).read()
        for kern in path["kernels"]:
            assert re.search(r"\b%s\b" % kern, text), (choice, kern)
