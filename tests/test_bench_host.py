"""Host-side logic of bench.py, on CPU:
* the workload description follows --N;
* --workloads accepts the secondary workloads by name and rejects others;
* the DRAM traffic of the profiled kernel is reported only while the kernel
  sources hash to the value recorded with the ncu capture, and only for the
  workload size it was captured on (else null in the bench line).
"""
import json
import sys

import pytest

import bench


def test_workload_description_follows_N():
    assert bench.workload(1 << 20).startswith("N=M=2^20 ")
    assert bench.workload(1 << 16).startswith("N=M=2^16 ")
    assert bench.workload(1000).startswith("N=M=1000 ")


def test_workloads_option(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workloads", "real_exponents,laplace"])
    args = bench.parse()
    assert set(args.workloads.split(",")) == {"real_exponents", "laplace"}
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    assert tuple(bench.parse().workloads.split(",")) == bench.SECONDARY
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workloads", "laplace,bogus"])
    with pytest.raises(SystemExit):
        bench.parse()


def _tree(root, src_text, recorded_hash, N):
    csrc = root / "paper_1606_03255_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text(src_text)
    prof = root / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.json").write_text(json.dumps({
        "source_hash": recorded_hash, "N": N,
        "kernels": {"fft_pass1": {"dram_bytes_per_launch": 123.0, "launches": 9}}}))


def test_traffic_only_for_the_captured_sources_and_size(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _tree(tmp_path, "kernel v1\n", "placeholder", 1 << 20)
    h1 = bench.source_hash()
    assert bench.ncu_traffic("fft_pass1", 1 << 20) is None       # recorded for other sources
    rec = tmp_path / "profiles" / "ncu_traffic.json"
    d = json.loads(rec.read_text())
    d["source_hash"] = h1
    rec.write_text(json.dumps(d))
    assert bench.ncu_traffic("fft_pass1", 1 << 20) == 123.0
    assert bench.ncu_traffic("fft_pass1", 1 << 16) is None       # another workload size
    assert bench.ncu_traffic("fft_pass2", 1 << 20) is None       # a kernel not captured
    (tmp_path / "paper_1606_03255_gb300" / "csrc" / "k.cu").write_text("kernel v2\n")
    assert bench.source_hash() != h1
    assert bench.ncu_traffic("fft_pass1", 1 << 20) is None       # sources changed since


def test_method_bytes_counts_every_grid_once_per_rhs():
    # 16 n bytes (complex64: one write and one read) per right-hand side of
    # every NFFT; a band split into P sub-bands has P grids of band_n points;
    # direct and empty bands add nothing; the last band has one right-hand side
    info = {"levels": 4, "band_route": [0, 1, 2, 1, 1], "band_n": [0, 1 << 10, 1 << 12, 1 << 13, 1 << 14],
            "band_parts": [1, 1, 1, 3, 1]}
    q = 5
    expect = q * 16 * (1 << 10) + q * 3 * 16 * (1 << 13) + 1 * 16 * (1 << 14)
    assert bench.method_bytes(info, q) == expect
    assert bench.method_bytes(info, q, n_min=4096) == q * 3 * 16 * (1 << 13) + 16 * (1 << 14)
