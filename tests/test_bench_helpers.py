"""Host logic of bench.py: the DRAM traffic it reports for the forward DP is
taken from the committed ncu summary only while that summary was captured on
the current DP kernel source (else the line carries null)."""
import json

import bench


def test_traffic_follows_the_dp_source_hash(tmp_path, monkeypatch):
    summary = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(summary))
    assert bench.traffic_for_current_kernel() is None          # no summary
    summary.write_text(json.dumps({"dp_source_sha": bench.dp_source_sha(),
                                   "dram_bytes_per_forward_pass": 1234}))
    assert bench.traffic_for_current_kernel() == 1234
    summary.write_text(json.dumps({"dp_source_sha": "0" * 16, "dram_bytes_per_forward_pass": 1234}))
    assert bench.traffic_for_current_kernel() is None          # taken on another source


def test_dp_source_hash_covers_the_dp_section_only(tmp_path, monkeypatch):
    src = open(bench.KERNEL_SOURCE).read()
    head, rest = src.split("// The DP kernel", 1)
    copy = tmp_path / "k.cu"
    monkeypatch.setattr(bench, "KERNEL_SOURCE", str(copy))
    copy.write_text(src)
    base = bench.dp_source_sha()
    copy.write_text(head + "// an edit before the DP section\n// The DP kernel" + rest)
    assert bench.dp_source_sha() == base
    dp, tail = rest.split("// Issue-rate probe", 1)
    copy.write_text(head + "// The DP kernel" + dp + "// an edit in it\n// Issue-rate probe" + tail)
    assert bench.dp_source_sha() != base
