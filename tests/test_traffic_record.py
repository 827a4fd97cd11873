"""The DRAM traffic record that bench.py reports beside the FP64 roofline: well formed, and
taken from the kernel text as it stands (bench.py reports null traffic otherwise)."""
import json
import os

import bench


def test_traffic_record_matches_kernel_source():
    rec = json.load(open(bench.TRAFFIC_FILE))
    for key in ("kernel", "source", "function", "kernel_source_sha256_16", "command", "captured_case",
                "scaling", "bytes_per_launch", "summary"):
        assert key in rec, key
    assert rec["bytes_per_launch"] > 0
    assert os.path.exists(os.path.join(bench.ROOT, rec["summary"]))
    assert "--clock-control none" in rec["command"]
    assert rec["kernel_source_sha256_16"] == bench.kernel_source_digest(rec["source"], rec["function"])
