"""Host-side helpers of bench.py that need no GPU: the DRAM traffic scaled
from single-kernel ncu captures with its source-hash guard, and the oracle
baseline spread over every host core."""
from __future__ import annotations

import json


def test_dram_traffic_scales_per_unit_and_checks_the_sources(tmp_path, monkeypatch):
    import bench

    srcs = ["lc_query.cu", "lc_internal.h"]
    prof = {"kernels": {"access": {
        "unit": "queries", "sources": srcs, "sources_sha256": bench.sources_sha256(srcs),
        "summary": "profiles/x.md",
        "captures": [{"workload": "a", "units_per_launch": 1e6, "dram_bytes_per_launch": 1e8},
                     {"workload": "b", "units_per_launch": 2e6, "dram_bytes_per_launch": 6e8}]}}}
    path = tmp_path / "t.json"
    path.write_text(json.dumps(prof))
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(path))
    tr, note = bench.dram_traffic("access", 1e8)
    assert abs(tr - 1e8 * (100 + 300) / 2) < 1e-3  # mean of 100 and 300 bytes per query
    assert "2 single-launch ncu captures" in note
    assert bench.dram_traffic("decode", 1e8) == (None, None)
    prof["kernels"]["access"]["sources_sha256"] = "0" * 64  # the sources changed since the capture
    path.write_text(json.dumps(prof))
    assert bench.dram_traffic("access", 1e8) == (None, None)


def test_oracle_all_cores_runs_the_sample_in_chunk_aligned_pieces():
    import os

    import numpy as np

    import bench
    import oracle
    from paper_2412_10770_gb300 import inputs

    oracle.build()
    cols = [inputs.column(g, 3 * 65536 + 123, seed=5, dtype=np.uint64) for g in ("lognormal", "clusters")]
    wall, procs = bench.oracle_all_cores(cols, 63, 1000)
    assert procs == (os.cpu_count() or 1)
    assert wall > 0
