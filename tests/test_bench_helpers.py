"""Host-side helpers of bench.py that need no GPU: the traffic profile built
from an ncu --csv metrics log with its source-hash guard, and the oracle
baseline spread over every host core."""
from __future__ import annotations

import json


def _csv(rows):
    hdr = ['"ID"', '"Process ID"', '"Process Name"', '"Host Name"', '"Kernel Name"', '"Context"', '"Stream"',
           '"Block Size"', '"Grid Size"', '"Device"', '"CC"', '"Section Name"', '"Metric Name"', '"Metric Unit"',
           '"Metric Value"']
    out = ["==PROF== Connected to process 1", ",".join(hdr)]
    for i, kernel, metric, unit, value in rows:
        out.append(",".join(f'"{x}"' for x in (i, 1, "python", "127.0.0.1", kernel, 1, 7, "(256, 1, 1)",
                                               "(1216, 1, 1)", 0, "10.3", "Command line profiler metrics", metric,
                                               unit, value)))
    return "\n".join(out) + "\n"


def test_write_traffic_means_per_launch_and_maps_names(tmp_path):
    import bench

    dec = "void lcx::<unnamed>::decode_kernel<unsigned long>(lcx::ColView, unsigned long, unsigned long)"
    rng = "void lcx::<unnamed>::decode_ranges_kernel<unsigned long>(lcx::ColView, const unsigned long *)"
    other = "void at::native::vectorized_elementwise_kernel<4>(int, float)"
    rows = []
    for i, rd, wr, ns in ((0, 100, 1000, 2000), (1, 300, 3000, 4000)):
        rows += [(i, dec, "dram__bytes_read.sum", "byte", f"{rd:,}"),
                 (i, dec, "dram__bytes_write.sum", "byte", f"{wr:,}"),
                 (i, dec, "gpu__time_duration.sum", "ns", f"{ns:,}")]
    rows += [(2, rng, "dram__bytes_read.sum", "Kbyte", "2"), (2, rng, "dram__bytes_write.sum", "byte", "0"),
             (2, rng, "gpu__time_duration.sum", "usecond", "5"),
             (3, other, "dram__bytes_read.sum", "byte", "7"), (3, other, "dram__bytes_write.sum", "byte", "7"),
             (3, other, "gpu__time_duration.sum", "ns", "7")]
    src = tmp_path / "t.csv"
    src.write_text(_csv(rows))
    out = tmp_path / "t.json"
    prof = bench.write_traffic(str(src), "cmd", str(out))
    assert json.loads(out.read_text()) == prof
    k = prof["kernels"]
    assert set(k) == {"decode", "decode_ranges"}
    assert k["decode"]["launches"] == 2
    assert k["decode"]["dram_read_bytes_per_launch"] == 200
    assert k["decode"]["dram_bytes_per_launch"] == 200 + 2000
    assert abs(k["decode"]["ms_per_launch_under_ncu"] - 0.003) < 1e-12
    assert k["decode_ranges"]["dram_bytes_per_launch"] == 2000
    assert prof["source_sha256"] == bench.kernel_sources_sha256()


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
