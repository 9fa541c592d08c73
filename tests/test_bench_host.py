"""Host-side pieces of bench.py (no GPU): the hash of the sources the profiled passes are compiled
from, and the reading of the committed column-pass summary that feeds the roofline's traffic."""
import os

import bench


def test_kernel_sources_exist_and_hash_is_stable():
    root = os.path.join(bench.ROOT, "paper_2411_18591_gb300", "csrc")
    for name in bench.KERNEL_SOURCES:
        assert os.path.exists(os.path.join(root, name)), name
    h = bench.kernel_source_hash()
    assert len(h) == 16 and h == bench.kernel_source_hash()


def test_profiled_traffic_reads_the_summary_or_declines():
    # a summary whose hash matches gives its DRAM bytes per field; otherwise None (never a guess)
    t = bench.profiled_traffic("cols")
    text = open(os.path.join(bench.ROOT, "profiles", "cols_summary.md")).read()
    if f"source_hash: {bench.kernel_source_hash()}" in text:
        assert t is not None and 33.5e6 < t < 80e6  # at least the algorithmic 32 n^2 bytes of a 1024^2 field
    else:
        assert t is None
    assert bench.profiled_traffic("no_such_kernel") is None
