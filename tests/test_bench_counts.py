"""The per-step operation counts bench.py's roofline uses were measured
(ncu sass counters) on the kernel sources as committed: the SHA-256 over
those sources matches the one recorded beside the counts, so the reported
roofline fraction is not computed from stale counts."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.mark.parametrize("precision", [64, 32])
def test_count_constants_match_kernel_sources(precision):
    import bench
    assert bench.kernel_sources_sha256(precision) == bench.COUNTS_SOURCE_SHA256[precision]
