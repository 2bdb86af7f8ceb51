"""Host-side checks of the benchmark's algorithmic work counts (no GPU): the
per-unit figures the roofline fractions divide by."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_preprocess_bytes_per_gaussian():
    # logit + centre in, depth + count out: 24 B; + scales and quaternion past the
    # opacity test: 28 B; + SH in (192 B) and the 52 B record out when visible
    assert bench.preprocess_bytes(1, 0, 0) == 24
    assert bench.preprocess_bytes(1, 1, 0) == 52
    assert bench.preprocess_bytes(1, 1, 1) == 296
    assert bench.preprocess_bytes(10, 7, 5) == 10 * 24 + 7 * 28 + 5 * 244


def test_cull_bytes():
    assert bench.cull_bytes(1, 0) == 24
    assert bench.cull_bytes(0, 1) == 12


def test_segmented_sort_counts():
    # 1080p: 120 x 68 tiles, 13 tile bits above bit 31 -> two partition passes
    assert bench.seg_partition_passes(31 + 13) == 2
    # 2160p: 240 x 135 tiles, 15 tile bits -> two passes
    assert bench.seg_partition_passes(31 + 15) == 2
    assert bench.seg_sort_bytes(1000, 44) == 1000 * (2 * 32 + 32)
    # 3 launches per partition pass + bounds + local sort
    assert bench.seg_sort_launches(44) == 8
