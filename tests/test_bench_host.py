"""Host-side parts of bench.py's CPU baseline, on CPU: the oracle's level 0
computed in z-slabs on threads equals the oracle's level 0 of the whole
volume (area-box footprints split only where they fill whole output slices),
and the histogram of z-slabs adds up to the whole volume's."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("shape,M", [((90, 23, 31), (16, 11, 32)), ((64, 20, 20), (10, 10, 16)),
                                     ((450, 18, 14), (9, 7, 64))])
def test_threaded_level0_equals_whole(orc, shape, M):
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(sum(shape))
    vol = rng.integers(0, 4096, size=shape).astype(np.uint16)
    keep = orc.keep_threshold(4096, 700)
    level, nslab = bench.oracle_level0_threaded(vol, 12, M, keep, 4)
    assert nslab > 1
    assert np.array_equal(level, orc.downsample(vol, 12, M, keep))


def test_threaded_histogram_adds_up(orc):
    rng = np.random.default_rng(3)
    vol = rng.integers(0, 5000, size=(37, 19, 23)).astype(np.uint16)
    whole, ov = orc.histogram(vol, 12, 4096)
    zs = np.linspace(0, 37, 6).astype(int)
    parts = [orc.histogram(vol, 12, 4096, int(zs[i]), int(zs[i + 1])) for i in range(5)]
    assert np.array_equal(sum(p[0] for p in parts), whole) and sum(p[1] for p in parts) == ov


def test_batch_launch_count():
    """The batched pass: 3 batched prepare launches per 64 volumes, the keep
    tables in one, a level-0 kernel per volume, 3 render kernels and one view
    upload per 128 views."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.batch_launches_per_step(64, 768) == 3 + 1 + 64 + 3 + 6
    assert bench.batch_launches_per_step(65, 1) == 6 + 1 + 65 + 3 + 1
