"""Pins of the CPU oracle's slicemap levels and atlas layout.

Integer area-box downsampling (reading: footprint [floor(iN/M), floor((i+1)N/M))
per axis, mean rounded half up) checked against a numpy block reduction for
integer factors, invariants for non-integer ones, and a hand-placed atlas.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_constant_volume_stays_constant(orc):
    for dims in [(3, 2, 4), (1, 1, 1), (7, 5, 6)]:
        vol = np.full((6, 5, 7), 123, np.uint8)
        lv = orc.downsample(vol, 8, dims)
        assert lv.shape == (dims[2], dims[1], dims[0])
        assert (lv == 123).all()


@pytest.mark.parametrize("f,dtype,bits", [((2, 2, 2), np.uint8, 8), ((3, 1, 2), np.uint16, 12),
                                          ((4, 4, 4), np.uint16, 16), ((1, 1, 1), np.uint8, 8)])
def test_integer_factor_is_block_mean(orc, f, dtype, bits):
    fx, fy, fz = f
    M = (5, 3, 4)
    rng = np.random.default_rng(5)
    vol = rng.integers(0, 1 << bits, size=(M[2] * fz, M[1] * fy, M[0] * fx)).astype(dtype)
    lv = orc.downsample(vol, bits, M)
    s = vol.astype(np.int64).reshape(M[2], fz, M[1], fy, M[0], fx).sum(axis=(1, 3, 5))
    cnt = fx * fy * fz
    assert np.array_equal(lv.astype(np.int64), (s + cnt // 2) // cnt)


def test_rounding_is_half_up(orc):
    vol = np.zeros((2, 2, 2), np.uint8)
    vol[0, 0, 0] = 4                      # mean 0.5 -> 1
    assert orc.downsample(vol, 8, (1, 1, 1))[0, 0, 0] == 1
    vol[0, 0, 0] = 3                      # mean 0.375 -> 0
    assert orc.downsample(vol, 8, (1, 1, 1))[0, 0, 0] == 0


@pytest.mark.parametrize("N,M", [(2016, 512), (1800, 512), (7, 3), (5, 3), (13, 13), (9, 1)])
def test_footprints_partition_the_axis(orc, N, M):
    # a hot voxel at x lands in exactly one output voxel, the covering ones
    # have widths floor(N/M) or ceil(N/M), and they tile the axis in order
    widths = []
    owner = []
    for x in range(N) if N < 64 else list(range(0, N, max(1, N // 61))) + [N - 1]:
        vol = np.zeros((1, 1, N), np.uint16)
        vol[0, 0, x] = 60000
        lv = orc.downsample(vol, 16, (M, 1, 1))[0, 0]
        nz = np.nonzero(lv)[0]
        assert nz.size == 1
        owner.append(int(nz[0]))
        widths.append(int(round(60000 / int(lv[nz[0]]))))
    assert owner == sorted(owner)
    assert set(widths) <= {N // M, -(-N // M)}


def test_ramp_maps_to_footprint_centres(orc):
    N, M = 2016, 512
    vol = np.arange(N, dtype=np.uint16).reshape(1, 1, N)
    lv = orc.downsample(vol, 12, (M, 1, 1))[0, 0].astype(np.int64)
    # the mean of the run lo..hi-1 is its centre (lo + hi - 1) / 2, rounded half up;
    # boundaries from float64 products, an independent route to floor(i N / M)
    b = np.floor(np.arange(M + 1) * (N / M) + 1e-9).astype(np.int64)
    assert np.array_equal(lv, (b[:-1] + b[1:] - 1 + 1) // 2)
    assert lv[0] == 1 and lv[-1] == N - 2
    assert set(np.diff(lv).tolist()) <= {3, 4, 5}


def test_sum_is_preserved_within_rounding(orc):
    rng = np.random.default_rng(9)
    vol = rng.integers(0, 4096, size=(11, 13, 17)).astype(np.uint16)
    M = (5, 4, 3)
    lv = orc.downsample(vol, 12, M).astype(np.int64)
    cnt = np.ones(M[::-1], np.int64)
    for ax, (n, m) in enumerate(zip((11, 13, 17), M[::-1])):
        w = np.array([((i + 1) * n) // m - (i * n) // m for i in range(m)])
        shape = [1, 1, 1]
        shape[ax] = m
        cnt = cnt * w.reshape(shape)
    total = int((lv * cnt).sum())
    assert cnt.sum() == vol.size
    assert abs(total - int(vol.astype(np.int64).sum())) <= int(cnt.sum()) // 2 + lv.size


def test_keep_table_applied_before_averaging(orc):
    vol = np.array([[[10, 200], [10, 200]], [[10, 200], [10, 200]]], np.uint8)
    keep = orc.keep_threshold(256, 100)
    lv = orc.downsample(vol, 8, (1, 1, 1), keep)
    assert lv[0, 0, 0] == 100           # (0*4 + 200*4 + 4) // 8
    lv2 = orc.downsample(vol, 8, (1, 1, 1))
    assert lv2[0, 0, 0] == 105          # (10*4 + 200*4 + 4) // 8


def test_levels_cascade_by_exact_halving(orc):
    rng = np.random.default_rng(2)
    vol = rng.integers(0, 256, size=(24, 20, 28)).astype(np.uint8)
    levels = orc.slicemap(vol, 8, [(8, 8, 8), (4, 4, 4), (2, 2, 2)])
    for a, b in zip(levels[:-1], levels[1:]):
        s = a.astype(np.int64).reshape(b.shape[0], 2, b.shape[1], 2, b.shape[2], 2).sum(axis=(1, 3, 5))
        assert np.array_equal(b.astype(np.int64), (s + 4) // 8)


def test_atlas_golden(orc):
    rows = []
    dims = tiles = None
    with open(os.path.join(GOLDEN, "atlas_2x2x3.txt")) as f:
        for line in f:
            if line.startswith("level_dims:"):
                dims = [int(v) for v in line.split(":")[1].split()]
            elif line.startswith("tiles:"):
                tiles = [int(v) for v in line.split(":")[1].split()]
            elif line.startswith("row:"):
                rows.append([int(v) for v in line.split(":")[1].split()])
    mx, my, mz = dims
    z, y, x = np.meshgrid(np.arange(mz), np.arange(my), np.arange(mx), indexing="ij")
    level = (100 * z + 10 * y + x + 1).astype(np.uint16)
    atlas = orc.atlas_pack(level, *tiles)
    assert np.array_equal(atlas, np.array(rows, np.uint16))


@pytest.mark.parametrize("mx,my,mz", [(128, 128, 128), (7, 5, 11), (16, 4, 3)])
def test_atlas_round_trip(orc, mx, my, mz):
    rng = np.random.default_rng(mz)
    level = rng.integers(0, 256, size=(mz, my, mx)).astype(np.uint8)
    tx, ty = orc.default_tiles(mz)
    atlas = orc.atlas_pack(level, tx, ty)
    assert atlas.shape == (ty * my, tx * mx)
    grid = atlas.reshape(ty, my, tx, mx).transpose(0, 2, 1, 3).reshape(ty * tx, my, mx)
    assert np.array_equal(grid[:mz], level)
    assert not grid[mz:].any()


def test_default_tiles():
    import oracle
    assert oracle.default_tiles(128) == (16, 8)
    assert oracle.default_tiles(256) == (16, 16)
    assert oracle.default_tiles(512) == (32, 16)
    assert oracle.default_tiles(1) == (1, 1)
    assert oracle.default_tiles(3) == (2, 2)


@pytest.mark.parametrize("shape,cell,dtype", [((16, 24, 40), 8, np.uint16), ((13, 9, 17), 8, np.uint8),
                                              ((20, 20, 20), 4, np.uint16), ((7, 5, 3), 8, np.uint8)])
def test_maxgrid_is_windowed_max(orc, shape, cell, dtype):
    from scipy.ndimage import maximum_filter
    rng = np.random.default_rng(sum(shape))
    level = rng.integers(0, 4096 if dtype == np.uint16 else 256, size=shape).astype(dtype)
    g = orc.maxgrid(level, cell)
    # window [c*cell, c*cell + cell]: a (cell+1)-wide maximum anchored at the cell's first voxel
    mf = maximum_filter(level, size=cell + 1, mode="nearest", origin=-(cell // 2))
    ref = mf[::cell, ::cell, ::cell]
    assert np.array_equal(g, ref)
