"""Pins of the oracle's container removal (orc_hough_circle, orc_mask_circle),
CPU only: rings drawn at known centres and radii, the phantom container's own
geometry, an image without edges, and disk masks counted point by point."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def orc():
    import oracle
    import phantom
    oracle.build()
    phantom.build(gpu=False)
    return oracle


@pytest.mark.parametrize("n,cx0,cy0,R,cell", [(120, 61.3, 57.8, 40.0, 4), (200, 97.0, 104.6, 83.5, 8),
                                               (333, 170.2, 160.9, 140.0, 8)])
def test_drawn_ring(orc, n, cx0, cy0, R, cell):
    # a bright wall from radius R to R + 6 on a dark background: the circle
    # found is the wall's inner boundary
    y, x = np.mgrid[0:n, 0:n]
    d = np.hypot(x - cx0, y - cy0)
    img = np.where((d >= R) & (d <= R + 6), 200, 20).astype(np.uint8)
    h = orc.hough_circle(img, 40, n // 8, n // 2, cell)
    fx, fy, fr = h["fit"]
    assert abs(fx - cx0) < 0.3 and abs(fy - cy0) < 0.3, h["fit"]
    assert abs(fr - (R - 0.5)) < 0.7, h["fit"]
    assert (h["cx"], h["cy"], h["r"]) == (int(np.floor(fx + 0.5)), int(np.floor(fy + 0.5)), int(np.floor(fr)))
    # the coarse cell with most votes holds the centre
    iy, ix = np.unravel_index(np.argmax(h["acc"]), h["acc"].shape)
    assert abs(ix * cell + (cell - 1) / 2 - cx0) <= cell and abs(iy * cell + (cell - 1) / 2 - cy0) <= cell


@pytest.mark.parametrize("n,seed", [(128, 1), (256, 2), (320, 3)])
def test_phantom_container(orc, n, seed):
    import phantom
    spec = phantom.VolumeSpec(n, n, 12, bits=8, seed=seed, n_ell=4, tube=True)
    tx, ty, r_in, r_out = phantom.tube_geometry(spec)
    top = phantom.generate_cpu(spec, ((0, n), (0, n), (0, 1)))[0]
    h = orc.hough_circle(top, 40, n // 8, n // 2, max(4, n // 32))
    fx, fy, fr = h["fit"]
    assert abs(fx - tx) < 0.3 and abs(fy - ty) < 0.3 and abs(fr - r_in) < 0.5, (h["fit"], (tx, ty, r_in))


def test_no_edges(orc):
    h = orc.hough_circle(np.full((64, 80), 30, np.uint8), 40, 8, 32, 4)
    assert (h["cx"], h["cy"], h["r"]) == (0, 0, -1)
    assert h["acc"].sum() == 0 and h["rhist"].sum() == 0


def test_mask_circle(orc):
    rng = np.random.default_rng(1)
    vol = rng.integers(1, 256, size=(3, 37, 41)).astype(np.uint8)
    for cx, cy, rk in [(20, 18, 10), (0, 0, 5), (40, 36, 0), (17, 11, 100)]:
        out = orc.mask_circle(vol, cx, cy, rk)
        inside = [(x, y) for y in range(37) for x in range(41) if (x - cx) ** 2 + (y - cy) ** 2 <= rk * rk]
        assert int((out[0] != 0).sum()) == len(inside)
        for x, y in inside[:50]:
            assert out[1, y, x] == vol[1, y, x]
    assert np.array_equal(orc.mask_circle(vol, 5, 5, -1), vol)  # no container found: keep everything
