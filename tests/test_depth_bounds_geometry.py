"""The depth bounds of the batched renderer, checked on the host against an
FP64 model of the rays.

For one view and one cell of the max grid, the set-up kernel (render_batch.cu,
batch_bounds_kernel) takes the cell's box of sample positions, level
coordinates [8c - 1, 8c + 9] per axis, projects it into the image with one
pixel of margin and records its depth range; a ray then marches the samples
k0 <= k < kend derived from that range with two samples of margin
(render_common.cuh, march_ray).  Skipping the other samples is exact only if
every sample whose lower corner lies in the cell is inside both.  This test
mirrors the kernel's FP32 formulas in numpy and checks that property against
sample positions computed in FP64, for axis-aligned, straight-down and random
views, steps from 0.3 to 3 voxels and cells on the level's faces and inside."""
import math

import numpy as np
import pytest

from ray_model import F, rays


def cell_bounds(R, N, M, cell, W, H):
    """The kernel's footprint and depth range of a cell, in FP32."""
    s = (N.astype(F) / M.astype(F)).astype(F)
    xr = [F(0), F(0)]
    xu = [F(0), F(0)]
    xb = [F(0), F(0)]
    for a in range(3):
        p0 = F((F(8 * cell[a] - 1) + F(0.5)) * s[a] - R["c"][a])
        p1 = F((F(8 * cell[a] + 9) + F(0.5)) * s[a] - R["c"][a])
        for acc, e in ((xr, R["r"]), (xu, R["u"]), (xb, R["b"])):
            acc[0] = F(acc[0] + min(F(p0 * e[a]), F(p1 * e[a])))
            acc[1] = F(acc[1] + max(F(p0 * e[a]), F(p1 * e[a])))
    invL = F(1) / R["L"]
    fx0 = F((xr[0] * invL + F(0.5)) * F(W) - F(0.5))
    fx1 = F((xr[1] * invL + F(0.5)) * F(W) - F(0.5))
    fy0 = F((F(0.5) - xu[1] * invL) * F(H) - F(0.5))
    fy1 = F((F(0.5) - xu[0] * invL) * F(H) - F(0.5))
    clampw = lambda v, hi: min(max(v, F(-2)), F(hi + 2))
    px0 = max(int(math.ceil(clampw(fx0, W))) - 1, 0)
    px1 = min(int(math.floor(clampw(fx1, W))) + 1, W - 1)
    py0 = max(int(math.ceil(clampw(fy0, H))) - 1, 0)
    py1 = min(int(math.floor(clampw(fy1, H))) + 1, H - 1)
    return (px0, px1, py0, py1), (F(R["L"] - xb[1]), F(R["L"] - xb[0]))


def sample_range(lo, hi, tmin, delta, n):
    """The march's [k0, kend) from a depth range, in FP32."""
    inv_d = F(1) / delta
    klo = ((lo - tmin) * inv_d - F(2.5)).astype(F)
    khi = ((hi - tmin) * inv_d + F(2.5)).astype(F)
    k0 = np.minimum(np.maximum(klo, F(0)), n.astype(F)).astype(np.int64)
    kend = np.minimum(np.maximum(khi, F(0)), (n - 1).astype(F)).astype(np.int64) + 1
    return k0, kend


VIEWS = [(0.0, 0.0), (90.0, 0.0), (180.0, 0.0), (270.0, 0.0), (0.0, 90.0), (0.0, -90.0), (45.0, 0.0),
         (33.0, 71.0), (-120.0, -35.0), (10.0, 20.0), (200.0, 55.0), (301.0, -80.0)]


@pytest.mark.parametrize("az,el", VIEWS)
@pytest.mark.parametrize("step", [0.3, 1.0, 3.0])
def test_marked_cell_samples_inside_bounds(az, el, step):
    N = np.array([83, 61, 50])
    M = np.array([40, 32, 24])
    W, H = 48, 40
    R = rays(N, M, az, el, W, H, step)
    sc = M / N  # FP64 truth of the level coordinates
    g = [(m + 7) // 8 for m in M]
    rng = np.random.default_rng(int(abs(az) * 7 + abs(el) * 3 + step * 100))
    cells = {(0, 0, 0), (g[0] - 1, g[1] - 1, g[2] - 1), (0, g[1] - 1, 1)}
    while len(cells) < 8:
        cells.add(tuple(int(rng.integers(gi)) for gi in g))
    kmax = int(R["n"].max())
    k = np.arange(kmax)
    t = (R["tmin"][..., None].astype(np.float64) + (k + 0.5) * float(R["delta"]))  # [H][W][K]
    q = (R["o"][..., None, :].astype(np.float64) + t[..., None] * R["d"].astype(np.float64)) * sc - 0.5
    corner = np.clip(np.floor(q).astype(np.int64), 0, M - 1)
    cellidx = corner >> 3
    valid = k[None, None, :] < R["n"][..., None]
    checked = 0
    for cell in cells:
        (px0, px1, py0, py1), (lo, hi) = cell_bounds(R, N, M, cell, W, H)
        inside = valid & np.all(cellidx == np.array(cell), axis=-1)
        ys, xs, ks = np.nonzero(inside)
        if len(ks) == 0:
            continue
        assert xs.min() >= px0 and xs.max() <= px1, (cell, xs.min(), xs.max(), px0, px1)
        assert ys.min() >= py0 and ys.max() <= py1, (cell, ys.min(), ys.max(), py0, py1)
        k0, kend = sample_range(np.full(len(ks), lo, F), np.full(len(ks), hi, F), R["tmin"][ys, xs], R["delta"],
                                R["n"][ys, xs])
        assert np.all(ks >= k0) and np.all(ks < kend), cell
        checked += len(ks)
    assert checked > 0
