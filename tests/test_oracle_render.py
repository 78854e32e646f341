"""Pins of the CPU oracle's renderer (server-side rendering, Sec. III-C).

The renderer's definition (camera, FP32 ray setup, trilinear sampling, linear
transfer function, front-to-back compositing with early exit) is this library's
reading, since the paper only names the step.  It is pinned by:
* the Beer-Lambert closed form A = 1 - (1 - a)^n on a constant volume,
* axis-aligned views along each of the three axes, compared with a
  product-form compositor sum_k a_k c_k prod_{j<k} (1 - a_j) over samples
  interpolated by scipy.ndimage.map_coordinates and a transfer function
  interpolated by numpy.interp,
* an empty volume, and the sample count of axis-aligned rays.
"""
import numpy as np
import pytest
from scipy.ndimage import map_coordinates


def _ramp(n):
    v = np.arange(n, dtype=np.float64) / (n - 1)
    return np.repeat(v[:, None], 4, axis=1).astype(np.float32)


def test_beer_lambert_slab(orc):
    N = (10, 6, 8)
    vol = np.full((N[2], N[1], N[0]), 77, np.uint8)
    a, c = 0.05, (0.9, 0.4, 0.2)
    lut = np.tile(np.array([[c[0], c[1], c[2], a]], np.float32), (4, 1))
    W = H = 8
    for az, el, step in [(0.0, 0.0, 0.3), (90.0, 0.0, 0.3), (0.0, 90.0, 0.3), (37.0, 21.0, 0.5)]:
        out = orc.render(vol, 8, N, lut, az, el, W, H, step=step, alpha_stop=0.99)
        for j in range(H):
            for i in range(W):
                _, _, _, _, n = orc.ray_params(N, N, az, el, W, H, step, i, j)
                # stop at the first k with 1 - (1-a)^k >= 0.99
                k = np.arange(1, n + 1)
                A_k = 1 - (1 - np.float64(np.float32(a))) ** k
                hit = np.nonzero(A_k >= 0.99)[0]
                m = int(hit[0]) + 1 if hit.size else n
                A = 1 - (1 - np.float64(np.float32(a))) ** m
                px = out["rgba"][j, i]
                assert px[3] == pytest.approx(A, abs=1e-12)
                assert px[:3] == pytest.approx(np.float32(c).astype(np.float64) * A, abs=1e-12)
                assert int(out["nsamp"][j, i, 1]) == m


def test_axis_aligned_sample_counts(orc):
    # rays along -x through a 10-voxel box with step 0.3: floor(10 / 0.3) = 33
    N = (10, 6, 8)
    _, d, t_near, delta, n = orc.ray_params(N, N, 0.0, 0.0, 4, 4, 0.3, 1, 1)
    assert d[0] == -1.0 and d[1] == 0.0 and d[2] == 0.0
    assert delta == np.float32(0.3)
    assert n == 33
    # a level at half resolution doubles the spacing and so the step length
    _, _, _, delta2, n2 = orc.ray_params((5, 3, 4), N, 0.0, 0.0, 4, 4, 0.3, 1, 1)
    assert delta2 == np.float32(0.6) and n2 == 16
    # rays outside the box's projection take no samples
    out = orc.render(np.full((8, 6, 10), 200, np.uint8), 8, N, _ramp(8), 0.0, 0.0, 64, 64)
    assert out["nsamp"][0, 0, 1] == 0 and out["rgba"][0, 0].sum() == 0


def test_empty_volume_renders_transparent(orc):
    vol = np.zeros((5, 6, 7), np.uint16)
    lut = _ramp(16)
    out = orc.render(vol, 12, (7, 6, 5), lut, 23.0, -31.0, 9, 7)
    assert not out["rgba"].any()


def _product_form(values, lut, alpha_stop):
    """sum_k a_k c_k prod_{j<k}(1-a_j), truncated at the first k where the
    accumulated opacity 1 - prod_{j<=k}(1-a_j) reaches alpha_stop."""
    n = lut.shape[0]
    x = values * (n - 1)
    grid = np.arange(n)
    rgba = np.stack([np.interp(x, grid, lut[:, ch].astype(np.float64)) for ch in range(4)], axis=1)
    a = rgba[:, 3]
    trans = np.concatenate([[1.0], np.cumprod(1 - a)])
    acc = 1 - trans[1:]
    stop = np.nonzero(acc >= alpha_stop)[0]
    m = int(stop[0]) + 1 if stop.size else len(a)
    w = a[:m] * trans[:m]
    return np.array([(w * rgba[:m, 0]).sum(), (w * rgba[:m, 1]).sum(), (w * rgba[:m, 2]).sum(),
                     1 - trans[m]])


@pytest.mark.parametrize("axis", ["x", "y", "z"])
@pytest.mark.parametrize("half", [False, True])
def test_axis_aligned_views_match_product_form(orc, axis, half):
    rng = np.random.default_rng({"x": 1, "y": 2, "z": 3}[axis])
    N = (9, 7, 8)                                   # nx, ny, nz
    bits = 12
    vol = rng.integers(0, 4096, size=(N[2], N[1], N[0])).astype(np.uint16)
    M = (5, 4, 4) if half else N
    level = orc.downsample(vol, bits, M) if half else vol
    lut = rng.uniform(0.0, 1.0, size=(12, 4)).astype(np.float32)
    lut[:, 3] *= 0.35
    W, H, step, stop = 11, 10, 0.45, 0.97
    az, el = {"x": (0.0, 0.0), "y": (90.0, 0.0), "z": (0.0, 90.0)}[axis]
    out = orc.render(level, bits, N, lut, az, el, W, H, step=step, alpha_stop=stop)
    Nf = np.array(N, np.float32)
    L = np.float32(np.sqrt(float(N[0] ** 2 + N[1] ** 2 + N[2] ** 2)))
    c = Nf / np.float32(2)
    s = np.array([N[k] / M[k] for k in range(3)])
    delta = np.float32(step) * np.float32(min(np.float32(N[k]) / np.float32(M[k]) for k in range(3)))
    for j in range(H):
        for i in range(W):
            sx = np.float32(np.float32(i + 0.5) / np.float32(W)) - np.float32(0.5)
            sy = np.float32(0.5) - np.float32(np.float32(j + 0.5) / np.float32(H))
            sxL, syL = np.float32(sx * L), np.float32(sy * L)
            if axis == "x":    # view from +x: right = +y, up = +z, ray along -x
                lat = {1: c[1] + sxL, 2: c[2] + syL}
                ray_axis = 0
            elif axis == "y":  # view from +y: right = -x, up = +z, ray along -y
                lat = {0: c[0] - sxL, 2: c[2] + syL}
                ray_axis = 1
            else:              # view from +z: right = +y, up = -x, ray along -z
                lat = {1: c[1] + sxL, 0: c[0] - syL}
                ray_axis = 2
            lat = {k: np.float32(v) for k, v in lat.items()}
            if any(not (0 <= lat[k] <= Nf[k]) for k in lat):
                assert out["rgba"][j, i].sum() == 0
                continue
            n = int(np.floor(np.float32(Nf[ray_axis] / delta)))
            t = (np.arange(n) + 0.5) * np.float64(delta)
            pos = np.zeros((3, n))
            for k in range(3):
                pos[k] = lat[k] if k in lat else Nf[ray_axis] - t
            q = pos / s[:, None] - 0.5                     # level voxel coordinates
            raw = map_coordinates(level.astype(np.float64), [q[2], q[1], q[0]], order=1, mode="nearest")
            v = np.minimum(raw / ((1 << bits) - 1), 1.0)
            ref = _product_form(v, lut, stop)
            np.testing.assert_allclose(out["rgba"][j, i], ref, atol=2e-5, rtol=0)


def test_ambiguous_stop_is_reported(orc):
    # a constant slab whose opacity crosses alpha_stop within eps of it
    N = (40, 40, 40)
    vol = np.full((40, 40, 40), 255, np.uint8)
    a = np.float32(0.1)
    lut = np.tile(np.array([[1, 1, 1, a]], np.float32), (2, 1))
    # A_k = 1 - 0.9^k crosses 0.99 at k = 44 (A_43 = 0.98922, A_44 = 0.99030)
    A44 = 1 - (1 - np.float64(a)) ** 44
    out = orc.render(vol, 8, N, lut, 0.0, 0.0, 4, 4, step=0.25, alpha_stop=float(np.float32(A44)),
                     eps=1e-4)
    ns = out["nsamp"][1, 1]
    assert ns[0] <= ns[1] <= ns[2]
    assert ns[2] - ns[0] >= 1                     # lo and hi stops differ: ambiguous ray
