"""Pins of the render oracle's oblique-view geometry (server-side rendering,
Sec. III-C; the orthographic turntable camera is this library's reading).

Every quantity here is computed independently of the oracle's FP32 set-up:
* the camera basis against hand-derived vectors (tests/golden/camera_basis.txt)
  and against what any such camera must satisfy (unit, orthogonal, right-handed,
  no roll, the centre ray through the box centre), recovered from the oracle's
  ray origins of neighbouring pixels;
* the sample count n of every ray against an FP64 ray-box chord computed from
  the hand basis, n = floor(chord / Delta), off by one only where the chord is
  within FP32 rounding of a multiple of Delta (or the ray grazes the box);
* oblique renders against a product-form compositor over FP64 sample
  positions (from the hand basis and the FP64 chord) interpolated by
  scipy.ndimage.map_coordinates, with numpy.interp for the transfer function.
A sign error in the up vector, a swapped slab bound or a wrong image-plane
offset fails one of them."""
import math
import os

import numpy as np
import pytest
from scipy.ndimage import map_coordinates

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "camera_basis.txt")


def _golden_bases():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, d, r, u = line.split("|")
            az, el = (float(x) for x in head.split())
            rows.append((az, el, np.array(d.split(), float), np.array(r.split(), float), np.array(u.split(), float)))
    return rows


def _hand_basis(az_deg, el_deg):
    """FP64 camera basis from the geometric description (camera on the unit
    vector at azimuth az about +z from +x and elevation el above the xy-plane;
    right horizontal; up completing a right-handed screen frame)."""
    az, el = math.radians(az_deg), math.radians(el_deg)
    b = np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    r = np.array([-math.sin(az), math.cos(az), 0.0])
    u = np.cross(b, r)
    return b, r, u


def _recovered_basis(orc, N, az, el, W=9, H=7, step=0.5):
    """Right, up and direction as the oracle's FP32 set-up realises them:
    o(i+1, j) - o(i, j) = (L/W) right, o(i, j) - o(i, j+1) = (L/H) up."""
    L = math.sqrt(sum(float(n) ** 2 for n in N))
    o00, d, _, _, _ = orc.ray_params(N, N, az, el, W, H, step, 0, 0)
    o10, _, _, _, _ = orc.ray_params(N, N, az, el, W, H, step, W - 1, 0)
    o01, _, _, _, _ = orc.ray_params(N, N, az, el, W, H, step, 0, H - 1)
    r = (o10.astype(float) - o00) / (L * (W - 1) / W)
    u = (o00.astype(float) - o01) / (L * (H - 1) / H)
    return d.astype(float), r, u


@pytest.mark.parametrize("row", range(4))
def test_camera_basis_matches_hand_derived(orc, row):
    az, el, d_ref, r_ref, u_ref = _golden_bases()[row]
    N = (20, 14, 11)
    d, r, u = _recovered_basis(orc, N, az, el)
    assert np.abs(d - d_ref).max() < 1e-6
    assert np.abs(r - r_ref).max() < 1e-5
    assert np.abs(u - u_ref).max() < 1e-5


@pytest.mark.parametrize("az,el", [(30.0, 20.0), (-73.0, 5.0), (135.0, -40.0), (250.0, 61.0), (0.0, 90.0),
                                   (45.0, -90.0), (179.0, 1.0)])
def test_camera_frame_properties(orc, az, el):
    N = (17, 12, 23)
    d, r, u = _recovered_basis(orc, N, az, el)
    tol = 2e-5
    assert abs(np.linalg.norm(d) - 1) < tol and abs(np.linalg.norm(r) - 1) < tol and abs(np.linalg.norm(u) - 1) < tol
    assert abs(d @ r) < tol and abs(d @ u) < tol and abs(r @ u) < tol
    assert np.abs(np.cross(r, u) + d).max() < tol          # right x up points back at the camera
    assert abs(r[2]) < tol                                 # no roll: right stays horizontal
    assert abs(d[2] + math.sin(math.radians(el))) < tol    # elevation above the xy-plane
    if abs(el) < 89.0:
        assert u[2] > 0                                    # image up is world up
        assert abs(math.atan2(-d[1], -d[0]) - math.atan2(math.sin(math.radians(az)), math.cos(math.radians(az)))) < tol
    # the ray of the centre pixel (odd W, H) passes through the box centre
    o, dd, _, _, _ = orc.ray_params(N, N, az, el, 9, 7, 0.5, 4, 3)
    c = np.array(N, float) / 2
    off = (c - o) - ((c - o) @ dd.astype(float)) * dd.astype(float)
    assert np.abs(off).max() < 1e-4


def _chord64(N, az, el, W, H, i, j):
    """FP64 image-plane origin from the hand basis and the Kay-Kajiya slab
    interval [t0, t1] of the ray o - t b against the box [0, N]."""
    b, r, u = _hand_basis(az, el)
    Nd = np.array(N, float)
    L = math.sqrt(float((Nd ** 2).sum()))
    c = Nd / 2
    sx = (i + 0.5) / W - 0.5
    sy = 0.5 - (j + 0.5) / H
    o = c + sx * L * r + sy * L * u + L * b
    d = -b
    t0, t1 = -math.inf, math.inf
    for a in range(3):
        if abs(d[a]) < 1e-12:
            if not (0.0 <= o[a] <= Nd[a]):
                return o, d, 0.0, 0.0, L
            continue
        s0, s1 = (0.0 - o[a]) / d[a], (Nd[a] - o[a]) / d[a]
        t0, t1 = max(t0, min(s0, s1)), min(t1, max(s0, s1))
    if t1 <= t0:
        return o, d, 0.0, 0.0, L
    return o, d, t0, t1, L


CASES = [((16, 16, 16), (16, 16, 16), 30.0, 20.0, 0.5),
         ((24, 13, 9), (12, 13, 9), 30.0, 20.0, 0.35),
         ((24, 13, 9), (24, 13, 9), -112.0, 47.0, 0.7),
         ((10, 31, 17), (5, 16, 9), 200.0, -33.0, 0.5),
         ((12, 12, 20), (12, 12, 20), 0.0, 90.0, 0.5),
         ((12, 12, 20), (6, 6, 10), 77.0, -90.0, 0.3),
         ((9, 7, 8), (9, 7, 8), 45.0, 35.26438968, 0.1)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_sample_counts_against_fp64_chord(orc, case):
    N, M, az, el, step = CASES[case]
    W, H = 13, 11
    delta = step * min(N[a] / M[a] for a in range(3))
    exact = 0
    for j in range(H):
        for i in range(W):
            _, _, t0, t1, L = _chord64(N, az, el, W, H, i, j)
            x = (t1 - t0) / delta
            n64 = int(math.floor(x))
            _, _, _, _, n = orc.ray_params(M, N, az, el, W, H, step, i, j)
            # FP32 set-up error: a few ulps of the distances involved (L and the box)
            slack = 64 * 2.0 ** -24 * (2 * L) / delta
            if n == n64:
                exact += 1
                continue
            frac = x - round(x)
            assert abs(n - n64) == 1 and (abs(frac) < slack or x < slack), (i, j, n, n64, x)
    assert exact >= 0.5 * W * H, exact


def _product_form(values, lut, alpha_stop):
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
    return np.array([(w * rgba[:m, 0]).sum(), (w * rgba[:m, 1]).sum(), (w * rgba[:m, 2]).sum(), 1 - trans[m]])


@pytest.mark.parametrize("case", [0, 1, 2, 3, 5])
def test_oblique_views_match_product_form(orc, case):
    N, M, az, el, step = CASES[case]
    rng = np.random.default_rng(100 + case)
    bits = 12
    # a smooth volume keeps the FP32-vs-FP64 position difference from mattering
    z, y, x = np.meshgrid(*(np.arange(n) for n in (N[2], N[1], N[0])), indexing="ij")
    f = 0.5 + 0.25 * np.sin(0.37 * x + 0.11 * y) * np.cos(0.23 * z - 0.19 * x) + 0.2 * np.sin(0.29 * y + 0.31 * z)
    vol = np.clip(np.rint(f * 4095 + rng.integers(-40, 40, f.shape)), 0, 4095).astype(np.uint16)
    level = orc.downsample(vol, bits, M) if tuple(M) != tuple(N) else vol
    lut = rng.uniform(0.0, 1.0, size=(12, 4)).astype(np.float32)
    lut[:, 3] *= 0.3
    W, H, stop = 13, 11, 0.97
    out = orc.render(level, bits, N, lut, az, el, W, H, step=step, alpha_stop=stop, eps=1e-4)
    delta = step * min(N[a] / M[a] for a in range(3))
    s = np.array([N[a] / M[a] for a in range(3)])
    checked = 0
    for j in range(H):
        for i in range(W):
            o, d, t0, t1, L = _chord64(N, az, el, W, H, i, j)
            x_ = (t1 - t0) / delta
            if abs(x_ - round(x_)) < 1e-3 and x_ > 0.5:
                continue                                   # FP32 may take one sample more or less
            n = int(math.floor(x_))
            if n == 0:
                assert out["rgba"][j, i].sum() == 0
                checked += 1
                continue
            t = t0 + (np.arange(n) + 0.5) * delta
            pos = o[:, None] + t[None, :] * d[:, None]
            q = pos / s[:, None] - 0.5
            raw = map_coordinates(level.astype(np.float64), [q[2], q[1], q[0]], order=1, mode="nearest")
            v = np.minimum(raw / ((1 << bits) - 1), 1.0)
            ref = _product_form(v, lut, stop)
            got = out["rgba"][j, i]
            if out["nsamp"][j, i, 0] != out["nsamp"][j, i, 2]:
                got_set = [out["lo"][j, i], got, out["hi"][j, i]]
                assert min(np.abs(g - ref).max() for g in got_set) < 1e-4
            else:
                np.testing.assert_allclose(got, ref, atol=1e-4, rtol=0)
            checked += 1
    assert checked >= 0.6 * W * H
