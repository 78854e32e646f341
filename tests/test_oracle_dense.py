"""Pins of the oracle's differentiable dense render (orc_render_dense) and its
FP64 gradient (orc_render_dense_grad), CPU only: agreement with orc_render on
the same level, the Beer-Lambert slab and its closed-form derivative, and
central finite differences along random directions."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _loss(orc, vol, src, lut, view, g, stop):
    az, el, w, h, step = view
    r, _ = orc.render_dense(vol, src, lut, az, el, w, h, step, stop)
    return float((r * g).sum())


def test_dense_equals_level_render(orc):
    import phantom
    vol = phantom.generate_cpu(phantom.VolumeSpec(40, 36, 32, bits=8, seed=81, n_ell=4))
    level = orc.downsample(vol, 8, (20, 18, 16))
    lut = phantom.preset_luts()[3]
    for az, el in [(0.0, 0.0), (37.0, 21.0), (-120.0, -50.0)]:
        ref = orc.render(level, 8, (40, 36, 32), lut, az, el, 24, 20, 0.5, 0.99, 0.0)
        got, ns = orc.render_dense(level.astype(np.float64) / 255.0, (40, 36, 32), lut.astype(np.float64), az, el,
                                   24, 20, 0.5, 0.99)
        assert np.abs(got - ref["rgba"]).max() < 1e-12
        assert np.array_equal(ns, ref["nsamp"][..., 1])


def test_dense_beer_lambert_and_slab_derivative(orc):
    a, c = 0.03, np.array([0.2, 0.5, 0.9])
    lut = np.tile(np.concatenate([c, [a]]), (8, 1))
    vol = np.full((6, 7, 8), 0.4)
    src = (16, 14, 12)
    r, ns = orc.render_dense(vol, src, lut, 25.0, 10.0, 9, 7, 0.5, 1.0)
    n = ns.astype(np.float64)
    A = 1.0 - (1.0 - a) ** n
    assert np.abs(r[..., 3] - A).max() < 1e-13
    assert np.abs(r[..., :3] - c * A[..., None]).max() < 1e-13
    # dA/da summed over the opacity entries of the table = n (1 - a)^(n - 1) per ray
    g = np.zeros((7, 9, 4))
    g[..., 3] = 1.0
    _, gl = orc.render_dense_grad(vol, src, lut, 25.0, 10.0, 9, 7, g, 0.5, 1.0)
    want = (n * (1.0 - a) ** (n - 1)).sum()
    assert abs(gl[:, 3].sum() - want) < 1e-9 * max(1.0, want)


@pytest.mark.parametrize("stop", [1.0, 0.9])
def test_dense_grad_matches_central_differences(orc, stop):
    rng = np.random.default_rng(int(stop * 10))
    vol = rng.uniform(0.05, 0.95, (8, 9, 10))
    lut = rng.uniform(0.0, 1.0, (16, 4))
    lut[:, 3] *= 0.25
    src = (20, 18, 16)
    view = (33.0, 17.0, 11, 9, 0.5)
    g = rng.normal(size=(9, 11, 4))
    gv, gl = orc.render_dense_grad(vol, src, lut, *view[:4], g, view[4], stop)
    h = 1e-6
    for _ in range(3):
        dv = rng.normal(size=vol.shape)
        fd = (_loss(orc, vol + h * dv, src, lut, view, g, stop) - _loss(orc, vol - h * dv, src, lut, view, g, stop)) / (2 * h)
        an = float((gv * dv).sum())
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)
        dl = rng.normal(size=lut.shape)
        fd = (_loss(orc, vol, src, lut + h * dl, view, g, stop) - _loss(orc, vol, src, lut - h * dl, view, g, stop)) / (2 * h)
        an = float((gl * dl).sum())
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_dense_grad_zero_where_clamped(orc):
    # intensities far above 1 saturate at the last table entry: no volume gradient
    vol = np.full((5, 5, 5), 3.0)
    lut = np.linspace(0, 1, 32)[:, None] * np.array([1.0, 0.5, 0.2, 0.1])
    g = np.ones((6, 6, 4))
    gv, gl = orc.render_dense_grad(vol, (10, 10, 10), lut, 10.0, 5.0, 6, 6, g, 0.5, 1.0)
    assert np.all(gv == 0.0)
    assert np.any(gl[-1] != 0.0)


def test_dense_band_edges_are_plain_renders(orc):
    """The band's lo / mid / hi results are the plain dense render stopped at
    alpha_stop - eps, alpha_stop and alpha_stop + eps (the early-exit straddle
    reading), with ordered sample counts."""
    rng = np.random.default_rng(21)
    vol = rng.uniform(0.05, 0.95, (9, 8, 10))
    lut = rng.uniform(0.0, 1.0, (16, 4))
    lut[:, 3] *= 0.4
    src, view, stop, eps = (30, 24, 27), (41.0, -23.0, 12, 10, 0.5), 0.95, 0.02
    band = orc.render_dense_band(vol, src, lut, *view, stop, eps)
    for key, level, col in (("lo", stop - eps, 0), ("rgba", stop, 1), ("hi", stop + eps, 2)):
        r, ns = orc.render_dense(vol, src, lut, *view, level)
        assert np.array_equal(band[key], r)
        assert np.array_equal(band["nsamp"][..., col], ns)
    ns = band["nsamp"].astype(np.int64)
    assert np.all(ns[..., 0] <= ns[..., 1]) and np.all(ns[..., 1] <= ns[..., 2])
    assert np.any(ns[..., 0] < ns[..., 2])
    flat = orc.render_dense_band(vol, src, lut, *view, stop, 0.0)
    assert np.array_equal(flat["lo"], flat["rgba"]) and np.array_equal(flat["hi"], flat["rgba"])


def test_dense_grad_magnitudes(orc):
    """The per-element magnitude is the sum of |terms|: it bounds |gradient|,
    is unchanged when the upstream gradient changes sign (the gradient flips),
    and scales with it."""
    rng = np.random.default_rng(22)
    vol = rng.uniform(0.05, 0.95, (6, 7, 8))
    lut = rng.uniform(0.0, 1.0, (8, 4))
    lut[:, 3] *= 0.3
    src, view = (16, 14, 12), (25.0, 10.0, 9, 7)
    g = rng.normal(size=(7, 9, 4))
    gv, gl, mv, ml = orc.render_dense_grad(vol, src, lut, *view, g, 0.5, 0.99, magnitudes=True)
    assert np.all(mv >= np.abs(gv) * (1 - 1e-12)) and np.all(ml >= np.abs(gl) * (1 - 1e-12))
    assert np.any(mv > np.abs(gv) * 1.01)          # terms of both signs meet in some voxels
    gv2, gl2, mv2, ml2 = orc.render_dense_grad(vol, src, lut, *view, -2.0 * g, 0.5, 0.99, magnitudes=True)
    assert np.allclose(gv2, -2.0 * gv, rtol=1e-12, atol=1e-15) and np.allclose(mv2, 2.0 * mv, rtol=1e-12, atol=1e-15)
    assert np.allclose(gl2, -2.0 * gl, rtol=1e-12, atol=1e-15) and np.allclose(ml2, 2.0 * ml, rtol=1e-12, atol=1e-15)
    gv3, gl3 = orc.render_dense_grad(vol, src, lut, *view, g, 0.5, 0.99)
    assert np.array_equal(gv3, gv) and np.array_equal(gl3, gl)
