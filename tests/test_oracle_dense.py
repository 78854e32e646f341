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
