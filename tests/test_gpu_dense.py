"""Differentiable dense render (mctp_render_dense / _backward) against the
FP64 oracle: images within 2e-4, gradients within a relative tolerance of
the oracle's reverse-mode gradient, directional derivatives against central
differences of the GPU forward (h = 1e-3, 16^3 volume); the loss and Adam
kernels against plain restatements; autograd plumbing; a small fit lowers
its loss."""
import numpy as np
import pytest

from gpu_common import RENDER_TOL, STOP_EPS, render_error, sample_bounds

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import phantom
    import paper_2311_15038_gb300 as mctp
    from paper_2311_15038_gb300 import diff
    return mctp, diff, oracle, phantom, torch.device("cuda:0")


def _case(phantom, seed, shape=(16, 16, 16)):
    rng = np.random.default_rng(seed)
    vol = rng.uniform(0.05, 0.95, shape).astype(np.float32)
    lut = phantom.preset_luts(16)[3 + seed % 4].astype(np.float32)
    lut[:, 3] *= 0.35
    return vol, lut


VIEWS = [(0.0, 0.0, 20, 20), (33.0, 17.0, 24, 18), (-121.0, -48.0, 17, 23), (90.0, 90.0, 16, 16)]


@pytest.mark.parametrize("stop", [1.0, 0.99])
def test_dense_forward_matches_oracle(env, stop):
    mctp, diff, oracle, phantom, dev = env
    vol, lut = _case(phantom, 1, (12, 14, 16))
    src = (40, 36, 30)
    views = [mctp.View(az, el, w, h, 0, 0.5) for az, el, w, h in VIEWS]
    flat, samples = diff.render_dense(torch.from_numpy(vol).to(dev), torch.from_numpy(lut).to(dev), views, src, stop)
    lo_total = hi_total = 0
    for v, img in zip(views, mctp.images(flat, views)):
        ref = oracle.render_dense_band(vol.astype(np.float64), src, lut.astype(np.float64), v.azimuth_deg,
                                       v.elevation_deg, v.width, v.height, v.step, stop, STOP_EPS)
        # rays whose opacity passes the stop level within the band may stop one sample
        # apart: they are judged against the oracle's states at the band's edges
        err, amb = render_error(img.cpu().numpy(), ref)
        print(f"dense view {v}: max|err| vs FP64 = {err.max():.3e}, ambiguous rays {int(amb.sum())}")
        assert err.max() <= RENDER_TOL
        lo, hi = sample_bounds(ref)
        lo_total += lo
        hi_total += hi
    assert lo_total <= int(samples.item()) <= hi_total
    if stop == 1.0:
        assert lo_total == hi_total


def test_dense_gradient_matches_oracle(env):
    mctp, diff, oracle, phantom, dev = env
    vol, lut = _case(phantom, 2)
    src = (48, 48, 48)
    rng = np.random.default_rng(5)
    views = [mctp.View(az, el, w, h, 0, 0.5) for az, el, w, h in VIEWS]
    g = [rng.normal(size=(v.height, v.width, 4)).astype(np.float32) for v in views]
    g_flat = torch.from_numpy(np.concatenate([x.ravel() for x in g])).to(dev)
    gv, gl = diff.render_dense_backward(torch.from_numpy(vol).to(dev), torch.from_numpy(lut).to(dev), views, src,
                                        g_flat, 1.0)
    rv = np.zeros(vol.shape)
    rl = np.zeros(lut.shape)
    for v, gi in zip(views, g):
        a, b = oracle.render_dense_grad(vol.astype(np.float64), src, lut.astype(np.float64), v.azimuth_deg,
                                        v.elevation_deg, v.width, v.height, gi.astype(np.float64), v.step, 1.0)
        rv += a
        rl += b
    ev = np.abs(gv.cpu().numpy() - rv).max() / np.abs(rv).max()
    el = np.abs(gl.cpu().numpy() - rl).max() / np.abs(rl).max()
    print(f"dense gradient vs FP64 oracle: volume rel. err {ev:.2e}, LUT rel. err {el:.2e}")
    assert ev < 1e-4 and el < 1e-4


# Rays that cross the adjoint's 64-sample checkpoints.  Axis-aligned views of a
# 16^3 volume over a 64^3 box give every ray that hits the box exactly the same
# count (64 = one whole segment, 65 = one sample into a second, 128 = two
# whole); the diagonal view of a 24^3 volume has rays from a few samples up to
# 1998, the most the adjoint takes (31 whole segments and a partial one).
LONG_CASES = {
    "n64": ((16, 16, 16), (64, 64, 64), [(0.0, 0.0), (90.0, 0.0), (0.0, 90.0)], 10, 0.25, 64),
    "n65": ((16, 16, 16), (64, 64, 64), [(0.0, 0.0), (180.0, 0.0)], 10, 0.245, 65),
    "n128": ((16, 16, 16), (64, 64, 64), [(270.0, 0.0), (0.0, -90.0)], 10, 0.125, 128),
    "n1998": ((24, 24, 24), (64, 64, 64), [(45.0, 35.26438968)], 13, 0.0208, 1998),
}


def _long_case(phantom, name, stop):
    M, src, angles, wh, step, nmax = LONG_CASES[name]
    rng = np.random.default_rng(list(LONG_CASES).index(name) * 1000 + int(stop * 100))
    vol = rng.uniform(0.05, 0.95, (M[2], M[1], M[0])).astype(np.float32)
    lut = phantom.preset_luts(16)[5].astype(np.float32)
    # opacity per sample such that the rays of 1.0 stay below it (A < 1 in FP32) and
    # the rays of 0.99 stop partway through their second-to-last segments
    total_depth = {1.0: 6.0, 0.99: 9.0 if nmax < 100 else 16.0}[stop]
    lut[:, 3] = np.clip(lut[:, 3], 0.2, 1.0) * np.float32(total_depth / (0.6 * nmax))
    return vol, lut, src, angles, wh, step, nmax


@pytest.mark.parametrize("stop", [1.0, 0.99])
@pytest.mark.parametrize("name", list(LONG_CASES))
def test_dense_adjoint_across_checkpoints(env, name, stop):
    """mctp_render_dense_backward against orc_render_dense_grad (the reverse
    sweep over each ray's full stored sample list) element by element, on rays
    of 64, 65, 128 and up to 1998 samples, with and without early exit.  Rays
    that may stop one sample apart (their FP64 opacity passes alpha_stop within
    the band) get a zero upstream gradient here, so both sides drop them; they
    are checked one by one in the next test.  Per element, the allowed error is
    a fraction of the sum of |terms| that the oracle adds into that element (a
    bound for the rounding of any summation order), not of the largest element."""
    mctp, diff, oracle, phantom, dev = env
    vol, lut, src, angles, wh, step, nmax = _long_case(phantom, name, stop)
    views = [mctp.View(az, el, wh, wh, 0, step) for az, el in angles]
    rng = np.random.default_rng(17)
    rv = np.zeros(vol.shape)
    rl = np.zeros(lut.shape)
    mv = np.zeros(vol.shape)
    ml = np.zeros(lut.shape)
    g_views = []
    counts = set()
    n_amb = 0
    for v in views:
        band = oracle.render_dense_band(vol.astype(np.float64), src, lut.astype(np.float64), v.azimuth_deg,
                                        v.elevation_deg, v.width, v.height, v.step, stop, STOP_EPS)
        ns = band["nsamp"].astype(np.int64)
        amb = ns[..., 0] != ns[..., 2]
        n_amb += int(amb.sum())
        for j in range(v.height):
            for i in range(v.width):
                counts.add(oracle.ray_params(LONG_CASES[name][0], src, v.azimuth_deg, v.elevation_deg, v.width,
                                             v.height, v.step, i, j)[4])
        g = rng.normal(size=(v.height, v.width, 4))
        g[amb] = 0.0
        g_views.append(g.astype(np.float32))
        a, b, c, d = oracle.render_dense_grad(vol.astype(np.float64), src, lut.astype(np.float64), v.azimuth_deg,
                                              v.elevation_deg, v.width, v.height, g.astype(np.float32).astype(np.float64),
                                              v.step, stop, magnitudes=True)
        rv += a
        rl += b
        mv += c
        ml += d
    if name == "n1998":
        assert max(counts) == nmax and min(c for c in counts if c > 0) < 64
    else:
        assert counts == {0, nmax}
    g_flat = torch.from_numpy(np.concatenate([x.ravel() for x in g_views])).to(dev)
    gv, gl = diff.render_dense_backward(torch.from_numpy(vol).to(dev), torch.from_numpy(lut).to(dev), views, src,
                                        g_flat, stop)
    gv = gv.cpu().numpy().astype(np.float64)
    gl = gl.cpu().numpy().astype(np.float64)
    # The FP32 transmittance after k samples carries a relative error of about k
    # roundings (k <= 2048 here), and each term's error is relative to the term:
    # 4 * 2048 * 2^-24 = 4.9e-4 of the sum of |terms| bounds any summation order.
    tol_rel = 4 * 2048 * 2.0 ** -24
    for what, got, ref, mag in (("volume", gv, rv, mv), ("LUT", gl, rl, ml)):
        err = np.abs(got - ref)
        scale = np.maximum(mag, 1e-30)
        worst = (err / scale).max()
        print(f"{name} stop {stop}: {what} max |err|/sum|terms| = {worst:.2e}, "
              f"max |err| = {err.max():.2e} (max |ref| {np.abs(ref).max():.2e}), ambiguous rays {n_amb}")
        assert np.all(err <= tol_rel * mag + 1e-12), what


def _level_for_count(oracle, vol, src, lut, v, lin, k, lo, hi):
    """A stop level at which the FP64 march of pixel lin takes exactly k
    samples (bisection on the level; the opacity rises strictly along a ray
    whose table has no zero opacity)."""
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        _, ns = oracle.render_dense(vol, src, lut, v.azimuth_deg, v.elevation_deg, v.width, v.height, v.step, mid,
                                    pixels=np.array([lin]))
        if int(ns[0]) == k:
            return mid
        if int(ns[0]) < k:
            lo = mid
        else:
            hi = mid
    return None


@pytest.mark.parametrize("name", ["n65", "n128", "n1998"])
def test_dense_adjoint_straddling_rays(env, name):
    """A ray whose FP64 opacity passes alpha_stop within the band has several
    correct gradients: the GPU's gradient of that ray alone must equal the
    oracle's gradient of the same ray stopped after one of the sample counts
    the band allows."""
    mctp, diff, oracle, phantom, dev = env
    stop = 0.99
    vol, lut, src, angles, wh, step, _ = _long_case(phantom, name, stop)
    vol64, lut64 = vol.astype(np.float64), lut.astype(np.float64)
    v = mctp.View(angles[0][0], angles[0][1], wh, wh, 0, step)
    eps = STOP_EPS
    band = oracle.render_dense_band(vol64, src, lut64, v.azimuth_deg, v.elevation_deg, v.width, v.height, v.step,
                                    stop, eps)
    ns = band["nsamp"].astype(np.int64)
    # widen the band until some rays straddle it (the test needs at least one)
    while not np.any(ns[..., 0] != ns[..., 2]) and eps < 0.01:
        eps *= 4
        band = oracle.render_dense_band(vol64, src, lut64, v.azimuth_deg, v.elevation_deg, v.width, v.height,
                                        v.step, stop, eps)
        ns = band["nsamp"].astype(np.int64)
    rays = np.argwhere(ns[..., 0] != ns[..., 2])[:4]
    assert len(rays) > 0
    tv, tl = torch.from_numpy(vol).to(dev), torch.from_numpy(lut).to(dev)
    rng = np.random.default_rng(3)
    for (j, i) in rays:
        g = np.zeros((v.height, v.width, 4), np.float32)
        g[j, i] = rng.normal(size=4)
        gv, gl = diff.render_dense_backward(tv, tl, [v], src, torch.from_numpy(g.ravel()).to(dev), stop)
        gv = gv.cpu().numpy().astype(np.float64)
        gl = gl.cpu().numpy().astype(np.float64)
        best = np.inf
        for k in range(int(ns[j, i, 0]), int(ns[j, i, 2]) + 1):
            level = _level_for_count(oracle, vol64, src, lut64, v, j * v.width + i, k, stop - eps, stop + eps)
            assert level is not None
            a, b, c, d = oracle.render_dense_grad(vol64, src, lut64, v.azimuth_deg, v.elevation_deg, v.width,
                                                  v.height, g.astype(np.float64), v.step, level, magnitudes=True)
            r = max((np.abs(gv - a) / np.maximum(c, 1e-30)).max(), (np.abs(gl - b) / np.maximum(d, 1e-30)).max())
            best = min(best, r)
        print(f"{name}: straddling ray ({i}, {j}) samples {ns[j, i, 0]}..{ns[j, i, 2]}: "
              f"closest allowed stop max |err|/sum|terms| = {best:.2e}")
        assert best <= 4 * 2048 * 2.0 ** -24


def test_dense_gradient_central_differences(env):
    """Directional derivatives of L = sum(g * images) on a 16^3 volume: the
    adjoint against (L(p + h d) - L(p - h d)) / 2h of the GPU forward, h = 1e-3.
    The tolerance allows for the kinks of the piecewise-linear transfer
    function that a step of h crosses (the FD is then a blend of two slopes)
    and for FP32 noise in L; the tight check is the FP64 oracle gradient."""
    mctp, diff, oracle, phantom, dev = env
    vol, lut = _case(phantom, 3)
    src = (32, 32, 32)
    rng = np.random.default_rng(7)
    views = [mctp.View(az, el, w, h, 0, 0.5) for az, el, w, h in VIEWS]
    tv, tl = torch.from_numpy(vol).to(dev), torch.from_numpy(lut).to(dev)
    total = sum(v.width * v.height * 4 for v in views)
    g = torch.from_numpy(rng.normal(size=total).astype(np.float32)).to(dev)

    def L(vv, ll):
        out, _ = diff.render_dense(vv, ll, views, src, 1.0)
        return float((out[:total].double() * g.double()).sum())

    gv, gl = diff.render_dense_backward(tv, tl, views, src, g, 1.0)
    h = 1e-3
    for i in range(4):
        d = torch.from_numpy(rng.normal(size=vol.shape).astype(np.float32)).to(dev)
        fd = (L(tv + h * d, tl) - L(tv - h * d, tl)) / (2 * h)
        an = float((gv.double() * d.double()).sum())
        print(f"volume direction {i}: adjoint {an:.6f}, central difference {fd:.6f}")
        assert abs(fd - an) <= 2e-2 * abs(an) + 5e-2
        d = torch.from_numpy(rng.normal(size=lut.shape).astype(np.float32)).to(dev)
        fd = (L(tv, tl + h * d) - L(tv, tl - h * d)) / (2 * h)
        an = float((gl.double() * d.double()).sum())
        print(f"LUT direction {i}: adjoint {an:.6f}, central difference {fd:.6f}")
        assert abs(fd - an) <= 2e-2 * abs(an) + 5e-2


def test_loss_and_adam_kernels(env):
    mctp, diff, oracle, phantom, dev = env
    rng = np.random.default_rng(11)
    x = rng.normal(size=10007).astype(np.float32)
    t = rng.normal(size=10007).astype(np.float32)
    grad = torch.empty(10007, dtype=torch.float32, device=dev)
    loss, _ = diff.l2_loss(torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev), 0.25, grad)
    d = x.astype(np.float64) - t
    assert abs(float(loss.item()) - 0.25 * (d * d).sum()) < 1e-4 * 0.25 * (d * d).sum()
    assert np.allclose(grad.cpu().numpy(), 0.5 * d, rtol=1e-6, atol=1e-6)
    # Adam (Kingma & Ba, bias-corrected) over three steps, clamped to [lo, hi]
    p = rng.uniform(0.2, 0.8, 5001).astype(np.float32)
    gs = [rng.normal(size=5001).astype(np.float32) for _ in range(3)]
    tp = torch.from_numpy(p).to(dev)
    m = torch.zeros_like(tp)
    v = torch.zeros_like(tp)
    P, M, V = p.astype(np.float64), np.zeros(5001), np.zeros(5001)
    for k, gk in enumerate(gs, start=1):
        diff.adam_step(tp, torch.from_numpy(gk).to(dev), m, v, k, 0.05, 0.9, 0.999, 1e-8, 0.0, 1.0)
        M = 0.9 * M + 0.1 * gk
        V = 0.999 * V + 0.001 * gk.astype(np.float64) ** 2
        P = np.clip(P - 0.05 * (M / (1 - 0.9 ** k)) / (np.sqrt(V / (1 - 0.999 ** k)) + 1e-8), 0.0, 1.0)
    assert np.abs(tp.cpu().numpy() - P).max() < 1e-5


def test_autograd_and_small_fit(env):
    mctp, diff, oracle, phantom, dev = env
    vol, lut = _case(phantom, 4, (16, 16, 16))
    src = (64, 64, 64)
    views = [mctp.View(30.0 * k, 20.0 if k % 2 else -20.0, 24, 24, 0, 0.5) for k in range(6)]
    tv = torch.from_numpy(vol).to(dev).requires_grad_(True)
    tl = torch.from_numpy(lut).to(dev).requires_grad_(True)
    out = diff.DenseRender.apply(tv, tl, views, src, 0.99)
    (out * out).sum().backward()
    gv, gl = diff.render_dense_backward(tv.detach(), tl.detach(), views, src, 2 * out.detach(), 0.99)
    assert torch.allclose(tv.grad, gv, rtol=1e-4, atol=1e-6) and torch.allclose(tl.grad, gl, rtol=1e-4, atol=1e-6)
    # fit a blurred, dimmed start back towards the target renders
    target, _ = diff.render_dense(torch.from_numpy(vol).to(dev), torch.from_numpy(lut).to(dev), views, src, 0.99)
    total = sum(v.width * v.height * 4 for v in views)
    start = torch.from_numpy(np.clip(vol * 0.6 + 0.1, 0, 1).astype(np.float32)).to(dev)
    f = diff.Fitter(start, torch.from_numpy(lut).to(dev), views, src, target[:total], 0.99, 2e-2, 5e-3)
    l0 = f.evaluate()
    for _ in range(40):
        f.step()
    l1 = f.evaluate()
    print(f"small fit: loss {l0:.4e} -> {l1:.4e}")
    assert l1 < 0.5 * l0


def test_fit_resumes_from_checkpoint(env, tmp_path):
    """A fit stopped after 6 steps, saved with torch.save and resumed in a new
    fitter continues as the uninterrupted fit does: after 6 more steps both
    reach the same loss and parameters (within the float-atomic summation
    order of the adjoint), and the resumed step count is 12."""
    mctp, diff, oracle, phantom, dev = env
    vol, lut = _case(phantom, 6, (16, 16, 16))
    src = (48, 48, 48)
    views = [mctp.View(40.0 * k, 15.0 if k % 2 else -15.0, 20, 20, 0, 0.5) for k in range(4)]
    target, _ = diff.render_dense(torch.from_numpy(vol).to(dev), torch.from_numpy(lut).to(dev), views, src, 0.99)
    total = sum(v.width * v.height * 4 for v in views)
    start = torch.from_numpy(np.clip(vol * 0.7 + 0.1, 0, 1).astype(np.float32)).to(dev)

    def fitter():
        return diff.Fitter(start, torch.from_numpy(lut).to(dev), views, src, target[:total], 0.99, 2e-2, 5e-3)
    whole = fitter()
    for _ in range(6):
        whole.step()
    path = tmp_path / "fit.pt"
    torch.save(whole.state_dict(), path)
    for _ in range(6):
        whole.step()
    resumed = fitter()
    resumed.load_state_dict(torch.load(path))
    for _ in range(6):
        resumed.step()
    torch.cuda.synchronize()
    assert resumed.t == whole.t == 12
    lw, lr = whole.evaluate(), resumed.evaluate()
    print(f"loss after 12 steps: uninterrupted {lw:.6e}, resumed {lr:.6e}")
    assert abs(lw - lr) <= 1e-4 * lw
    assert torch.allclose(whole.vol, resumed.vol, rtol=0, atol=1e-4)
    assert torch.allclose(whole.lut, resumed.lut, rtol=0, atol=1e-4)
