"""Differentiable dense render (mctp_render_dense / _backward) against the
FP64 oracle: images within 2e-4, gradients within a relative tolerance of
the oracle's reverse-mode gradient, directional derivatives against central
differences of the GPU forward (h = 1e-3, 16^3 volume); the loss and Adam
kernels against plain restatements; autograd plumbing; a small fit lowers
its loss."""
import numpy as np
import pytest

from gpu_common import RENDER_TOL

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
    total_ref = 0
    for v, img in zip(views, mctp.images(flat, views)):
        ref, ns = oracle.render_dense(vol.astype(np.float64), src, lut.astype(np.float64), v.azimuth_deg,
                                      v.elevation_deg, v.width, v.height, v.step, stop)
        got = img.cpu().numpy().astype(np.float64)
        err = np.abs(got - ref).max(axis=-1)
        # rays whose opacity passes the stop level within FP32 noise may stop one sample apart
        amb = (np.abs(ref[..., 3] - stop) < 1e-4) | (np.abs(got[..., 3] - stop) < 1e-4)
        print(f"dense view {v}: max|err| vs FP64 = {err[~amb].max():.3e}, ambiguous rays {int(amb.sum())}")
        assert err[~amb].max() <= RENDER_TOL
        total_ref += int(ns.sum())
    if stop == 1.0:
        assert int(samples.item()) == total_ref


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
