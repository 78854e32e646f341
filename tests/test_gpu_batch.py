"""Batched rendering (mctp_render_batch): many slicemaps of uneven sizes,
levels and transfer functions in one persistent launch.  Every image and the
total sample count must be bit-identical to rendering each view alone with
mctp_render_views (the per-view path the oracle checks), for every launch
shape; a subset is also checked against the FP64 oracle directly, and a
CUDA-graph replay must reproduce the eager call."""
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
    return mctp, oracle, phantom, torch.device("cuda:0")


def up(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _slicemaps(env, specs, bits=8):
    """(volume, slicemap, level arrays from the oracle) per (spec, level dims, maxgrid)."""
    mctp, oracle, phantom, dev = env
    out = []
    for spec, dims, grid in specs:
        vol = phantom.generate_cpu(spec)
        nbins = 256 if bits == 8 else 4096
        h, _ = oracle.histogram(vol, bits, nbins)
        keep = oracle.keep_threshold(nbins, oracle.otsu(h)[0])
        sm = mctp.Slicemap.allocate((spec.nx, spec.ny, spec.nz), dims[0], len(dims),
                                    torch.from_numpy(vol[:1, :1, :1]).dtype, bits, dev, maxgrid=grid)
        mctp.build_slicemap(up(vol, dev), bits, sm, up(keep, dev))
        out.append((vol, sm, keep))
    return out


def _luts(phantom, n=256):
    luts = phantom.preset_luts(n)
    opaque0 = luts[3].copy()
    opaque0[0, 3] = 0.05  # entry 0 visible: no cell can be skipped
    return np.stack(luts[:4] + [opaque0])


def _mixed_views(mctp, nsm, nlevels, nluts, count, seed):
    rng = np.random.default_rng(seed)
    views, vsm, vlut = [], [], []
    sizes = [(1, 1), (17, 9), (40, 33), (64, 48), (5, 70), (96, 80)]
    for i in range(count):
        s = int(rng.integers(nsm))
        w, h = sizes[i % len(sizes)]
        views.append(mctp.View(float(rng.uniform(-180, 180)), float(rng.uniform(-60, 60)), w, h,
                               int(rng.integers(nlevels[s])), float(rng.choice([0.5, 0.7, 1.0]))))
        vsm.append(s)
        vlut.append(int(rng.integers(nluts)))
    return views, vsm, vlut


def _alone(mctp, sms, views, vsm, vlut, luts_dev, stop=0.99):
    """Each view rendered by itself with render_views: (flat buffer, total samples)."""
    parts, total = [], 0
    for v, s, l in zip(views, vsm, vlut):
        flat, smp = mctp.render_views(sms[s], [v], luts_dev[l], stop)
        parts.append(flat[:v.width * v.height * 4])
        total += int(smp.item())
    return torch.cat(parts), total


def _specs(phantom):
    V = phantom.VolumeSpec
    return [
        (V(72, 64, 56, bits=8, seed=41, n_ell=5), [(36, 32, 28), (18, 16, 14)], True),
        (V(90, 41, 77, bits=8, seed=42, n_ell=4), [(45, 41, 38)], True),
        (V(48, 48, 48, bits=8, seed=43, n_ell=3), [(24, 24, 24), (12, 12, 12)], False),
        (V(33, 65, 40, bits=8, seed=44, n_ell=3), [(33, 64, 40)], True),
    ]


@pytest.fixture(scope="module")
def mixed(env):
    mctp, oracle, phantom, dev = env
    built = _slicemaps(env, _specs(phantom))
    sms = [b[1] for b in built]
    luts = _luts(phantom)
    luts_dev = up(luts, dev)
    views, vsm, vlut = _mixed_views(mctp, len(sms), [len(sm.dims) for sm in sms], len(luts), 60, seed=7)
    ref, ref_samples = _alone(mctp, sms, views, vsm, vlut, luts_dev)
    return built, sms, luts, luts_dev, views, vsm, vlut, ref, ref_samples


@pytest.mark.parametrize("warp_w,chunk,ctas", [(8, 2, 0), (4, 1, 0), (16, 3, 0), (32, 64, 0), (8, 5, 1)])
def test_batch_equals_views_alone(env, mixed, warp_w, chunk, ctas):
    mctp, oracle, phantom, dev = env
    built, sms, luts, luts_dev, views, vsm, vlut, ref, ref_samples = mixed
    tun = mctp.BatchTuning(warp_w, chunk, ctas)
    flat, samples, _ = mctp.render_batch(sms, views, vsm, vlut, luts_dev, 0.99, tun)
    total = sum(v.width * v.height * 4 for v in views)
    assert torch.equal(flat[:total], ref)
    assert int(samples.item()) == ref_samples


def test_batch_against_oracle(env, mixed):
    """A few batched views straight against the FP64 oracle."""
    mctp, oracle, phantom, dev = env
    built, sms, luts, luts_dev, views, vsm, vlut, ref, ref_samples = mixed
    pick = [i for i, v in enumerate(views) if v.width * v.height <= 40 * 33][:8]
    sub_v = [views[i] for i in pick]
    sub_s = [vsm[i] for i in pick]
    sub_l = [vlut[i] for i in pick]
    flat, samples, _ = mctp.render_batch(sms, sub_v, sub_s, sub_l, luts_dev, 0.99)
    lo_tot = hi_tot = 0
    for v, s, l, img in zip(sub_v, sub_s, sub_l, mctp.images(flat, sub_v)):
        vol, sm, keep = built[s]
        levels = oracle.slicemap(vol, 8, sm.dims, keep)
        r = oracle.render(levels[v.level], 8, sm.src_dims, luts[l], v.azimuth_deg, v.elevation_deg, v.width,
                          v.height, v.step, 0.99, STOP_EPS)
        err, amb = render_error(img.cpu().numpy(), r)
        print(f"batched view {v} lut {l}: max|err| vs FP64 = {err.max():.3e}, ambiguous rays {int(amb.sum())}")
        assert err.max() <= RENDER_TOL
        lo, hi = sample_bounds(r)
        lo_tot += lo
        hi_tot += hi
    assert lo_tot <= int(samples.item()) <= hi_tot


def test_batch_u16_and_global_luts(env):
    """12-bit slicemaps; 4096-entry tables too large for shared memory (read through the cache)."""
    mctp, oracle, phantom, dev = env
    V = phantom.VolumeSpec
    specs = [(V(70, 60, 50, bits=12, seed=45, n_ell=4, n_cyl=10), [(35, 30, 25)], True),
             (V(64, 80, 40, bits=12, seed=46, n_ell=4, n_cyl=10), [(64, 80, 40), (32, 40, 20)], True)]
    built = _slicemaps(env, specs, bits=12)
    sms = [b[1] for b in built]
    rng = np.random.default_rng(9)
    luts = np.stack(phantom.preset_luts(4096, count=4))
    luts[2, :, 3] = rng.uniform(0, 0.3, 4096).astype(np.float32)  # nonzero everywhere: no skipping
    luts_dev = up(luts, dev)
    views, vsm, vlut = _mixed_views(mctp, 2, [1, 2], 4, 24, seed=11)
    ref, ref_samples = _alone(mctp, sms, views, vsm, vlut, luts_dev)
    flat, samples, _ = mctp.render_batch(sms, views, vsm, vlut, luts_dev, 0.99, mctp.BatchTuning(16, 4))
    total = sum(v.width * v.height * 4 for v in views)
    assert torch.equal(flat[:total], ref)
    assert int(samples.item()) == ref_samples


def test_batch_graph_replay_and_empty(env, mixed):
    mctp, oracle, phantom, dev = env
    built, sms, luts, luts_dev, views, vsm, vlut, ref, ref_samples = mixed
    total = sum(v.width * v.height * 4 for v in views)
    out = torch.empty(total, dtype=torch.float32, device=dev)
    samples = torch.empty(1, dtype=torch.uint64, device=dev)
    nb = mctp.render_batch_workspace(sms, views, vsm, vlut, len(luts))
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):  # warm-up outside capture
        mctp.render_batch(sms, views, vsm, vlut, luts_dev, 0.99, out=out, samples=samples, workspace=ws)
    torch.cuda.current_stream(dev).wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        mctp.render_batch(sms, views, vsm, vlut, luts_dev, 0.99, out=out, samples=samples, workspace=ws)
    for _ in range(2):
        out.fill_(-1.0)
        samples.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        assert int(samples.item()) == ref_samples
    # an empty batch renders nothing and counts no samples
    e_out, e_s, _ = mctp.render_batch(sms, [], [], [], luts_dev, 0.99)
    assert int(e_s.item()) == 0


def test_batch_pipeline_graph_and_autotune(env):
    """The batched preview path (per-volume histogram, Otsu, slicemap; one render
    launch) captured as a CUDA graph: replays equal the eager pass, whose images
    equal per-volume render_views calls on slicemaps checked against the oracle."""
    mctp, oracle, phantom, dev = env
    from paper_2311_15038_gb300 import batch as bt
    from paper_2311_15038_gb300 import pipeline as pl
    specs = phantom.batch_specs(3, lo=40, hi=72, seed=5)
    vols = []
    for sp in specs:
        v = torch.empty(sp.shape, dtype=torch.uint8, device=dev)
        phantom.generate_gpu(sp, v)
        vols.append(v)
    luts = up(np.stack(phantom.preset_luts()[:2]), dev)
    views = pl.turntable(3, 24, 0, 0.5, 20.0, 30.0)
    items = [bt.BatchItem(v, 8, views, i % 2) for i, v in enumerate(vols)]
    stream = torch.cuda.Stream(dev)
    pipe = bt.BatchPipeline(items, (32, 32, 32), 1, luts, 256, "otsu", 0.99, device=dev, stream=stream)
    best, timings = pipe.autotune(reps=1)
    assert best in timings and len(timings) >= 4
    with torch.cuda.stream(stream):
        pipe.run()
    torch.cuda.synchronize(dev)
    eager = pipe.images.clone()
    eager_s = int(pipe.samples.item())
    for i, (v, sp) in enumerate(zip(vols, specs)):
        # slicemaps equal the oracle's (Otsu keep table applied)
        cpu = v.cpu().numpy()
        h, _ = oracle.histogram(cpu, 8, 256)
        keep = oracle.keep_threshold(256, oracle.otsu(h)[0])
        lv = oracle.slicemap(cpu, 8, [(32, 32, 32)], keep)[0]
        atlas = oracle.atlas_pack(lv, *pipe.slicemaps[i].tiles[0])
        assert np.array_equal(pipe.slicemaps[i].atlases[0].cpu().numpy(), atlas)
        ref, s = mctp.render_views(pipe.slicemaps[i], views, luts[i % 2], 0.99)
        n = len(views) * 24 * 24 * 4
        assert torch.equal(eager[i * n:(i + 1) * n], ref[:n])
    pipe.capture()
    for _ in range(2):
        pipe.images.fill_(0)
        with torch.cuda.stream(stream):
            pipe.replay()
        torch.cuda.synchronize(dev)
        assert torch.equal(pipe.images, eager)
        assert int(pipe.samples.item()) == eager_s


def test_preview_pipeline_renderers_agree(env):
    """PreviewPipeline renders through the work-queue launch with atlas
    textures by default; its images, sample count and best view equal the
    render_views path and the work-queue launch without textures, before and
    after autotuning the launch shape."""
    mctp, oracle, phantom, dev = env
    from paper_2311_15038_gb300 import pipeline as pl
    spec = phantom.VolumeSpec(150, 130, 90, bits=12, seed=21, n_ell=5)
    vol = torch.from_numpy(phantom.generate_cpu(spec)).to(dev)
    lut = up(phantom.ramp_lut(256), dev)
    views = pl.turntable(5, 40, 0, 0.5, 15.0) + pl.turntable(3, 33, 1, 0.75, -30.0)
    out = {}
    for renderer, tex in (("views", False), ("batch-loads", False), ("batch", True)):
        cfg = pl.PreviewConfig((150, 130, 90), 12, 4096, (64, 64, 48), 2, views, "otsu",
                               renderer=renderer.split("-")[0], texture=tex)
        pipe = pl.PreviewPipeline(cfg, torch.uint16, dev)
        assert (pipe.sm.textures is not None) == tex
        pipe.run(vol, lut)
        torch.cuda.synchronize(dev)
        out[renderer] = (pipe.images.clone(), int(pipe.samples.item()), int(pipe.best.item()))
        if renderer == "batch":
            best, timings = pl.autotune(pipe, lut, reps=1)
            assert best in timings and pipe.tuning == best
            pipe.run(vol, lut)
            torch.cuda.synchronize(dev)
            out["tuned"] = (pipe.images.clone(), int(pipe.samples.item()), int(pipe.best.item()))
    ref = out["views"]
    assert ref[1] > 0
    for k in ("batch-loads", "batch", "tuned"):
        assert torch.equal(out[k][0], ref[0]) and out[k][1:] == ref[1:], k
    with pytest.raises(ValueError):
        pl.PreviewPipeline(pl.PreviewConfig((150, 130, 90), 12, 4096, (64, 64, 48), 2, views, renderer="x"),
                           torch.uint16, dev)


def test_depth_bounds_edge_cases(env):
    """The per-tile depth bounds of the marked cells: a small off-centre object
    (most rays meet no marked cell), views along the axes and straight down,
    steps from 0.05 to 64 voxels (cell skipping off at the largest), 1 x 1 and
    ragged image sizes, a single-level slicemap at both ends of u8: all equal
    to render_views, image and sample count."""
    mctp, oracle, phantom, dev = env
    vol = np.zeros((40, 56, 72), np.uint8)
    vol[30:36, 8:15, 50:61] = 200   # a small block near a corner
    vol[2:4, 40:42, 3:5] = 90
    sm = mctp.Slicemap.allocate((72, 56, 40), (36, 28, 20), 2, torch.uint8, 8, dev)
    mctp.build_slicemap(up(vol, dev), 8, sm, None)
    luts = up(np.stack(phantom.preset_luts()[:2]), dev)
    views = []
    for az, el in [(0.0, 0.0), (90.0, 0.0), (180.0, 0.0), (270.0, 0.0), (0.0, 90.0), (0.0, -90.0), (33.0, 71.0)]:
        for step in (0.05, 0.5, 1.0, 64.0):
            for (w, h) in ((1, 1), (37, 23), (64, 64)):
                views.append(mctp.View(az, el, w, h, int(step > 0.9), step))
    n = len(views)
    vsm, vlut = [0] * n, [i % 2 for i in range(n)]
    ref, ref_s = _alone(mctp, [sm], views, vsm, vlut, luts)
    for tun in (mctp.BatchTuning(8, 1, 0), mctp.BatchTuning(32, 2, 0), mctp.BatchTuning(4, 3, 0)):
        flat, smp, _ = mctp.render_batch([sm], views, vsm, vlut, luts, 0.99, tun)
        assert torch.equal(flat[:ref.numel()], ref) and int(smp.item()) == ref_s, tun
    sm.make_textures()
    sm.update_textures()
    flat, smp, _ = mctp.render_batch([sm], views, vsm, vlut, luts, 0.99)
    assert torch.equal(flat[:ref.numel()], ref) and int(smp.item()) == ref_s


def test_binding_refuses_short_outputs_on_the_device(env):
    """A caller-supplied image buffer one element short, a sample counter of
    the wrong type or a workspace too small is refused before the launch, in
    both batched entry points (the kernels would write past its end)."""
    mctp, oracle, phantom, dev = env
    sms = _slicemaps(env, [(phantom.VolumeSpec(40, 36, 32, bits=8, seed=9, n_ell=3), [(20, 18, 16)], True)])
    views = [mctp.View(20.0, 10.0, 16, 12, 0, 0.5), mctp.View(-40.0, 5.0, 9, 7, 0, 0.5)]
    luts = up(_luts(phantom), dev)
    total = sum(v.width * v.height * 4 for v in views)
    short = torch.empty(total - 1, dtype=torch.float32, device=dev)
    with pytest.raises(ValueError, match="elements"):
        mctp.render_batch([sms[0][1]], views, [0, 0], [0, 1], luts, out=short)
    with pytest.raises(ValueError, match="elements"):
        mctp.render_batch_static([sms[0][1]], views, [0, 0], [0, 1], luts, out=short)
    with pytest.raises(ValueError, match="uint64"):
        mctp.render_batch_static([sms[0][1]], views, [0, 0], [0, 1], luts,
                                 samples=torch.empty(1, dtype=torch.int64, device=dev))
    with pytest.raises(ValueError, match="elements"):
        mctp.render_batch([sms[0][1]], views, [0, 0], [0, 1], luts,
                          workspace=torch.empty(64, dtype=torch.uint8, device=dev))
    # the exact size is accepted and renders what render_views renders
    exact = torch.empty(total, dtype=torch.float32, device=dev)
    out, samples = mctp.render_batch_static([sms[0][1]], views, [0, 0], [0, 1], luts, out=exact)
    ref0, _ = mctp.render_views(sms[0][1], views[:1], luts[0])
    torch.cuda.synchronize()
    assert torch.equal(out[:ref0.numel()], ref0[:16 * 12 * 4])
