"""Atlas textures (mctp_atlas_texture_*): with a texture on a level, the
batched renderer gathers each sample's in-slice corner quads through it.  The
gathered values are the atlas values, so images and sample counts must equal
those of loads from the atlas (which the batch tests tie to render_views and
the FP64 oracle), bit for bit: u8 and 12-bit u16 slicemaps of uneven sizes
(atlas rows with and without whole 16-byte vectors, so both the surface-store
and the 2D-copy update run), every level, rays clamped at the level's faces
and along the axes, an atlas at an unaligned address, a rebuilt slicemap,
and the limits of the texture calls."""
import numpy as np
import pytest

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


def _build(env, spec, dims, bits, grid=True):
    mctp, oracle, phantom, dev = env
    vol = phantom.generate_cpu(spec)
    nbins = 256 if bits == 8 else 4096
    h, _ = oracle.histogram(vol, bits, nbins)
    keep = oracle.keep_threshold(nbins, oracle.otsu(h)[0])
    dt = torch.uint8 if bits == 8 else torch.uint16
    sm = mctp.Slicemap.allocate((spec.nx, spec.ny, spec.nz), dims[0], len(dims), dt, bits, dev, maxgrid=grid)
    mctp.build_slicemap(up(vol, dev), bits, sm, up(keep, dev))
    return sm


def _views(mctp, nlevels, seed):
    rng = np.random.default_rng(seed)
    views = []
    # along the axes and straight down/up: rays on the faces, clamped corners
    for az, el in [(0.0, 0.0), (90.0, 0.0), (180.0, 0.0), (-90.0, 0.0), (0.0, 90.0), (0.0, -90.0), (45.0, 0.0)]:
        for k in range(nlevels):
            views.append(mctp.View(az, el, 37, 29, k, 0.5))
    for i in range(24):
        views.append(mctp.View(float(rng.uniform(-180, 180)), float(rng.uniform(-70, 70)),
                               int(rng.integers(1, 70)), int(rng.integers(1, 70)), int(rng.integers(nlevels)),
                               float(rng.choice([0.4, 0.5, 1.0]))))
    return views


def _render(mctp, sms, views, vsm, luts_dev, tun=None):
    n = len(views)
    flat, smp, _ = mctp.render_batch(sms, views, vsm, [i % luts_dev.shape[0] for i in range(n)], luts_dev, 0.99, tun)
    return flat[:sum(v.width * v.height * 4 for v in views)].clone(), int(smp.item())


CASES = [
    # (spec args, level dims, bits): rows of 45 * tiles u8 texels hold no whole 16-byte vectors
    (dict(nx=90, ny=41, nz=77, seed=42, n_ell=4), [(45, 41, 38)], 8),
    (dict(nx=72, ny=64, nz=56, seed=41, n_ell=5), [(36, 32, 28), (18, 16, 14)], 8),
    (dict(nx=130, ny=120, nz=100, seed=43, n_ell=5), [(64, 64, 48), (32, 32, 24), (16, 16, 12)], 12),
    (dict(nx=61, ny=47, nz=39, seed=44, n_ell=3), [(61, 47, 39)], 12),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_texture_equals_loads(env, case):
    mctp, oracle, phantom, dev = env
    args, dims, bits = CASES[case]
    sm = _build(env, phantom.VolumeSpec(bits=bits, **args), dims, bits)
    luts_dev = up(np.stack(phantom.preset_luts()[:3]), dev)
    views = _views(mctp, len(dims), seed=case)
    vsm = [0] * len(views)
    ref, ref_s = _render(mctp, [sm], views, vsm, luts_dev)
    sm.make_textures()
    sm.update_textures()
    for tun in (mctp.BatchTuning(8, 1, 0), mctp.BatchTuning(4, 2, 0), mctp.BatchTuning(32, 3, 0)):
        got, got_s = _render(mctp, [sm], views, vsm, luts_dev, tun)
        assert torch.equal(got, ref) and got_s == ref_s, tun
    # also without occupancy data (every sample through the gathers)
    bare = sm.without_maxgrid()
    ref2, ref2_s = _render(mctp, [bare.without_textures()], views, vsm, luts_dev)
    got2, got2_s = _render(mctp, [bare], views, vsm, luts_dev)
    assert torch.equal(got2, ref2) and got2_s == ref2_s
    assert torch.equal(got2, ref) and got2_s == ref_s  # skipping is exact


def test_texture_is_what_is_read(env):
    """A stale texture (slicemap rebuilt from another volume, no update) gives
    other images, so the gathers really read the texture; after the update the
    images equal loads from the new atlas again."""
    mctp, oracle, phantom, dev = env
    dims = [(48, 40, 36)]
    sm = _build(env, phantom.VolumeSpec(96, 80, 72, bits=8, seed=51, n_ell=5), dims, 8)
    luts_dev = up(np.stack(phantom.preset_luts()[:1]), dev)
    views = _views(mctp, 1, seed=9)
    vsm = [0] * len(views)
    sm.make_textures()
    sm.update_textures()
    first, _ = _render(mctp, [sm], views, vsm, luts_dev)
    vol2 = phantom.generate_cpu(phantom.VolumeSpec(96, 80, 72, bits=8, seed=52, n_ell=5))
    mctp.build_slicemap(up(vol2, dev), 8, sm, None)
    loads, loads_s = _render(mctp, [sm.without_textures()], views, vsm, luts_dev)
    stale, _ = _render(mctp, [sm], views, vsm, luts_dev)
    assert not torch.equal(stale, loads)
    sm.update_textures()
    fresh, fresh_s = _render(mctp, [sm], views, vsm, luts_dev)
    assert torch.equal(fresh, loads) and fresh_s == loads_s


def test_texture_unaligned_atlas(env):
    """Atlases that start 2 bytes past a 16-byte boundary fill their padded
    textures as aligned ones do; a batch of two slicemaps, both textured,
    renders as loads do."""
    mctp, oracle, phantom, dev = env
    a = _build(env, phantom.VolumeSpec(100, 90, 80, bits=12, seed=61, n_ell=4), [(64, 48, 40), (32, 24, 20)], 12)
    b = _build(env, phantom.VolumeSpec(70, 70, 70, bits=12, seed=62, n_ell=4), [(32, 32, 32)], 12)
    moved = []
    for at in a.atlases:
        buf = torch.zeros(at.numel() + 8, dtype=at.dtype, device=dev)
        view = buf[1:1 + at.numel()].view(at.shape)
        view.copy_(at)
        assert view.data_ptr() % 16 == 2
        moved.append(view)
    a2 = mctp.Slicemap(a.src_dims, a.dims, a.tiles, moved, a.bits, a.dtype, a.maxgrids)
    luts_dev = up(np.stack(phantom.preset_luts()[:2]), dev)
    va = _views(mctp, 2, seed=3)
    vb = _views(mctp, 1, seed=4)
    views = va + vb
    vsm = [0] * len(va) + [1] * len(vb)
    ref, ref_s = _render(mctp, [a, b], views, vsm, luts_dev)
    a2.make_textures()
    a2.update_textures()
    b.make_textures()
    b.update_textures()
    got, got_s = _render(mctp, [a2, b], views, vsm, luts_dev)
    assert torch.equal(got, ref) and got_s == ref_s
    # only one of the two textured: the batch renders from loads, same images
    got3, got3_s = _render(mctp, [a2.without_textures(), b], views, vsm, luts_dev)
    assert torch.equal(got3, ref) and got3_s == ref_s


def test_texture_limits(env):
    mctp, oracle, phantom, dev = env
    from paper_2311_15038_gb300 import _lib
    small = torch.zeros(16, dtype=torch.uint16, device=dev)
    # 40 tiles of 1024 texels: wider than the gather limit (the atlas is never read)
    wide = mctp.Slicemap((1024, 1024, 1024), [(1024, 1024, 1024)], [(40, 26)], [small], 12, torch.uint16)
    with pytest.raises(mctp.MctpError) as e:
        wide.make_textures()
    assert e.value.code == _lib.MCTP_ESIZE
    sm = _build(env, phantom.VolumeSpec(40, 40, 40, bits=8, seed=5, n_ell=2), [(20, 20, 20), (10, 10, 10)], 8)
    t = mctp.AtlasTexture(sm, 0)
    other = _build(env, phantom.VolumeSpec(40, 40, 40, bits=8, seed=6, n_ell=2), [(40, 40, 40)], 8)
    with pytest.raises(mctp.MctpError) as e:
        t.update(other)  # another geometry
    assert e.value.code == _lib.MCTP_EINVAL
    with pytest.raises(mctp.MctpError):
        mctp.AtlasTexture(sm, 2)
    t.close()
    t.close()
    assert t.handle == 0


def test_evaluated_count(env):
    """MCTP_BATCH_COUNT_EVALUATED: the images and sample counts are those of
    the uncounted launch; the evaluated count is the same for every launch
    shape and with or without textures, equals the samples taken when
    nothing can be skipped, and is 0 without the flag."""
    mctp, oracle, phantom, dev = env
    sm = _build(env, phantom.VolumeSpec(120, 100, 90, bits=8, seed=71, n_ell=5), [(60, 50, 44), (30, 25, 22)], 8)
    luts_dev = up(np.stack(phantom.preset_luts()[:2]), dev)
    views = _views(mctp, 2, seed=11)
    n = len(views)
    vsm, vlut = [0] * n, [i % 2 for i in range(n)]
    ref, ref_s = _render(mctp, [sm], views, vsm, luts_dev)
    counts = set()
    for s2 in (sm.without_textures(), sm.make_textures()):
        sm.update_textures()
        for w, c in ((8, 1), (4, 3), (32, 2)):
            flat, smp, ws = mctp.render_batch([s2], views, vsm, vlut, luts_dev, 0.99,
                                              mctp.BatchTuning(w, c, 0, count_evaluated=True))
            total = ref.numel()
            assert torch.equal(flat[:total], ref) and int(smp.item()) == ref_s
            counts.add(mctp.batch_samples_evaluated(ws))
    assert len(counts) == 1
    ev = counts.pop()
    assert 0 < ev < ref_s  # the phantom's background is skipped
    _, _, ws = mctp.render_batch([sm], views, vsm, vlut, luts_dev, 0.99)
    assert mctp.batch_samples_evaluated(ws) == 0
    bare = sm.without_maxgrid()
    _, smp, ws = mctp.render_batch([bare], views, vsm, vlut, luts_dev, 0.99, mctp.BatchTuning(count_evaluated=True))
    assert mctp.batch_samples_evaluated(ws) == int(smp.item())  # no skipping: every sample is evaluated


def test_evaluated_count_matches_marked_samples(env):
    """The evaluated-sample count is the number of samples whose lower corner
    lies in a marked cell, and the sample count is the sum of the rays'
    n: both checked against a host model of the rays (FP32 set-up as the
    kernel, FP64 sample positions) with a transfer function too faint to stop
    a ray, so every ray takes all of its samples."""
    mctp, oracle, phantom, dev = env
    import sys
    import os
    sys.path.insert(0, os.path.dirname(__file__))
    from ray_model import rays
    src = (72, 64, 56)
    dims = [(36, 32, 28), (18, 16, 14)]
    sm = _build(env, phantom.VolumeSpec(*src, bits=8, seed=81, n_ell=5), dims, 8)
    faint = phantom.ramp_lut(256).copy()
    faint[:, 3] *= 0.02  # entry 0 transparent, every other entry slightly opaque: the skip threshold is 0
    luts_dev = up(faint[None], dev)
    # steps below one level voxel, so every view walks the cells (at a step of a
    # whole voxel or more along an axis the march evaluates every sample of its
    # depth range instead)
    views = [mctp.View(az, el, 40, 30, lv, st) for az, el, lv, st in
             [(0.0, 0.0, 0, 0.5), (37.0, 21.0, 0, 0.5), (120.0, -50.0, 1, 0.7), (0.0, 90.0, 0, 0.9),
              (250.0, 10.0, 1, 0.5)]]
    n = len(views)
    sm.make_textures()
    sm.update_textures()
    flat, smp, ws = mctp.render_batch([sm], views, [0] * n, [0] * n, luts_dev, 1.0,
                                      mctp.BatchTuning(8, 1, 0, count_evaluated=True))
    ev = mctp.batch_samples_evaluated(ws)
    taken = int(smp.item())
    N = np.array(src)
    want_taken, want_ev = 0, 0
    for v in views:
        M = np.array(dims[v.level])
        R = rays(N, M, v.azimuth_deg, v.elevation_deg, v.width, v.height, v.step)
        occ = sm.maxgrids[v.level].cpu().numpy() > 0  # [gz][gy][gx]
        sc = M / N
        kmax = int(R["n"].max())
        k = np.arange(kmax)
        t = R["tmin"][..., None].astype(np.float64) + (k + 0.5) * float(R["delta"])
        q = (R["o"][..., None, :].astype(np.float64) + t[..., None] * R["d"].astype(np.float64)) * sc - 0.5
        cell = np.clip(np.floor(q).astype(np.int64), 0, M - 1) >> 3
        valid = k[None, None, :] < R["n"][..., None]
        marked = occ[cell[..., 2], cell[..., 1], cell[..., 0]]
        want_taken += int(R["n"].sum())
        want_ev += int((marked & valid).sum())
    assert taken == want_taken
    assert ev == want_ev
    assert 0 < ev < taken


def test_texture_16bit_and_global_luts(env):
    """Full 16-bit grey values (up to 65535) gathered through u16 textures,
    with 4096-entry transfer functions too large for shared memory (the
    variant that reads them through the cache): equal to loads."""
    mctp, oracle, phantom, dev = env
    spec = phantom.VolumeSpec(90, 70, 64, bits=16, seed=91, n_ell=5, n_cyl=8)
    vol = phantom.generate_cpu(spec)
    assert vol.max() > 4096
    dims = [(64, 48, 32), (32, 24, 16)]
    sm = mctp.Slicemap.allocate((90, 70, 64), dims[0], 2, torch.uint16, 16, dev)
    mctp.build_slicemap(up(vol, dev), 16, sm, None)
    rng = np.random.default_rng(12)
    luts = np.stack(phantom.preset_luts(4096, count=3))
    luts[1, :, 3] = rng.uniform(0, 0.2, 4096).astype(np.float32)  # nonzero everywhere: no skipping
    luts_dev = up(luts, dev)
    views = _views(mctp, 2, seed=13)
    vsm = [0] * len(views)
    ref, ref_s = _render(mctp, [sm], views, vsm, luts_dev)
    sm.make_textures()
    sm.update_textures()
    for tun in (mctp.BatchTuning(8, 1, 0), mctp.BatchTuning(16, 4, 0)):
        got, got_s = _render(mctp, [sm], views, vsm, luts_dev, tun)
        assert torch.equal(got, ref) and got_s == ref_s, tun
