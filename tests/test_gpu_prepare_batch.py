"""Batched preparation of many volumes (mctp_build_histogram_batch,
mctp_select_threshold_batch, mctp_build_slicemap_batch,
mctp_atlas_texture_update_batch): every result must equal the per-volume
entry point on the same volume (histograms, keep tables, atlases, max grids,
rendered textures), and the histograms also the oracle's.  Cases cover more
volumes than one launch takes, volumes that start off a 16-byte boundary,
volumes smaller than one 16-byte vector, and values past 2^bits."""
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


def _volumes(dev, dtype, shapes, bits, seed, offsets=None, top=None):
    """Random volumes, volume i placed `offsets[i]` elements past an aligned allocation."""
    rng = np.random.default_rng(seed)
    out = []
    for i, sh in enumerate(shapes):
        hi = top if top is not None else (1 << bits)
        a = rng.integers(0, hi, size=sh).astype(np.uint8 if dtype == torch.uint8 else np.uint16)
        off = offsets[i] if offsets else 0
        n = int(np.prod(sh))
        buf = torch.zeros(n + off + 16, dtype=dtype, device=dev)
        v = buf[off:off + n].view(sh)
        v.copy_(torch.from_numpy(a).to(dev))
        out.append(v)
    return out


HIST_CASES = [
    # dtype, bits, nbins, shapes, offsets, top
    ("u8_full", torch.uint8, 8, 256, [(9, 13, 17), (1, 1, 5), (20, 33, 41), (3, 7, 31)], [0, 3, 7, 15], None),
    ("u8_64bins", torch.uint8, 8, 64, [(11, 12, 13), (5, 6, 7)], [1, 0], None),
    ("u16_12bit_ovf", torch.uint16, 12, 256, [(7, 9, 33), (2, 3, 5), (13, 17, 19)], [0, 5, 3], 1 << 16),
    ("u16_12bit_4096", torch.uint16, 12, 4096, [(7, 9, 33), (5, 6, 7)], [2, 0], 1 << 16),
    ("u8_many", torch.uint8, 8, 256, [(3 + i % 5, 4 + i % 3, 5 + i % 7) for i in range(70)],
     [i % 16 for i in range(70)], None),
]


@pytest.mark.parametrize("name,dtype,bits,nbins,shapes,offsets,top", HIST_CASES)
def test_histogram_batch_equals_single(env, name, dtype, bits, nbins, shapes, offsets, top):
    mctp, oracle, phantom, dev = env
    vols = _volumes(dev, dtype, shapes, bits, seed=len(name), offsets=offsets, top=top)
    hist, ovf = mctp.build_histogram_batch(vols, bits, nbins)
    for i, v in enumerate(vols):
        h1, o1 = mctp.build_histogram(v, bits, nbins)
        assert torch.equal(hist[i], h1), (name, i)
        assert int(ovf[i].item()) == int(o1.item()), (name, i)
        ref, ref_ov = oracle.histogram(v.cpu().numpy(), bits, nbins)
        assert np.array_equal(hist[i].cpu().numpy(), ref), (name, i)
        assert int(ovf[i].item()) == ref_ov


def test_histogram_batch_refusals(env):
    mctp, oracle, phantom, dev = env
    a = torch.zeros((2, 3, 4), dtype=torch.uint8, device=dev)
    b = torch.zeros((2, 3, 4), dtype=torch.uint16, device=dev)
    with pytest.raises(mctp.MctpError):
        mctp.build_histogram_batch([a, b], 8, 256)          # mixed dtypes
    with pytest.raises(ValueError):
        mctp.build_histogram_batch([a], 8, 256, hist=torch.empty(3, dtype=torch.uint64, device=dev))
    with pytest.raises(mctp.MctpError):
        mctp.build_histogram_batch([a], 8, 100)             # not a power of two


def _slicemaps(mctp, vols, dims_of, bits, dev, maxgrid=True):
    out = []
    for v in vols:
        nz, ny, nx = v.shape
        out.append(mctp.Slicemap.allocate((nx, ny, nz), dims_of(nx, ny, nz), 1 if bits == 8 else 2, v.dtype, bits,
                                          dev, maxgrid=maxgrid))
    return out


@pytest.mark.parametrize("count", [1, 2, 3, 70])
@pytest.mark.parametrize("filtered", [True, False])
def test_slicemap_batch_equals_single(env, count, filtered):
    """u8 volumes take the row kernel (one level); atlases and max grids equal
    per-volume builds, the max grids of all volumes coming from one launch
    (two for 70 volumes).  One volume stays on the caller's stream; from two
    on the builds are spread over forked streams."""
    mctp, oracle, phantom, dev = env
    rng = np.random.default_rng(count + 7 * filtered)
    shapes = [tuple(int(x) for x in rng.integers(9, 40, size=3)) for _ in range(count)]
    vols = _volumes(dev, torch.uint8, shapes, 8, seed=count, offsets=[i % 16 for i in range(count)])
    dims_of = lambda nx, ny, nz: (max(1, nx // 3), max(1, ny // 2), max(1, nz // 3))  # noqa: E731
    keep = None
    if filtered:
        hist, _ = mctp.build_histogram_batch(vols, 8, 256)
        keep, _ = mctp.select_threshold_batch(hist, "otsu")
    batch = _slicemaps(mctp, vols, dims_of, 8, dev)
    mctp.build_slicemap_batch(vols, 8, batch, keep)
    single = _slicemaps(mctp, vols, dims_of, 8, dev)
    for i, v in enumerate(vols):
        mctp.build_slicemap(v, 8, single[i], keep[i] if keep is not None else None)
        for a, b in zip(batch[i].atlases, single[i].atlases):
            assert torch.equal(a, b), i
        for a, b in zip(batch[i].maxgrids, single[i].maxgrids):
            assert torch.equal(a, b), i


def test_slicemap_batch_u16_levels(env):
    """u16 volumes with two levels (the level-0 kernel with a fused level)."""
    mctp, oracle, phantom, dev = env
    shapes = [(20, 24, 28), (17, 19, 23), (30, 16, 18)]
    vols = _volumes(dev, torch.uint16, shapes, 12, seed=3, offsets=[0, 1, 3])
    dims_of = lambda nx, ny, nz: ((nx // 2) & ~1, (ny // 2) & ~1, (nz // 2) & ~1)  # noqa: E731
    hist, _ = mctp.build_histogram_batch(vols, 12, 4096)
    keep, _ = mctp.select_threshold_batch(hist, "its")
    batch = _slicemaps(mctp, vols, dims_of, 12, dev)
    mctp.build_slicemap_batch(vols, 12, batch, keep)
    for i, v in enumerate(vols):
        nz, ny, nx = v.shape
        one = mctp.Slicemap.allocate((nx, ny, nz), dims_of(nx, ny, nz), 2, v.dtype, 12, dev)
        mctp.build_slicemap(v, 12, one, keep[i])
        for a, b in zip(batch[i].atlases, one.atlases):
            assert torch.equal(a, b), i
        for a, b in zip(batch[i].maxgrids, one.maxgrids):
            assert torch.equal(a, b), i


def test_texture_update_batch(env):
    """Textures filled in one launch render exactly as textures filled one by
    one (and as loads from the atlases)."""
    mctp, oracle, phantom, dev = env
    specs = phantom.batch_specs(5, lo=30, hi=70, seed=9)
    vols = []
    for sp in specs:
        v = torch.empty(sp.shape, dtype=torch.uint8, device=dev)
        phantom.generate_gpu(sp, v)
        vols.append(v)
    dims_of = lambda nx, ny, nz: (max(1, nx // 2), max(1, ny // 2), max(1, nz // 2))  # noqa: E731
    sms = _slicemaps(mctp, vols, dims_of, 8, dev)
    mctp.build_slicemap_batch(vols, 8, sms, None)
    for sm in sms:
        sm.make_textures()
    mctp.update_textures_batch(sms)
    from paper_2311_15038_gb300 import pipeline as pl
    views = pl.turntable(2, 20, 0, 0.5, 20.0, 60.0)
    allv, vsm = [], []
    for i in range(len(sms)):
        allv += views
        vsm += [i] * len(views)
    luts = torch.from_numpy(np.stack(phantom.preset_luts()[:1])).to(dev)
    got, got_s, _ = mctp.render_batch(sms, allv, vsm, [0] * len(allv), luts, 0.99)
    ref, ref_s, _ = mctp.render_batch([sm.without_textures() for sm in sms], allv, vsm, [0] * len(allv), luts,
                                      0.99)
    assert torch.equal(got, ref) and int(got_s.item()) == int(ref_s.item())
    for sm in sms:
        sm.update_textures()
    one, one_s, _ = mctp.render_batch(sms, allv, vsm, [0] * len(allv), luts, 0.99)
    assert torch.equal(one, got) and int(one_s.item()) == int(got_s.item())
