"""GPU parity: every C-ABI entry point against the CPU oracle on the same
seeded inputs.  Integer outputs (histograms, thresholds, keep tables,
filtered volumes, atlases) must match bit for bit; rendered RGBA within
2e-4 per channel of the FP64 oracle, with the error printed per result.
Sizes span several tiles with ragged tails; edge cases cover empty slabs,
unaligned bases, overflow values, one-bin histograms, 65536 bins, keep-all /
keep-none tables, multi-launch view lists and rays along the box axes."""
import zlib

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


# ---------------------------------------------------------------- histogram

HIST_CASES = [
    ("phantom256", None, 8, 256),
    ("u8_ragged", (23, 29, 37), 8, 256),
    ("u8_64bins", (23, 29, 37), 8, 64),
    ("u8_1bin", (5, 7, 11), 8, 1),
    ("u16_12bit_ovf", (17, 31, 45), 12, 4096),
    ("u16_12bit_512", (17, 31, 45), 12, 512),
    ("u16_12bit_256_ovf", (19, 33, 47), 12, 256),   # lane-column kernel with the overflow check
    ("u16_16bit_65536", (9, 33, 41), 16, 65536),
]


@pytest.mark.parametrize("name,shape,bits,nbins", HIST_CASES)
def test_histogram(env, name, shape, bits, nbins):
    mctp, oracle, phantom, dev = env
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    if shape is None:
        vol = phantom.generate_cpu(phantom.SMALL)
    elif bits == 8:
        vol = rng.integers(0, 256, size=shape).astype(np.uint8)
    else:
        vol = rng.integers(0, 65536 if "ovf" in name or bits == 16 else 1 << bits, size=shape).astype(np.uint16)
    g = up(vol, dev)
    nz = vol.shape[0]
    for z0, z1 in [(0, nz), (1, nz - 1), (2, 2), (nz - 1, nz)]:
        h, ov = mctp.build_histogram(g, bits, nbins, z0, z1)
        ref, ref_ov = oracle.histogram(vol, bits, nbins, z0, z1)
        assert np.array_equal(h.cpu().numpy(), ref), (name, z0, z1)
        assert int(ov.item()) == ref_ov


# ---------------------------------------------------------------- threshold

def _hists(oracle, phantom):
    rng = np.random.default_rng(4)
    out = {}
    v = phantom.generate_cpu(phantom.SMALL)
    out["phantom"] = oracle.histogram(v, 8, 256)[0]
    for nb in (1, 2, 16, 256, 4096, 65536):
        h = rng.integers(0, 1000, size=nb).astype(np.uint64)
        h[rng.integers(0, nb, size=max(1, nb // 4))] = 0
        out[f"random{nb}"] = h
    big = np.zeros(4096, np.uint64)
    big[300:400] = 10 ** 9            # counts near those of a 7e9-voxel volume
    big[2000:2100] = 7 * 10 ** 8
    out["huge_counts"] = big
    out["golden"] = np.array([2, 0, 1, 1, 0, 2], np.uint64)[:4]  # 4 bins (power of two)
    two = np.zeros(256, np.uint64)
    two[3], two[200] = 13, 4
    out["two_delta"] = two
    out["empty"] = np.zeros(64, np.uint64)
    one = np.zeros(16, np.uint64)
    one[10] = 5
    out["single"] = one
    return out


def test_select_threshold(env):
    mctp, oracle, phantom, dev = env
    for name, h in _hists(oracle, phantom).items():
        nb = h.size
        g = up(h, dev)
        # Otsu
        keep, res = mctp.select_threshold(g, mode="otsu")
        T, _ = oracle.otsu(h)
        r = res.cpu().numpy()
        assert r[0] == T, (name, "otsu", r, T)
        assert np.array_equal(keep.cpu().numpy(), oracle.keep_threshold(nb, T)), name
        # ITS, converged and capped
        for cap in (256, 5, 1):
            keep, res = mctp.select_threshold(g, mode="its", its_max_iter=cap)
            T, it, conv, _ = oracle.its(h, max_iter=cap)
            r = res.cpu().numpy()
            assert (r[0], r[1], r[2]) == (T, it, int(conv)), (name, "its", cap, r, (T, it, conv))
            assert np.array_equal(keep.cpu().numpy(), oracle.keep_threshold(nb, T)), name
        # top-slab filtering and explicit thresholds
        for kmin in (1, 3):
            keep, res = mctp.select_threshold(g, mode="topslab", topslab_kmin=kmin)
            assert np.array_equal(keep.cpu().numpy(), oracle.keep_topslab(h, kmin)), name
            assert res.cpu().numpy()[0] == -1
        for T in (0, nb // 3, nb):
            keep, _ = mctp.select_threshold(None, nbins=nb, mode="explicit", explicit_T=T, device=dev)
            assert np.array_equal(keep.cpu().numpy(), oracle.keep_threshold(nb, T)), name


def test_select_threshold_batch(env):
    """One launch for many histograms: row i equals the single-histogram
    selection of row i (which the test above pins to the oracle)."""
    mctp, oracle, phantom, dev = env
    rng = np.random.default_rng(11)
    for nb, count in ((256, 64), (4096, 5), (1, 3), (16, 1)):
        h = rng.integers(0, 1000, size=(count, nb)).astype(np.uint64)
        h[0, :] = 0                                   # an empty histogram
        if count > 2:
            h[2, :] = 0
            h[2, nb // 2] = 7                         # a single occupied bin
        g = up(h, dev)
        for mode, kw in (("otsu", {}), ("its", dict(its_max_iter=3)), ("topslab", dict(topslab_kmin=2)),
                         ("explicit", dict(explicit_T=nb // 3))):
            keep, res = mctp.select_threshold_batch(g, mode, **kw)
            for i in range(count):
                k1, r1 = mctp.select_threshold(g[i].contiguous(), mode=mode, **kw)
                assert torch.equal(keep[i], k1), (nb, mode, i)
                assert torch.equal(res[i], r1), (nb, mode, i)
            if mode == "otsu":
                for i in range(count):
                    T, _ = oracle.otsu(h[i])
                    assert int(res[i, 0]) == T
    empty = torch.empty((0, 256), dtype=torch.uint64, device=dev)
    keep, res = mctp.select_threshold_batch(empty)
    assert keep.numel() == 0 and res.numel() == 0
    with pytest.raises(ValueError):
        mctp.select_threshold_batch(g, keep=torch.empty(1, dtype=torch.uint8, device=dev))


# ------------------------------------------------------------------- filter

@pytest.mark.parametrize("dtype,bits,nbins,shape", [(np.uint8, 8, 256, (13, 17, 19)), (np.uint8, 8, 16, (8, 8, 64)),
                                                    (np.uint16, 12, 4096, (11, 13, 7)),
                                                    (np.uint16, 12, 64, (3, 5, 1001)), (np.uint8, 8, 1, (2, 3, 5))])
def test_filter(env, dtype, bits, nbins, shape):
    mctp, oracle, phantom, dev = env
    rng = np.random.default_rng(nbins)
    hi = 256 if dtype == np.uint8 else 5000
    vol = rng.integers(0, hi, size=shape).astype(dtype)
    keep = rng.integers(0, 2, size=nbins).astype(np.uint8)
    ref = oracle.filter_volume(vol, bits, keep)
    g = up(vol, dev)
    k = up(keep, dev)
    out = mctp.filter_threshold(g, bits, k)
    assert np.array_equal(out.cpu().numpy(), ref)
    # in place, and on an unaligned sub-range (a slab starting at z = 1)
    mctp.filter_threshold(g, bits, k, out=g)
    assert np.array_equal(g.cpu().numpy(), ref)
    g2 = up(vol, dev)
    sub = g2[1:]
    out2 = torch.empty_like(sub)
    mctp.filter_threshold(sub, bits, k, out=out2)
    assert np.array_equal(out2.cpu().numpy(), ref[1:])


# ----------------------------------------------------------------- slicemap

def _check_atlases(sm, levels, oracle, tiles=None):
    for k, lv in enumerate(levels):
        tx, ty = tiles[k] if tiles else oracle.default_tiles(lv.shape[0])
        ref = oracle.atlas_pack(lv, tx, ty)
        got = sm.atlases[k].cpu().numpy()
        assert got.shape == ref.shape, k
        assert np.array_equal(got, ref), f"level {k}: {(got != ref).sum()} voxels differ"
        if sm.maxgrids is not None:
            assert np.array_equal(sm.maxgrids[k].cpu().numpy(), oracle.maxgrid(lv, 8)), f"maxgrid {k}"


@pytest.mark.parametrize("case", ["small_cfg", "u16_4levels_otsu", "u8_topslab", "scalar_rows", "identity",
                                  "to_one_voxel", "nofilter_u16"])
def test_slicemap(env, case):
    mctp, oracle, phantom, dev = env
    if case == "small_cfg":          # 256^3 u8 -> 128^3, Otsu filter (workload "small")
        vol = phantom.generate_cpu(phantom.SMALL)
        bits, nbins, dims, mode = 8, 256, [(128, 128, 128)], "otsu"
    elif case == "u16_4levels_otsu":
        vol = phantom.generate_cpu(phantom.VolumeSpec(200, 176, 150, bits=12, seed=5, n_ell=8, n_cyl=30))
        bits, nbins, dims, mode = 12, 4096, [(96, 88, 72), (48, 44, 36), (24, 22, 18), (12, 11, 9)], "otsu"
    elif case == "u8_topslab":       # keep table that is not a step: per-voxel lookup
        vol = phantom.generate_cpu(phantom.VolumeSpec(160, 144, 128, bits=8, seed=6, n_ell=8))
        bits, nbins, dims, mode = 8, 256, [(64, 64, 64), (32, 32, 32)], "topslab"
    elif case == "scalar_rows":      # rows not a multiple of 16 bytes
        vol = phantom.generate_cpu(phantom.VolumeSpec(37, 41, 29, bits=8, seed=7, n_ell=4))
        bits, nbins, dims, mode = 8, 256, [(13, 9, 7)], "its"
    elif case == "identity":
        vol = phantom.generate_cpu(phantom.VolumeSpec(48, 40, 24, bits=8, seed=8, n_ell=4))
        bits, nbins, dims, mode = 8, 256, [(48, 40, 24), (24, 20, 12)], "otsu"
    elif case == "to_one_voxel":
        vol = phantom.generate_cpu(phantom.VolumeSpec(16, 24, 8, bits=8, seed=9, n_ell=2))
        bits, nbins, dims, mode = 8, 256, [(4, 4, 4), (2, 2, 2), (1, 1, 1)], "otsu"
    else:
        vol = phantom.generate_cpu(phantom.VolumeSpec(120, 112, 104, bits=12, seed=10, n_ell=6))
        bits, nbins, dims, mode = 12, 4096, [(40, 56, 26), (20, 28, 13)], None
    g = up(vol, dev)
    keep_ref = None
    keep = None
    if mode is not None:
        if mode == "topslab":
            ht, _ = oracle.histogram(vol, bits, nbins, 0, 3)
            keep_ref = oracle.keep_topslab(ht, 1)
            hg, _ = mctp.build_histogram(g, bits, nbins, 0, 3)
            keep, _ = mctp.select_threshold(hg, mode="topslab")
        else:
            h, _ = oracle.histogram(vol, bits, nbins)
            T = oracle.otsu(h)[0] if mode == "otsu" else oracle.its(h)[0]
            keep_ref = oracle.keep_threshold(nbins, T)
            hg, _ = mctp.build_histogram(g, bits, nbins)
            keep, _ = mctp.select_threshold(hg, mode=mode)
        assert np.array_equal(keep.cpu().numpy(), keep_ref)
    sm = mctp.Slicemap.allocate((vol.shape[2], vol.shape[1], vol.shape[0]), dims[0], len(dims),
                                torch.from_numpy(vol[:1, :1, :1]).dtype, bits, dev)
    for a in sm.atlases:
        a.fill_(0x5A)                # unused tiles must be overwritten with zero
    mctp.build_slicemap(g, bits, sm, keep)
    levels = oracle.slicemap(vol, bits, dims, keep_ref)
    _check_atlases(sm, levels, oracle)


@pytest.mark.parametrize("T", [0, 1456, 4096])
def test_slicemap_packed_path_with_out_of_depth_values(env, T):
    # 12-bit volume holding values up to 65535: the step keep table must drop
    # every value >= 4096 (and >= 32768) exactly on the two-lane path
    mctp, oracle, phantom, dev = env
    rng = np.random.default_rng(T)
    vol = rng.integers(0, 65536, size=(64, 48, 40)).astype(np.uint16)
    vol[::3] = rng.integers(0, 4096, size=vol[::3].shape)
    keep_ref = oracle.keep_threshold(4096, T)
    dims = [(16, 16, 16), (8, 8, 8)]
    sm = mctp.Slicemap.allocate((40, 48, 64), dims[0], 2, torch.uint16, 12, dev)
    mctp.build_slicemap(up(vol, dev), 12, sm, up(keep_ref, dev))
    _check_atlases(sm, oracle.slicemap(vol, 12, dims, keep_ref), oracle)


@pytest.mark.parametrize("shape,bits,mode", [((29, 37, 385), 8, "otsu"), ((29, 37, 385), 8, "topslab"),
                                             ((29, 37, 385), 8, None), ((23, 19, 101), 12, "otsu"),
                                             ((23, 19, 101), 12, None), ((40, 33, 999), 8, "its")])
def test_slicemap_unaligned_rows(env, shape, bits, mode):
    # rows that do not start on 16-byte boundaries (the batched workload's
    # volumes have random sizes), plus an unaligned base pointer (z >= 1 slab)
    mctp, oracle, phantom, dev = env
    nz, ny, nx = shape
    spec = phantom.VolumeSpec(nx, ny, nz, bits=bits, seed=nx + ny, n_ell=5)
    full = phantom.generate_cpu(spec)
    for vol in (full, full[1:]):
        vol = np.ascontiguousarray(vol)
        nbins = 256 if bits == 8 else 4096
        keep_ref = None
        if mode == "topslab":
            keep_ref = oracle.keep_topslab(oracle.histogram(vol, bits, nbins, 0, 3)[0], 1)
        elif mode is not None:
            h, _ = oracle.histogram(vol, bits, nbins)
            keep_ref = oracle.keep_threshold(nbins, oracle.otsu(h)[0] if mode == "otsu" else oracle.its(h)[0])
        dims = [(vol.shape[2] // 3 // 2 * 2, vol.shape[1] // 2 // 2 * 2, vol.shape[0] // 2 // 2 * 2)]
        dims.append(tuple(d // 2 for d in dims[0]))
        g = torch.from_numpy(full).to(dev)[1:] if vol.shape != full.shape else up(vol, dev)
        sm = mctp.Slicemap.allocate((vol.shape[2], vol.shape[1], vol.shape[0]), dims[0], 2,
                                    torch.from_numpy(vol[:1, :1, :1]).dtype, bits, dev)
        mctp.build_slicemap(g, bits, sm, up(keep_ref, dev) if keep_ref is not None else None)
        _check_atlases(sm, oracle.slicemap(vol, bits, dims, keep_ref), oracle)


@pytest.mark.parametrize("shape,dims,bits,mode", [
    ((77, 41, 90), (38, 41, 45), 8, "otsu"),      # several level-0 rows per pass, ragged 4 x 4 groups
    ((50, 61, 400), (64, 30, 25), 8, "topslab"),  # table lookup, unaligned 400-byte rows
    ((33, 35, 96), (96, 35, 11), 8, None),        # aligned rows, identity in x and y
    ((21, 30, 70), (33, 13, 7), 12, "otsu"),      # u16, ragged groups
])
def test_slicemap_single_level_groups(env, shape, dims, bits, mode):
    # dims are (mx, my, mz); shape is (nz, ny, nx)
    # one level (nothing fused): a CTA takes 4 x 4 level-0 rows, clipped at the
    # level's edges, and accumulates as many rows at once as its threads cover
    mctp, oracle, phantom, dev = env
    nz, ny, nx = shape
    vol = phantom.generate_cpu(phantom.VolumeSpec(nx, ny, nz, bits=bits, seed=nx * 7 + nz, n_ell=5))
    nbins = 256 if bits == 8 else 4096
    keep_ref = None
    if mode == "topslab":
        keep_ref = oracle.keep_topslab(oracle.histogram(vol, bits, nbins, 0, 3)[0], 1)
    elif mode is not None:
        keep_ref = oracle.keep_threshold(nbins, oracle.otsu(oracle.histogram(vol, bits, nbins)[0])[0])
    sm = mctp.Slicemap.allocate((nx, ny, nz), dims, 1, torch.from_numpy(vol[:1, :1, :1]).dtype, bits, dev)
    mctp.build_slicemap(up(vol, dev), bits, sm, up(keep_ref, dev) if keep_ref is not None else None)
    _check_atlases(sm, oracle.slicemap(vol, bits, [dims], keep_ref), oracle)


@pytest.mark.parametrize("shape,dims,mode,offset", [
    ((40, 36, 1024), (256, 18, 20), "otsu", 0),      # the longest rows the warp-per-row kernel takes
    ((40, 36, 1023), (300, 12, 13), "topslab", 1),   # odd rows, unaligned base, table lookup
    ((64, 64, 100), (50, 4, 4), "its", 0),           # 16 x 16 footprints: 256 rows per level-0 row
    ((9, 7, 1), (1, 3, 2), None, 0),                 # one-byte rows
    ((23, 29, 31), (31, 29, 23), None, 3),           # identity, rows shorter than a lane's 32 bytes
    ((50, 41, 545), (128, 40, 25), "otsu", 5),       # uneven x footprints straddling lanes
])
def test_slicemap_u8_rows_kernel(env, shape, dims, mode, offset):
    """Single u8 levels with rows of at most 1024 bytes (the warp-per-row
    kernel): bit-exact against the oracle for every keep-table kind, any
    row alignment (the volume starts `offset` bytes into its buffer), footprints
    from 1 to 16 voxels per axis."""
    mctp, oracle, phantom, dev = env
    nz, ny, nx = shape
    vol = phantom.generate_cpu(phantom.VolumeSpec(nx, ny, nz, bits=8, seed=nx + 3 * nz, n_ell=5))
    keep_ref = None
    if mode == "topslab":
        keep_ref = oracle.keep_topslab(oracle.histogram(vol, 8, 256, 0, 3)[0], 1)
    elif mode is not None:
        h, _ = oracle.histogram(vol, 8, 256)
        keep_ref = oracle.keep_threshold(256, oracle.otsu(h)[0] if mode == "otsu" else oracle.its(h)[0])
    buf = torch.zeros(vol.size + 64, dtype=torch.uint8, device=dev)
    g = buf[offset:offset + vol.size].view(nz, ny, nx)
    g.copy_(torch.from_numpy(vol))
    sm = mctp.Slicemap.allocate((nx, ny, nz), dims, 1, torch.uint8, 8, dev)
    mctp.build_slicemap(g, 8, sm, up(keep_ref, dev) if keep_ref is not None else None)
    _check_atlases(sm, oracle.slicemap(vol, 8, [dims], keep_ref), oracle)


def test_slicemap_custom_tiles(env):
    mctp, oracle, phantom, dev = env
    vol = phantom.generate_cpu(phantom.VolumeSpec(64, 48, 52, bits=8, seed=12, n_ell=4))
    g = up(vol, dev)
    dims, tiles = [(32, 24, 26), (16, 12, 13)], [(3, 9), (5, 3)]
    atl = [torch.full((ty * d[1], tx * d[0]), 7, dtype=torch.uint8, device=dev) for d, (tx, ty) in zip(dims, tiles)]
    sm = mctp.Slicemap((64, 48, 52), dims, tiles, atl, 8, torch.uint8)
    mctp.build_slicemap(g, 8, sm, None)
    _check_atlases(sm, oracle.slicemap(vol, 8, dims, None), oracle, tiles)


# ------------------------------------------------------------------- render

def _render_case(env, vol, bits, dims, views, lut, stop=0.99, keep_mode="otsu", nbins=256):
    mctp, oracle, phantom, dev = env
    g = up(vol, dev)
    keep = keep_ref = None
    if keep_mode:
        h, _ = oracle.histogram(vol, bits, nbins)
        keep_ref = oracle.keep_threshold(nbins, oracle.otsu(h)[0])
        keep = up(keep_ref, dev)
    sm = mctp.Slicemap.allocate((vol.shape[2], vol.shape[1], vol.shape[0]), dims[0], len(dims),
                                torch.from_numpy(vol[:1, :1, :1]).dtype, bits, dev)
    mctp.build_slicemap(g, bits, sm, keep)
    levels = oracle.slicemap(vol, bits, dims, keep_ref)
    _check_atlases(sm, levels, oracle)
    flat, samples = mctp.render_views(sm, views, up(lut, dev), stop)
    # skipping zero-opacity cells is exact: the same images and counts as a full march
    flat_full, samples_full = mctp.render_views(sm.without_maxgrid(), views, up(lut, dev), stop)
    assert torch.equal(flat, flat_full)
    assert int(samples.item()) == int(samples_full.item())
    imgs = mctp.images(flat, views)
    lo_tot = hi_tot = 0
    worst = 0.0
    for v, img in zip(views, imgs):
        ref = oracle.render(levels[v.level], bits, (vol.shape[2], vol.shape[1], vol.shape[0]), lut,
                            v.azimuth_deg, v.elevation_deg, v.width, v.height, v.step, stop, STOP_EPS)
        err, amb = render_error(img.cpu().numpy(), ref)
        print(f"view az={v.azimuth_deg} el={v.elevation_deg} {v.width}x{v.height} level {v.level}: "
              f"max|err| vs FP64 = {err.max():.3e}, ambiguous rays {int(amb.sum())}")
        assert err.max() <= RENDER_TOL
        worst = max(worst, float(err.max()))
        lo, hi = sample_bounds(ref)
        lo_tot += lo
        hi_tot += hi
    s = int(samples.item())
    assert lo_tot <= s <= hi_tot, (lo_tot, s, hi_tot)
    return worst


def test_render_small_workload(env):
    """Workload 'small': 256^3 u8 phantom, Otsu, 128^3 level, one view 256x256, az=el=0, step 0.5."""
    mctp, oracle, phantom, dev = env
    vol = phantom.generate_cpu(phantom.SMALL)
    views = [mctp.View(0.0, 0.0, 256, 256, 0, 0.5)]
    _render_case(env, vol, 8, [(128, 128, 128)], views, phantom.ramp_lut(256))


def test_render_oblique_multilevel_u16(env):
    mctp, oracle, phantom, dev = env
    vol = phantom.generate_cpu(phantom.VolumeSpec(150, 130, 110, bits=12, seed=21, n_ell=8, n_cyl=20))
    views = [mctp.View(37.0, 21.0, 100, 77, 0, 0.5), mctp.View(-123.5, -40.0, 61, 90, 1, 0.7),
             mctp.View(10.0, 0.0, 33, 17, 2, 0.25)]
    luts = phantom.preset_luts()
    _render_case(env, vol, 12, [(64, 64, 48), (32, 32, 24), (16, 16, 12)], views, luts[3], nbins=4096)


def test_render_axis_views_and_grazing(env):
    mctp, oracle, phantom, dev = env
    vol = phantom.generate_cpu(phantom.VolumeSpec(72, 64, 56, bits=8, seed=22, n_ell=5))
    views = [mctp.View(0.0, 0.0, 40, 40, 0), mctp.View(90.0, 0.0, 40, 40, 0), mctp.View(0.0, 90.0, 40, 40, 0),
             mctp.View(180.0, -90.0, 41, 39, 0), mctp.View(45.0, 35.264389682754654, 48, 48, 0)]
    _render_case(env, vol, 8, [(36, 32, 28)], views, phantom.preset_luts()[5])


def test_render_many_views_two_launches(env):
    mctp, oracle, phantom, dev = env
    vol = phantom.generate_cpu(phantom.VolumeSpec(48, 48, 48, bits=8, seed=23, n_ell=4))
    views = [mctp.View(5.0 * i, 10.0 * ((i % 7) - 3), 9 + i % 5, 7 + i % 3, i % 2, 0.5) for i in range(70)]
    _render_case(env, vol, 8, [(24, 24, 24), (12, 12, 12)], views, phantom.ramp_lut(256))


def test_render_constant_slab_no_early_exit(env):
    mctp, oracle, phantom, dev = env
    vol = np.full((20, 24, 28), 180, np.uint8)
    lut = np.array([[0.2, 0.5, 0.9, 0.03], [0.2, 0.5, 0.9, 0.03]], np.float32)
    views = [mctp.View(30.0, 10.0, 32, 32, 0, 0.5)]
    _render_case(env, vol, 8, [(14, 12, 10)], views, lut, stop=1.0, keep_mode=None)


def test_render_big_lut_and_empty(env):
    mctp, oracle, phantom, dev = env
    rng = np.random.default_rng(3)
    vol = phantom.generate_cpu(phantom.VolumeSpec(40, 36, 32, bits=8, seed=24, n_ell=3))
    lut = rng.uniform(0, 1, size=(4096, 4)).astype(np.float32)
    lut[:, 3] *= 0.2
    _render_case(env, vol, 8, [(20, 18, 16)], [mctp.View(12.0, 34.0, 30, 30, 0, 0.5)], lut)
    empty = np.zeros((16, 16, 16), np.uint8)
    _render_case(env, empty, 8, [(8, 8, 8)], [mctp.View(12.0, 34.0, 20, 20, 0, 0.5)], phantom.ramp_lut(256),
                 keep_mode=None)
    # no views: nothing rendered, sample count zero
    sm = mctp.Slicemap.allocate((16, 16, 16), (8, 8, 8), 1, torch.uint8, 8, dev)
    mctp.build_slicemap(up(empty, dev), 8, sm)
    out = torch.zeros(4, dtype=torch.float32, device=dev)
    _, s = mctp.render_views(sm, [], up(phantom.ramp_lut(256), dev), 0.99, out=out)
    assert int(s.item()) == 0
