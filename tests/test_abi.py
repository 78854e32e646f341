"""The C-ABI library: loads, exports every symbol include/*.h declares, and
rejects bad arguments on the host before touching a GPU.  No compute calls
run here (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2311_15038_gb300 import _lib, build
    build.build()
    return _lib.load()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(mctp_\w+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(lib):
    from paper_2311_15038_gb300 import _lib
    names = _declared()
    assert {"mctp_build_histogram", "mctp_select_threshold", "mctp_filter_threshold", "mctp_build_slicemap",
            "mctp_render_views", "mctp_render_batch", "mctp_render_batch_workspace",
            "mctp_render_batch_static"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n
        assert n in _lib.EXPORTS, f"{n} has no ctypes signature"


def test_host_utilities(lib):
    assert lib.mctp_version() == 1
    tx, ty = ctypes.c_int32(), ctypes.c_int32()
    for mz, want in [(128, (16, 8)), (256, (16, 16)), (512, (32, 16)), (1, (1, 1)), (3, (2, 2))]:
        assert lib.mctp_default_tiles(mz, ctypes.byref(tx), ctypes.byref(ty)) == 0
        assert (tx.value, ty.value) == want
    assert lib.mctp_default_tiles(0, ctypes.byref(tx), ctypes.byref(ty)) == -1
    assert lib.mctp_atlas_bytes(512, 512, 32, 16, 2) == 16384 * 8192 * 2
    assert lib.mctp_atlas_bytes(0, 512, 32, 16, 2) == 0
    assert lib.mctp_atlas_bytes(4, 4, 1, 1, 7) == 0
    assert lib.mctp_maxgrid_bytes(512, 512, 512) == 64 ** 3 * 2
    assert lib.mctp_maxgrid_bytes(9, 8, 17) == 2 * 1 * 3 * 2
    assert lib.mctp_maxgrid_bytes(0, 8, 8) == 0
    for code in (0, -1, -2, -3, -4):
        assert lib.mctp_status_string(code)
    assert lib.mctp_status_string(-99) == b"unknown status"


def _desc(nx=8, ny=8, nz=8, dtype=1, bits=8):
    from paper_2311_15038_gb300 import _lib
    return _lib.VolumeDesc(nx, ny, nz, dtype, bits)


FAKE = ctypes.c_void_p(0x10000)   # never dereferenced: every call below fails its host checks


@pytest.mark.parametrize("desc,z0,z1,nbins,want", [
    (dict(), 0, 8, 256, None),                 # null outputs -> EINVAL (checked separately)
    (dict(nx=0), 0, 8, 256, -1),
    (dict(dtype=1, bits=12), 0, 8, 256, -2),
    (dict(dtype=3), 0, 8, 256, -2),
    (dict(dtype=2, bits=17), 0, 8, 256, -2),
    (dict(), 0, 9, 256, -1),
    (dict(), 5, 4, 256, -1),
    (dict(), -1, 4, 256, -1),
    (dict(), 0, 8, 3, -1),
    (dict(), 0, 8, 512, -1),
    (dict(dtype=2, bits=12), 0, 8, 8192, -1),
])
def test_histogram_rejects(lib, desc, z0, z1, nbins, want):
    d = _desc(**desc)
    if want is None:
        assert lib.mctp_build_histogram(FAKE, ctypes.byref(d), z0, z1, nbins, None, FAKE, None) == -1
        assert lib.mctp_build_histogram(None, ctypes.byref(d), z0, z1, nbins, FAKE, FAKE, None) == -1
        assert lib.mctp_build_histogram(FAKE, None, z0, z1, nbins, FAKE, FAKE, None) == -1
    else:
        assert lib.mctp_build_histogram(FAKE, ctypes.byref(d), z0, z1, nbins, FAKE, FAKE, None) == want


def test_select_threshold_rejects(lib):
    from paper_2311_15038_gb300 import _lib
    p = _lib.ThrParams(0, 0, 256, 0, 1)
    assert lib.mctp_select_threshold(FAKE, 3, ctypes.byref(p), FAKE, None, None) == -1
    assert lib.mctp_select_threshold(FAKE, 0, ctypes.byref(p), FAKE, None, None) == -1
    assert lib.mctp_select_threshold(FAKE, 131072, ctypes.byref(p), FAKE, None, None) == -1
    assert lib.mctp_select_threshold(None, 256, ctypes.byref(p), FAKE, None, None) == -1
    assert lib.mctp_select_threshold(FAKE, 256, ctypes.byref(p), None, None, None) == -1
    assert lib.mctp_select_threshold(FAKE, 256, None, FAKE, None, None) == -1
    bad_mode = _lib.ThrParams(9, 0, 256, 0, 1)
    assert lib.mctp_select_threshold(FAKE, 256, ctypes.byref(bad_mode), FAKE, None, None) == -2
    its0 = _lib.ThrParams(1, 0, 0, 0, 1)
    assert lib.mctp_select_threshold(FAKE, 256, ctypes.byref(its0), FAKE, None, None) == -1
    kmin0 = _lib.ThrParams(2, 0, 256, 0, 0)
    assert lib.mctp_select_threshold(FAKE, 256, ctypes.byref(kmin0), FAKE, None, None) == -1


def test_filter_rejects(lib):
    d = _desc()
    assert lib.mctp_filter_threshold(None, ctypes.byref(d), FAKE, 256, FAKE, None) == -1
    assert lib.mctp_filter_threshold(FAKE, ctypes.byref(d), None, 256, FAKE, None) == -1
    assert lib.mctp_filter_threshold(FAKE, ctypes.byref(d), FAKE, 100, FAKE, None) == -1
    # partial overlap of input and output
    assert lib.mctp_filter_threshold(ctypes.c_void_p(0x10000), ctypes.byref(d), FAKE, 256,
                                     ctypes.c_void_p(0x10010), None) == -1


def _slicemap(levels, src=(64, 64, 64), tiles=None, dtype=1, bits=8):
    from paper_2311_15038_gb300 import _lib
    s = _lib.SlicemapDesc()
    s.nlevels = len(levels)
    s.dtype, s.bits = dtype, bits
    for a in range(3):
        s.src_dims[a] = src[a]
    for k, d in enumerate(levels):
        for a in range(3):
            s.dims[k][a] = d[a]
        tx, ty = tiles[k] if tiles else (8, 8)
        s.tiles_x[k], s.tiles_y[k] = tx, ty
        s.atlas[k] = 0x10000
        s.maxgrid[k] = None
    return s


@pytest.mark.parametrize("levels,tiles,want", [
    ([(65, 32, 32)], None, -1),                       # level larger than the source
    ([(32, 32, 32), (16, 16, 15)], None, -1),        # not an exact halving
    ([(31, 32, 32), (15, 16, 16)], None, -1),        # odd dimension halved
    ([(32, 32, 32)], [(4, 4)], -3),                   # 16 tiles for 32 slices
    ([], None, -1),
])
def test_slicemap_rejects(lib, levels, tiles, want):
    d = _desc(64, 64, 64)
    s = _slicemap(levels, tiles=tiles)
    assert lib.mctp_build_slicemap(FAKE, ctypes.byref(d), None, 0, ctypes.byref(s), None) == want


def test_slicemap_rejects_mismatched_source(lib):
    d = _desc(64, 64, 60)
    s = _slicemap([(32, 32, 32)])
    assert lib.mctp_build_slicemap(FAKE, ctypes.byref(d), None, 0, ctypes.byref(s), None) == -1
    d2 = _desc(64, 64, 64, dtype=2, bits=12)
    assert lib.mctp_build_slicemap(FAKE, ctypes.byref(d2), None, 0, ctypes.byref(s), None) == -1


def test_render_rejects(lib):
    from paper_2311_15038_gb300 import _lib
    s = _slicemap([(32, 32, 32)])
    v = (_lib.ViewDesc * 1)(_lib.ViewDesc(0.0, 0.0, 16, 16, 0, 0.5))
    ok = dict(views=v, n=1, lut=FAKE, nlut=256, stop=0.99, out=FAKE)

    def call(**kw):
        a = dict(ok, **kw)
        return lib.mctp_render_views(ctypes.byref(s), a["views"], a["n"], a["lut"], a["nlut"], a["stop"],
                                     a["out"], None, None)
    assert call(nlut=1) == -1
    assert call(nlut=5000) == -1
    assert call(stop=0.0) == -1
    assert call(stop=1.5) == -1
    assert call(lut=None) == -1
    assert call(out=ctypes.c_void_p(0x10004)) == -1                   # misaligned output
    bad = (_lib.ViewDesc * 1)(_lib.ViewDesc(0.0, 0.0, 16, 16, 1, 0.5))  # level out of range
    assert call(views=bad) == -1
    bad = (_lib.ViewDesc * 1)(_lib.ViewDesc(0.0, 0.0, 0, 16, 0, 0.5))
    assert call(views=bad) == -1
    bad = (_lib.ViewDesc * 1)(_lib.ViewDesc(0.0, 0.0, 16, 16, 0, 0.0))
    assert call(views=bad) == -1
    big = (_lib.ViewDesc * 1)(_lib.ViewDesc(0.0, 0.0, 1 << 15, 1 << 14, 0, 0.5))
    assert call(views=big) == -3


def _batch(lib, sms, views, vsm, vlut, nluts):
    from paper_2311_15038_gb300 import _lib
    S = (_lib.SlicemapDesc * len(sms))(*sms)
    V = (_lib.ViewDesc * len(views))(*[_lib.ViewDesc(*v) for v in views])
    A = (ctypes.c_int32 * len(vsm))(*vsm)
    B = (ctypes.c_int32 * len(vlut))(*vlut)
    return S, V, A, B


def test_render_batch_workspace(lib):
    s1 = _slicemap([(32, 32, 32), (16, 16, 16)])
    s2 = _slicemap([(64, 48, 40)], src=(64, 48, 40), tiles=[(8, 5)])
    s2.maxgrid[0] = 0x20000
    nb = ctypes.c_size_t()

    def size(views, vsm, vlut, nluts=2, sms=(s1, s2)):
        S, V, A, B = _batch(lib, sms, views, vsm, vlut, nluts)
        rc = lib.mctp_render_batch_workspace(S, len(sms), V, A, B, len(views), nluts, ctypes.byref(nb))
        return rc, nb.value

    one = (0.0, 0.0, 16, 16, 0, 0.5)
    rc, base = size([one], [0], [0])
    assert rc == 0 and base > 0 and base % 256 == 0
    # a second view of the same (slicemap, level, LUT) adds only its record
    rc, same = size([one, one], [0, 0], [0, 0])
    assert rc == 0 and base <= same <= base + 512
    # another LUT on a slicemap with a max grid adds slice offsets and a bitmap
    rc, a = size([one, one], [1, 1], [0, 0])
    rc2, b = size([one, one], [1, 1], [0, 1])
    assert rc == rc2 == 0 and b >= a + 2 * 256
    assert size([one], [2], [0])[0] == -1                    # slicemap index out of range
    assert size([one], [0], [2])[0] == -1                    # LUT index out of range
    assert size([(0.0, 0.0, 16, 16, 2, 0.5)], [0], [0])[0] == -1   # level out of range
    s3 = _slicemap([(32, 32, 32)], dtype=2, bits=12)
    assert size([one], [0], [0], sms=(s1, s3))[0] == -2      # one element type per batch


def test_render_batch_rejects(lib):
    from paper_2311_15038_gb300 import _lib
    s1 = _slicemap([(32, 32, 32)])
    S, V, A, B = _batch(lib, [s1], [(0.0, 0.0, 16, 16, 0, 0.5)], [0], [0], 1)
    nb = ctypes.c_size_t()
    assert lib.mctp_render_batch_workspace(S, 1, V, A, B, 1, 1, ctypes.byref(nb)) == 0
    WS = ctypes.c_void_p(0x100000)
    ok = dict(lut=FAKE, nluts=1, nlut=256, stop=0.99, tun=None, out=FAKE, ws=WS, wsb=nb.value)

    def call(**kw):
        a = dict(ok, **kw)
        t = a["tun"]
        return lib.mctp_render_batch(S, 1, V, A, B, 1, a["lut"], a["nluts"], a["nlut"], a["stop"],
                                     ctypes.byref(t) if t is not None else None, a["out"], None, a["ws"],
                                     a["wsb"], None)
    assert call(wsb=nb.value - 1) == -3                      # workspace too small
    assert call(ws=ctypes.c_void_p(0x100010)) == -1          # workspace not 256-byte aligned
    assert call(ws=None) == -1
    assert call(nlut=1) == -1
    assert call(stop=0.0) == -1
    assert call(lut=ctypes.c_void_p(0x10004)) == -1
    assert call(out=None) == -1
    for w, c, k in [(2, 1, 0), (64, 1, 0), (12, 1, 0), (8, 65, 0), (8, -1, 0), (8, 1, -1)]:
        assert call(tun=_lib.BatchTuning(w, c, k, 0)) == -1
    assert call(tun=_lib.BatchTuning(8, 2, 0, 2)) == -1      # unknown flag


def test_render_batch_static_rejects_oversized_batch(lib):
    from paper_2311_15038_gb300 import _lib
    # a 1600^3 level with a max grid needs a ~1.1 MiB cell bitmap per transfer
    # function: eight of them exceed the fixed scratch and are refused on the host
    big = _slicemap([(1600, 1600, 1600)], src=(1600, 1600, 1600), tiles=[(64, 25)])
    big.maxgrid[0] = 0x20000
    n = 8
    views = [(0.0, 0.0, 16, 16, 0, 0.5)] * n
    S, V, A, B = _batch(lib, [big], views, [0] * n, list(range(n)), n)
    nb = ctypes.c_size_t()
    assert lib.mctp_render_batch_workspace(S, 1, V, A, B, n, n, ctypes.byref(nb)) == 0
    assert nb.value > _lib.MCTP_BATCH_STATIC_SCRATCH
    assert lib.mctp_render_batch_static(S, 1, V, A, B, n, FAKE, n, 256, 0.99, None, FAKE, None, None) == -3
    # bad arguments are refused as by mctp_render_batch
    assert lib.mctp_render_batch_static(S, 1, V, A, B, n, FAKE, n - 1, 256, 0.99, None, FAKE, None, None) == -1


def test_server_rejects(lib):
    from paper_2311_15038_gb300 import _lib
    s1 = _slicemap([(32, 32, 32)])
    S = (_lib.SlicemapDesc * 1)(s1)
    out = ctypes.c_void_p()
    ARENA = ctypes.c_void_p(0x1000000)

    def create(mode=0, views=64, inflight=2, reserved=0, arena=ARENA, nbytes=1 << 30, nlut=256, stop=0.99,
               sms=S, nsm=1, handle=True):
        p = _lib.ServeParams(mode, views, inflight, reserved, _lib.BatchTuning(0, 0, 0, 0))
        return lib.mctp_server_create(sms, nsm, FAKE, 1, nlut, stop, arena, nbytes, ctypes.byref(p),
                                      ctypes.byref(out) if handle else None)
    assert create(handle=False) == -1
    assert create(mode=2) == -1
    assert create(inflight=0) == -1
    assert create(inflight=9) == -1
    assert create(views=0) == -1
    assert create(views=5000) == -1
    assert create(reserved=1) == -1
    assert create(arena=ctypes.c_void_p(0x1000010)) == -1    # arena not 256-byte aligned
    assert create(nlut=1) == -1
    assert create(stop=0.0) == -1
    assert create(nbytes=4096) == -3                          # smaller than counters + batch workspaces
    s3 = _slicemap([(32, 32, 32)], dtype=2, bits=12)
    assert create(sms=(_lib.SlicemapDesc * 2)(s1, s3), nsm=2) == -2
    # calls on no server
    tk = ctypes.c_uint64()
    v = _lib.ViewDesc(0.0, 0.0, 8, 8, 0, 0.5)
    n = ctypes.c_int32()
    assert lib.mctp_server_submit(None, ctypes.byref(v), 0, 0, ctypes.byref(tk)) == -1
    assert lib.mctp_server_poll(None, None, 0, ctypes.byref(n)) == -1
    assert lib.mctp_server_release(None, 1) == -1
    assert lib.mctp_server_stats(None, None, None, None) == -1
    assert lib.mctp_server_destroy(None) == -1
    assert lib.mctp_now() > 0.0


def test_dense_rejects(lib):
    from paper_2311_15038_gb300 import _lib
    src = (ctypes.c_int64 * 3)(64, 64, 64)
    v = (_lib.ViewDesc * 1)(_lib.ViewDesc(0.0, 0.0, 16, 16, 0, 0.5))
    v1 = (_lib.ViewDesc * 1)(_lib.ViewDesc(0.0, 0.0, 16, 16, 1, 0.5))      # only level 0 exists
    fine = (_lib.ViewDesc * 1)(_lib.ViewDesc(0.0, 0.0, 16, 16, 0, 1.0 / 256))  # rays of > 2048 samples

    def fwd(vol=FAKE, m=(16, 16, 16), views=v, lut=FAKE, nlut=16, stop=0.99, out=FAKE, srcd=src):
        return lib.mctp_render_dense(vol, *m, srcd, views, 1, lut, nlut, stop, out, None, None)
    assert fwd(vol=None) == -1
    assert fwd(m=(0, 16, 16)) == -1
    assert fwd(views=v1) == -1
    assert fwd(nlut=1) == -1
    assert fwd(stop=1.5) == -1
    assert fwd(out=ctypes.c_void_p(0x10004)) == -1
    assert fwd(srcd=None) == -1
    assert fwd(m=(2048, 2048, 1024)) == -3
    assert lib.mctp_render_dense_backward(FAKE, 16, 16, 16, src, fine, 1, FAKE, 16, 0.99, FAKE, FAKE, FAKE,
                                          None) == -3  # refused on the host before anything is enqueued
    assert lib.mctp_render_dense_backward(FAKE, 16, 16, 16, src, v, 1, FAKE, 16, 0.99, None, FAKE, FAKE, None) == -1
    assert lib.mctp_l2_loss(None, FAKE, 4, 1.0, None, FAKE, None) == -1
    assert lib.mctp_adam_step(FAKE, FAKE, FAKE, FAKE, 4, 0.1, 0.9, 0.999, 1e-8, 0, 0.0, 1.0, None) == -1
    assert lib.mctp_adam_step(FAKE, FAKE, FAKE, FAKE, 4, 0.1, 1.0, 0.999, 1e-8, 1, 0.0, 1.0, None) == -1


def test_no_fallback_when_library_missing(tmp_path, monkeypatch):
    from paper_2311_15038_gb300 import _lib, build
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()


def test_atlas_texture_rejects(lib):
    """Argument checks of the atlas-texture calls, all before any CUDA call."""
    s = _slicemap([(32, 32, 32), (16, 16, 16)])
    out, h = ctypes.c_void_p(), ctypes.c_uint64()
    assert lib.mctp_atlas_texture_create(ctypes.byref(s), 0, None, ctypes.byref(h)) == -1
    assert lib.mctp_atlas_texture_create(ctypes.byref(s), 0, ctypes.byref(out), None) == -1
    assert lib.mctp_atlas_texture_create(None, 0, ctypes.byref(out), ctypes.byref(h)) == -1
    for level in (-1, 2):
        assert lib.mctp_atlas_texture_create(ctypes.byref(s), level, ctypes.byref(out), ctypes.byref(h)) == -1
        assert out.value is None and h.value == 0
    bad = _slicemap([(32, 32, 32)], tiles=[(4, 4)])  # 16 tiles for 32 slices
    assert lib.mctp_atlas_texture_create(ctypes.byref(bad), 0, ctypes.byref(out), ctypes.byref(h)) == -3
    assert lib.mctp_atlas_texture_update(None, ctypes.byref(s), 0, None) == -1
    assert lib.mctp_atlas_texture_destroy(None) == 0


def test_binding_refuses_short_or_mistyped_outputs():
    """The library cannot see the size of a buffer behind a pointer, so the
    binding checks every caller-supplied output before the call: a buffer too
    small for the batch (the kernel would write past its end), of the wrong
    element type, or not on a CUDA device is refused with ValueError."""
    import torch
    import paper_2311_15038_gb300 as mctp
    with pytest.raises(ValueError, match="elements"):
        mctp._out(torch.empty(3, dtype=torch.float32), "out", torch.float32, 16, None)
    with pytest.raises(ValueError, match="float32"):
        mctp._out(torch.empty(64, dtype=torch.float64), "out", torch.float32, 16, None)
    with pytest.raises(ValueError, match="uint64"):
        mctp._out(torch.empty(1, dtype=torch.int64), "samples", torch.uint64, 1, None)
    with pytest.raises(ValueError, match="CUDA"):
        mctp._out(torch.empty(64, dtype=torch.float32), "out", torch.float32, 16, None)


def test_normal_library_is_not_the_checked_build(lib):
    import ctypes
    assert lib.mctp_checked_build() == 0
    bits = ctypes.c_uint32(7)
    assert lib.mctp_checked_status(ctypes.byref(bits), 0) == -2 and bits.value == 0
    assert lib.mctp_checked_selftest(None) == -2


def test_batched_preparation_rejects(lib):
    """The batched entry points check counts, pointers, dtypes and bins on the
    host; an empty batch launches nothing and succeeds."""
    from paper_2311_15038_gb300 import _lib
    d8, d16 = _desc(), _desc(dtype=2, bits=12)
    vols = (ctypes.c_void_p * 2)(0x10000, 0x20000)
    mixed = (_lib.VolumeDesc * 2)(d8, d16)
    same = (_lib.VolumeDesc * 2)(d8, d8)
    # histograms
    assert lib.mctp_build_histogram_batch(vols, same, -1, 256, FAKE, FAKE, None) == -1
    assert lib.mctp_build_histogram_batch(None, same, 2, 256, FAKE, FAKE, None) == -1
    assert lib.mctp_build_histogram_batch(vols, same, 2, 256, None, FAKE, None) == -1
    assert lib.mctp_build_histogram_batch(vols, mixed, 2, 256, FAKE, FAKE, None) == -1
    assert lib.mctp_build_histogram_batch(vols, same, 2, 100, FAKE, FAKE, None) == -1
    assert lib.mctp_build_histogram_batch(vols, same, 2, 512, FAKE, FAKE, None) == -1   # > 2^bits bins
    assert lib.mctp_build_histogram_batch(None, None, 0, 256, None, None, None) == 0
    # keep tables
    p = _lib.ThrParams(0, 0, 256, 0, 1)
    assert lib.mctp_select_threshold_batch(FAKE, -1, 256, ctypes.byref(p), FAKE, None, None) == -1
    assert lib.mctp_select_threshold_batch(FAKE, 2, 3, ctypes.byref(p), FAKE, None, None) == -1
    assert lib.mctp_select_threshold_batch(None, 2, 256, ctypes.byref(p), FAKE, None, None) == -1
    assert lib.mctp_select_threshold_batch(FAKE, 2, 256, ctypes.byref(p), None, None, None) == -1
    assert lib.mctp_select_threshold_batch(FAKE, 1 << 20, 4096, ctypes.byref(p), FAKE, None, None) == -1
    assert lib.mctp_select_threshold_batch(None, 0, 256, ctypes.byref(p), None, None, None) == 0
    # slicemaps
    sm = (_lib.SlicemapDesc * 2)()
    assert lib.mctp_build_slicemap_batch(vols, same, None, 0, sm, -1, None) == -1
    assert lib.mctp_build_slicemap_batch(None, same, None, 0, sm, 2, None) == -1
    assert lib.mctp_build_slicemap_batch(vols, same, None, 0, None, 2, None) == -1
    assert lib.mctp_build_slicemap_batch(vols, same, None, 0, sm, 2, None) < 0          # empty slicemap descs
    assert lib.mctp_build_slicemap_batch(None, None, None, 0, None, 0, None) == 0
    # textures
    lv = (_lib.C_I32 * 2)(0, 0)
    tex = (ctypes.c_void_p * 2)(None, None)
    assert lib.mctp_atlas_texture_update_batch(tex, sm, lv, -1, None) == -1
    assert lib.mctp_atlas_texture_update_batch(None, sm, lv, 2, None) == -1
    assert lib.mctp_atlas_texture_update_batch(tex, sm, lv, 2, None) == -1              # null textures
    assert lib.mctp_atlas_texture_update_batch(None, None, None, 0, None) == 0


def test_batched_bindings_refuse_host_tensors():
    """The Python bindings refuse CPU tensors and malformed shapes before the library is called."""
    torch = pytest.importorskip("torch")
    import paper_2311_15038_gb300 as mctp
    v = torch.zeros((2, 3, 4), dtype=torch.uint8)
    with pytest.raises(ValueError):
        mctp.build_histogram_batch([v], 8, 256)
    with pytest.raises(ValueError):
        mctp.build_histogram_batch([], 8, 256)
    with pytest.raises(ValueError):
        mctp.select_threshold_batch(torch.zeros((2, 256), dtype=torch.int64))
    with pytest.raises(ValueError):
        mctp.build_slicemap_batch([v], 8, [])
