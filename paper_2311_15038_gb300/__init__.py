"""GB300 micro-CT preview library: Python binding of libmctp (include/mctp.h).

Every function here only marshals arguments (torch CUDA tensors -> device
pointers, the current CUDA stream) and calls the C ABI of the same name; the
work runs in the library's sm_103a kernels.  Hot path of "Low-latency Visual
Previews of Large Synchrotron Micro-CT Datasets" (arXiv 2311.15038):
histogram (Sec. III-A), threshold selection (Alg. 1, Alg. 2, Sec. III-D),
keep/discard filter (Sec. III-A), slicemap atlases (Sec. II, III) and
server-side rendering (Sec. III-C).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import MctpError  # noqa: F401

__all__ = ["build_histogram", "build_histogram_batch", "build_slicemap_batch", "update_textures_batch",
           "select_threshold", "select_threshold_batch", "filter_threshold", "build_slicemap",
           "render_views",
           "render_batch", "render_batch_workspace", "render_batch_static", "batch_samples_evaluated", "BatchTuning",
           "image_entropy",
           "find_container", "mask_container", "Slicemap", "AtlasTexture", "View", "default_tiles",
           "atlas_bytes", "version", "MctpError"]

_DTYPES = {torch.uint8: (_lib.MCTP_U8, 1), torch.uint16: (_lib.MCTP_U16, 2), torch.int16: (_lib.MCTP_U16, 2)}
_MODES = {"otsu": _lib.MCTP_THR_OTSU, "its": _lib.MCTP_THR_ITS, "topslab": _lib.MCTP_THR_TOPSLAB,
          "explicit": _lib.MCTP_THR_EXPLICIT}


def _stream(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _cuda(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    return t


def _out(t: torch.Tensor, name: str, dtype: torch.dtype, numel: int, device) -> torch.Tensor:
    """Check a caller-supplied output buffer before its pointer reaches the
    library, which cannot see its size: a contiguous CUDA tensor of `dtype`
    with at least `numel` elements on `device`."""
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, {numel} needed")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if device is not None and t.device != torch.device(device):
        raise ValueError(f"{name} is on {t.device}, the inputs on {device}")
    return t


def volume_desc(vol: torch.Tensor, bits: int) -> _lib.VolumeDesc:
    if vol.dim() != 3 or vol.dtype not in _DTYPES:
        raise ValueError("volume must be a 3-D uint8/uint16 tensor [nz][ny][nx]")
    nz, ny, nx = vol.shape
    return _lib.VolumeDesc(nx, ny, nz, _DTYPES[vol.dtype][0], bits)


def version() -> int:
    return _lib.load().mctp_version()


def default_tiles(mz: int) -> tuple[int, int]:
    tx, ty = _lib.C_I32(), _lib.C_I32()
    _lib.check(_lib.load().mctp_default_tiles(mz, ctypes.byref(tx), ctypes.byref(ty)), "mctp_default_tiles")
    return tx.value, ty.value


def atlas_bytes(mx: int, my: int, tiles_x: int, tiles_y: int, dtype) -> int:
    return _lib.load().mctp_atlas_bytes(mx, my, tiles_x, tiles_y, _DTYPES[dtype][0])


def build_histogram(vol: torch.Tensor, bits: int, nbins: int, z0: int = 0, z1: int | None = None,
                    hist: torch.Tensor | None = None, overflow: torch.Tensor | None = None, stream=None):
    """Histogram of slices [z0, z1) -> (hist uint64[nbins], overflow uint64[1]) on the device."""
    _cuda(vol, "vol")
    d = volume_desc(vol, bits)
    z1 = vol.shape[0] if z1 is None else z1
    if hist is None:
        hist = torch.empty(nbins, dtype=torch.uint64, device=vol.device)
    if overflow is None:
        overflow = torch.empty(1, dtype=torch.uint64, device=vol.device)
    _out(hist, "hist", torch.uint64, nbins, vol.device)
    _out(overflow, "overflow", torch.uint64, 1, vol.device)
    _lib.check(_lib.load().mctp_build_histogram(_ptr(vol), ctypes.byref(d), z0, z1, nbins, _ptr(hist),
                                                _ptr(overflow), _stream(stream)), "mctp_build_histogram")
    return hist, overflow


def _volume_arrays(vols, bits):
    for v in vols:
        _cuda(v, "vol")
    n = len(vols)
    return (ctypes.c_void_p * max(n, 1))(*[v.data_ptr() for v in vols]), \
        (_lib.VolumeDesc * max(n, 1))(*[volume_desc(v, bits) for v in vols])


def build_histogram_batch(vols: list[torch.Tensor], bits: int, nbins: int, hist: torch.Tensor | None = None,
                          overflow: torch.Tensor | None = None, stream=None):
    """Whole-volume histograms of every volume in vols (one dtype) in one
    launch -> (hist uint64[count, nbins], overflow uint64[count, 1])."""
    if not vols:
        raise ValueError("no volumes")
    dev = vols[0].device
    ptrs, descs = _volume_arrays(vols, bits)
    n = len(vols)
    if hist is None:
        hist = torch.empty((n, nbins), dtype=torch.uint64, device=dev)
    if overflow is None:
        overflow = torch.empty((n, 1), dtype=torch.uint64, device=dev)
    _out(hist, "hist", torch.uint64, n * nbins, dev)
    _out(overflow, "overflow", torch.uint64, n, dev)
    _lib.check(_lib.load().mctp_build_histogram_batch(ptrs, descs, n, nbins, _ptr(hist), _ptr(overflow),
                                                      _stream(stream)), "mctp_build_histogram_batch")
    return hist, overflow


def select_threshold(hist: torch.Tensor | None, nbins: int | None = None, mode: str = "otsu",
                     explicit_T: int = 0, its_max_iter: int = 256, topslab_kmin: int = 1,
                     keep: torch.Tensor | None = None, result: torch.Tensor | None = None,
                     device=None, stream=None):
    """Keep table from a histogram -> (keep uint8[nbins], result int32[4] = T, iters, converged, 0)."""
    if hist is not None:
        _cuda(hist, "hist")
        nbins = hist.numel() if nbins is None else nbins
        device = hist.device
    if nbins is None:
        raise ValueError("nbins needed without a histogram")
    p = _lib.ThrParams(_MODES[mode], explicit_T, its_max_iter, 0, topslab_kmin)
    if keep is None:
        keep = torch.empty(nbins, dtype=torch.uint8, device=device)
    if result is None:
        result = torch.empty(4, dtype=torch.int32, device=device)
    _out(keep, "keep", torch.uint8, nbins, device)
    _out(result, "result", torch.int32, 4, device)
    _lib.check(_lib.load().mctp_select_threshold(_ptr(hist), nbins, ctypes.byref(p), _ptr(keep), _ptr(result),
                                                 _stream(stream)), "mctp_select_threshold")
    return keep, result


def select_threshold_batch(hist: torch.Tensor, mode: str = "otsu", explicit_T: int = 0, its_max_iter: int = 256,
                           topslab_kmin: int = 1, keep: torch.Tensor | None = None,
                           result: torch.Tensor | None = None, stream=None):
    """Keep tables of the rows of hist [count, nbins] in one launch ->
    (keep uint8[count, nbins], result int32[count, 4]); row i as select_threshold(hist[i])."""
    _cuda(hist, "hist")
    if hist.dim() != 2 or hist.dtype != torch.uint64:
        raise ValueError("hist must be uint64 [count, nbins]")
    count, nbins = hist.shape
    p = _lib.ThrParams(_MODES[mode], explicit_T, its_max_iter, 0, topslab_kmin)
    if keep is None:
        keep = torch.empty((count, nbins), dtype=torch.uint8, device=hist.device)
    if result is None:
        result = torch.empty((count, 4), dtype=torch.int32, device=hist.device)
    _out(keep, "keep", torch.uint8, count * nbins, hist.device)
    _out(result, "result", torch.int32, count * 4, hist.device)
    _lib.check(_lib.load().mctp_select_threshold_batch(_ptr(hist), count, nbins, ctypes.byref(p), _ptr(keep),
                                                       _ptr(result), _stream(stream)), "mctp_select_threshold_batch")
    return keep, result


def filter_threshold(vol: torch.Tensor, bits: int, keep: torch.Tensor, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
    """Keep/discard every voxel (out may be vol for in place)."""
    _cuda(vol, "vol")
    _cuda(keep, "keep")
    d = volume_desc(vol, bits)
    if out is None:
        out = torch.empty_like(vol)
    _out(out, "out", vol.dtype, vol.numel(), vol.device)
    _lib.check(_lib.load().mctp_filter_threshold(_ptr(vol), ctypes.byref(d), _ptr(keep), keep.numel(), _ptr(out),
                                                 _stream(stream)), "mctp_filter_threshold")
    return out


@dataclass
class Slicemap:
    """Device atlases of a multi-resolution slicemap plus their geometry."""
    src_dims: tuple[int, int, int]
    dims: list[tuple[int, int, int]]
    tiles: list[tuple[int, int]]
    atlases: list[torch.Tensor]
    bits: int
    dtype: torch.dtype
    maxgrids: list[torch.Tensor] | None = None
    textures: list["AtlasTexture | None"] | None = None  # per level; see make_textures

    @classmethod
    def allocate(cls, src_dims, level0_dims, nlevels: int, dtype: torch.dtype, bits: int, device="cuda",
                 maxgrid: bool = True):
        dims = [tuple(level0_dims)]
        for _ in range(1, nlevels):
            dims.append(tuple(v // 2 for v in dims[-1]))
        tiles = [default_tiles(d[2]) for d in dims]
        atlases = [torch.empty((ty * d[1], tx * d[0]), dtype=dtype, device=device)
                   for d, (tx, ty) in zip(dims, tiles)]
        grids = None
        if maxgrid:
            c = _lib.MCTP_MAXGRID_CELL
            grids = [torch.empty((-(-d[2] // c), -(-d[1] // c), -(-d[0] // c)), dtype=torch.uint16, device=device)
                     for d in dims]
        return cls(tuple(src_dims), dims, tiles, atlases, bits, dtype, grids)

    def desc(self) -> _lib.SlicemapDesc:
        s = _lib.SlicemapDesc()
        s.nlevels = len(self.dims)
        s.dtype = _DTYPES[self.dtype][0]
        s.bits = self.bits
        for a in range(3):
            s.src_dims[a] = self.src_dims[a]
        for k, (d, (tx, ty), at) in enumerate(zip(self.dims, self.tiles, self.atlases)):
            _cuda(at, "atlas")
            for a in range(3):
                s.dims[k][a] = d[a]
            s.tiles_x[k] = tx
            s.tiles_y[k] = ty
            s.atlas[k] = at.data_ptr()
            if self.maxgrids is not None and self.maxgrids[k] is not None:
                s.maxgrid[k] = _cuda(self.maxgrids[k], "maxgrid").data_ptr()
            if self.textures is not None and self.textures[k] is not None:
                s.texture[k] = self.textures[k].handle
        return s

    def make_textures(self, levels=None) -> "Slicemap":
        """Give the listed levels (default: all) an atlas texture; the batched
        renderer then gathers corner quads through it.  Call update_textures
        after every build_slicemap."""
        levels = range(len(self.dims)) if levels is None else levels
        if self.textures is None:
            self.textures = [None] * len(self.dims)
        for k in levels:
            if self.textures[k] is None:
                self.textures[k] = AtlasTexture(self, k)
        return self

    def update_textures(self, stream=None) -> None:
        """Copy the atlases into their textures (device to device, on stream)."""
        for t in self.textures or []:
            if t is not None:
                t.update(self, stream)

    def without_maxgrid(self) -> "Slicemap":
        """The same atlases with no occupancy data (renders evaluate every sample)."""
        return Slicemap(self.src_dims, self.dims, self.tiles, self.atlases, self.bits, self.dtype, None,
                        self.textures)

    def without_textures(self) -> "Slicemap":
        """The same atlases and max grids, rendered with loads from the atlases."""
        return Slicemap(self.src_dims, self.dims, self.tiles, self.atlases, self.bits, self.dtype, self.maxgrids)

    @property
    def nbytes(self) -> int:
        return sum(a.numel() * a.element_size() for a in self.atlases)


class AtlasTexture:
    """Level `level` of a slicemap's atlas as a 2D texture (mctp_atlas_texture_*),
    owning a CUDA array of the atlas's size; freed by close() or when collected."""

    def __init__(self, sm: "Slicemap", level: int):
        self.level = level
        self._ptr = ctypes.c_void_p()
        h = ctypes.c_uint64()
        d = sm.desc()
        _lib.check(_lib.load().mctp_atlas_texture_create(ctypes.byref(d), level, ctypes.byref(self._ptr),
                                                          ctypes.byref(h)), "mctp_atlas_texture_create")
        self.handle = h.value

    def update(self, sm: "Slicemap", stream=None) -> None:
        d = sm.desc()
        _lib.check(_lib.load().mctp_atlas_texture_update(self._ptr, ctypes.byref(d), self.level, _stream(stream)),
                   "mctp_atlas_texture_update")

    def close(self) -> None:
        if self._ptr:
            _lib.check(_lib.load().mctp_atlas_texture_destroy(self._ptr), "mctp_atlas_texture_destroy")
            self._ptr = ctypes.c_void_p()
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_slicemap(vol: torch.Tensor, bits: int, sm: Slicemap, keep: torch.Tensor | None = None,
                   stream=None) -> Slicemap:
    """Fill sm's atlases (and max grids) from vol, keep table applied first when given."""
    _cuda(vol, "vol")
    d = volume_desc(vol, bits)
    s = sm.desc()
    nb = keep.numel() if keep is not None else 0
    _lib.check(_lib.load().mctp_build_slicemap(_ptr(vol), ctypes.byref(d), _ptr(keep), nb, ctypes.byref(s),
                                               _stream(stream)), "mctp_build_slicemap")
    return sm


def build_slicemap_batch(vols: list[torch.Tensor], bits: int, sms: list[Slicemap],
                         keep: torch.Tensor | None = None, stream=None) -> list[Slicemap]:
    """build_slicemap for every (vols[i], sms[i]) with keep table keep[i]
    (uint8 [count, nbins], or None); the max grids of all of them are filled
    in one launch."""
    if len(vols) != len(sms):
        raise ValueError("one slicemap per volume")
    if not vols:
        return sms
    ptrs, descs = _volume_arrays(vols, bits)
    n = len(vols)
    smd = (_lib.SlicemapDesc * n)(*[sm.desc() for sm in sms])
    nb = 0
    if keep is not None:
        _cuda(keep, "keep")
        if keep.dim() != 2 or keep.shape[0] < n or keep.dtype != torch.uint8:
            raise ValueError("keep must be uint8 [count, nbins]")
        nb = keep.shape[1]
    _lib.check(_lib.load().mctp_build_slicemap_batch(ptrs, descs, _ptr(keep), nb, smd, n, _stream(stream)),
               "mctp_build_slicemap_batch")
    return sms


def update_textures_batch(sms: list[Slicemap], stream=None) -> None:
    """Slicemap.update_textures for every slicemap in one launch."""
    items = [(t, sm) for sm in sms for t in (sm.textures or []) if t is not None]
    if not items:
        return
    n = len(items)
    tex = (ctypes.c_void_p * n)(*[t._ptr.value for t, _ in items])
    smd = (_lib.SlicemapDesc * n)(*[sm.desc() for _, sm in items])
    levels = (_lib.C_I32 * n)(*[t.level for t, _ in items])
    _lib.check(_lib.load().mctp_atlas_texture_update_batch(tex, smd, levels, n, _stream(stream)),
               "mctp_atlas_texture_update_batch")


@dataclass(frozen=True)
class View:
    azimuth_deg: float
    elevation_deg: float
    width: int
    height: int
    level: int = 0
    step: float = 0.5


def view_array(views) -> ctypes.Array:
    arr = (_lib.ViewDesc * max(1, len(views)))()
    for i, v in enumerate(views):
        arr[i] = _lib.ViewDesc(v.azimuth_deg, v.elevation_deg, v.width, v.height, v.level, v.step)
    return arr


def render_views(sm: Slicemap, views, lut: torch.Tensor, alpha_stop: float = 0.99,
                 out: torch.Tensor | None = None, samples: torch.Tensor | None = None, stream=None):
    """Render views -> (flat float32 RGBA buffer, samples uint64[1]); see images() to split it."""
    _cuda(lut, "lut")
    if lut.dtype != torch.float32 or lut.dim() != 2 or lut.shape[1] != 4:
        raise ValueError("lut must be float32 [n][4]")
    total = sum(v.width * v.height * 4 for v in views)
    dev = lut.device
    if out is None:
        out = torch.empty(max(total, 4), dtype=torch.float32, device=dev)
    if samples is None:
        samples = torch.empty(1, dtype=torch.uint64, device=dev)
    _out(out, "out", torch.float32, total, dev)
    _out(samples, "samples", torch.uint64, 1, dev)
    s = sm.desc()
    arr = view_array(views)
    _lib.check(_lib.load().mctp_render_views(ctypes.byref(s), arr, len(views), _ptr(lut), lut.shape[0],
                                             alpha_stop, _ptr(out), _ptr(samples), _stream(stream)),
               "mctp_render_views")
    return out, samples


def images(flat: torch.Tensor, views) -> list[torch.Tensor]:
    """Split a render_views buffer into [H][W][4] images."""
    out, off = [], 0
    for v in views:
        n = v.width * v.height * 4
        out.append(flat[off:off + n].view(v.height, v.width, 4))
        off += n
    return out


@dataclass(frozen=True)
class BatchTuning:
    """Launch shape of render_batch (speed only; results do not depend on it)."""
    warp_w: int = 8       # a warp covers warp_w x 32/warp_w pixels (4, 8, 16 or 32)
    chunk: int = 2        # warp tiles taken per queue access (1..64)
    ctas_per_sm: int = 0  # cap on resident CTAs per SM (0 = occupancy limit)
    count_evaluated: bool = False  # count evaluated samples (batch_samples_evaluated); a little slower

    def c(self) -> _lib.BatchTuning:
        return _lib.BatchTuning(self.warp_w, self.chunk, self.ctas_per_sm,
                                _lib.MCTP_BATCH_COUNT_EVALUATED if self.count_evaluated else 0)


class _BatchArgs:
    """Host arrays of one batch (slicemap descriptors, views, indices)."""

    def __init__(self, slicemaps, views, view_slicemap, view_lut):
        n = len(views)
        if len(view_slicemap) != n or len(view_lut) != n:
            raise ValueError("views, view_slicemap and view_lut differ in length")
        self.sms = (_lib.SlicemapDesc * max(1, len(slicemaps)))()
        for i, sm in enumerate(slicemaps):
            self.sms[i] = sm.desc()
        self.nsm = len(slicemaps)
        self.views = view_array(views)
        self.vsm = (_lib.C_I32 * max(1, n))(*view_slicemap)
        self.vlut = (_lib.C_I32 * max(1, n))(*view_lut)
        self.n = n


def _luts3(luts: torch.Tensor) -> torch.Tensor:
    _cuda(luts, "luts")
    if luts.dim() == 2:
        luts = luts.unsqueeze(0)
    if luts.dtype != torch.float32 or luts.dim() != 3 or luts.shape[2] != 4:
        raise ValueError("luts must be float32 [nluts][nlut][4] (or [nlut][4])")
    return luts


def render_batch_workspace(slicemaps, views, view_slicemap, view_lut, nluts: int) -> int:
    """Bytes of device workspace render_batch needs for this batch."""
    a = _BatchArgs(slicemaps, views, view_slicemap, view_lut)
    nb = ctypes.c_size_t()
    _lib.check(_lib.load().mctp_render_batch_workspace(a.sms, a.nsm, a.views, a.vsm, a.vlut, a.n, nluts,
                                                       ctypes.byref(nb)), "mctp_render_batch_workspace")
    return nb.value


def render_batch(slicemaps, views, view_slicemap, view_lut, luts: torch.Tensor, alpha_stop: float = 0.99,
                 tuning: BatchTuning | None = None, out: torch.Tensor | None = None,
                 samples: torch.Tensor | None = None, workspace: torch.Tensor | None = None, stream=None):
    """Render view i from slicemaps[view_slicemap[i]] with luts[view_lut[i]], all in one persistent launch.

    Returns (flat float32 RGBA buffer, samples uint64[1], workspace); images() splits the buffer.
    Pass the returned workspace back in to reuse it (e.g. for CUDA-graph capture)."""
    luts = _luts3(luts)
    a = _BatchArgs(slicemaps, views, view_slicemap, view_lut)
    dev = luts.device
    nb = ctypes.c_size_t()
    lib = _lib.load()
    _lib.check(lib.mctp_render_batch_workspace(a.sms, a.nsm, a.views, a.vsm, a.vlut, a.n, luts.shape[0],
                                               ctypes.byref(nb)), "mctp_render_batch_workspace")
    if workspace is None:
        workspace = torch.empty(nb.value, dtype=torch.uint8, device=dev)
    _out(workspace, "workspace", torch.uint8, nb.value, dev)
    total = sum(v.width * v.height * 4 for v in views)
    if out is None:
        out = torch.empty(max(total, 4), dtype=torch.float32, device=dev)
    if samples is None:
        samples = torch.empty(1, dtype=torch.uint64, device=dev)
    _out(out, "out", torch.float32, total, dev)
    _out(samples, "samples", torch.uint64, 1, dev)
    t = (tuning or BatchTuning()).c()
    _lib.check(lib.mctp_render_batch(a.sms, a.nsm, a.views, a.vsm, a.vlut, a.n, _ptr(luts), luts.shape[0],
                                     luts.shape[1], alpha_stop, ctypes.byref(t), _ptr(out), _ptr(samples),
                                     _ptr(workspace), workspace.numel(), _stream(stream)), "mctp_render_batch")
    return out, samples, workspace


def batch_samples_evaluated(workspace: torch.Tensor) -> int:
    """Samples the last render_batch call on this workspace evaluated (taken
    minus those skipped as empty) when it ran with count_evaluated, else 0;
    waits for all work on the workspace's device first."""
    torch.cuda.synchronize(workspace.device)
    return int(workspace[8:16].view(torch.int64).item())


def render_batch_static(slicemaps, views, view_slicemap, view_lut, luts: torch.Tensor, alpha_stop: float = 0.99,
                        tuning: BatchTuning | None = None, out: torch.Tensor | None = None,
                        samples: torch.Tensor | None = None, stream=None):
    """render_batch with the library's fixed device scratch instead of a workspace (no allocation in the call;
    calls that can overlap on the device must not be issued concurrently).  Returns (flat RGBA, samples)."""
    luts = _luts3(luts)
    a = _BatchArgs(slicemaps, views, view_slicemap, view_lut)
    dev = luts.device
    total = sum(v.width * v.height * 4 for v in views)
    if out is None:
        out = torch.empty(max(total, 4), dtype=torch.float32, device=dev)
    if samples is None:
        samples = torch.empty(1, dtype=torch.uint64, device=dev)
    _out(out, "out", torch.float32, total, dev)
    _out(samples, "samples", torch.uint64, 1, dev)
    t = (tuning or BatchTuning()).c()
    _lib.check(_lib.load().mctp_render_batch_static(a.sms, a.nsm, a.views, a.vsm, a.vlut, a.n, _ptr(luts),
                                                    luts.shape[0], luts.shape[1], alpha_stop, ctypes.byref(t),
                                                    _ptr(out), _ptr(samples), _stream(stream)),
               "mctp_render_batch_static")
    return out, samples


def image_entropy(flat: torch.Tensor, views, hist: torch.Tensor | None = None, entropy: torch.Tensor | None = None,
                  best: torch.Tensor | None = None, stream=None):
    """Eq. 2 per view of a render_views buffer -> (hist uint64[V][256], H float64[V], best int32[1])."""
    _cuda(flat, "images")
    dev = flat.device
    n = len(views)
    _out(flat, "images", torch.float32, sum(v.width * v.height * 4 for v in views), dev)
    if hist is None:
        hist = torch.empty((max(n, 1), 256), dtype=torch.uint64, device=dev)
    if entropy is None:
        entropy = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
    if best is None:
        best = torch.empty(1, dtype=torch.int32, device=dev)
    _out(hist, "hist", torch.uint64, n * 256, dev)
    _out(entropy, "entropy", torch.float64, n, dev)
    _out(best, "best", torch.int32, 1, dev)
    _lib.check(_lib.load().mctp_image_entropy(_ptr(flat), view_array(views), n, _ptr(hist), _ptr(entropy), _ptr(best),
                                              _stream(stream)), "mctp_image_entropy")
    return hist, entropy, best


def find_container(vol: torch.Tensor, bits: int, z: int = 0, thr: int = 40, rmin: int | None = None,
                   rmax: int | None = None, cell: int | None = None, stream=None):
    """Container circle on slice z -> dict(circle int32[3], fit float64[3], acc, rhist) on the device."""
    _cuda(vol, "vol")
    d = volume_desc(vol, bits)
    nz, ny, nx = vol.shape
    n = min(nx, ny)
    rmin = n // 8 if rmin is None else rmin
    rmax = n // 2 if rmax is None else rmax
    cell = max(4, n // 32) if cell is None else cell
    dev = vol.device
    lib = _lib.load()
    acc = torch.empty((-(-ny // cell), -(-nx // cell)), dtype=torch.int32, device=dev)
    rhist = torch.empty(rmax + 1, dtype=torch.int32, device=dev)
    nb = lib.mctp_container_workspace(nx, ny)
    ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=dev)
    circle = torch.empty(3, dtype=torch.int32, device=dev)
    fit = torch.empty(3, dtype=torch.float64, device=dev)
    _lib.check(lib.mctp_find_container(_ptr(vol), ctypes.byref(d), z, thr, rmin, rmax, cell, _ptr(acc), _ptr(rhist),
                                       _ptr(ws), ws.numel(), _ptr(circle), _ptr(fit), _stream(stream)),
               "mctp_find_container")
    return dict(circle=circle, fit=fit, acc=acc, rhist=rhist)


def mask_container(vol: torch.Tensor, bits: int, circle: torch.Tensor, margin: int = 2,
                   out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """vol with everything outside the container circle zeroed (out may be vol)."""
    _cuda(vol, "vol")
    d = volume_desc(vol, bits)
    if out is None:
        out = torch.empty_like(vol)
    _out(out, "out", vol.dtype, vol.numel(), vol.device)
    _lib.check(_lib.load().mctp_mask_container(_ptr(vol), ctypes.byref(d), _ptr(circle), margin, _ptr(out),
                                               _stream(stream)), "mctp_mask_container")
    return out
