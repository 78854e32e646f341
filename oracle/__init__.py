"""CPU oracle for the micro-CT preview hot path (TEST INFRASTRUCTURE).

Plain, slow reference written from the paper (arXiv 2311.15038) in C
(``oracle.c``), FP64 wherever the method is floating point.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may
import this package; the CUDA library never does, and the two share no code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None

C_I64 = ctypes.c_int64
C_I32 = ctypes.c_int32
C_VP = ctypes.c_void_p


def build() -> None:
    """Compile oracle.c (gcc, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           os.path.join(_HERE, "oracle.c"), "-o", _SO, "-lm"])


class View(ctypes.Structure):
    _fields_ = [("az_deg", ctypes.c_float), ("el_deg", ctypes.c_float),
                ("width", C_I32), ("height", C_I32), ("step", ctypes.c_float)]


def _L():
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            build()
        lib = ctypes.CDLL(_SO)
        lib.orc_histogram.argtypes = [C_VP, ctypes.c_int, C_I64, C_I64, C_I64, ctypes.c_int,
                                      C_I64, C_I64, ctypes.c_int, C_VP, C_VP]
        lib.orc_otsu.argtypes = [C_VP, ctypes.c_int, C_VP, C_VP]
        lib.orc_its.argtypes = [C_VP, ctypes.c_int, ctypes.c_int, C_VP, C_VP, C_VP, C_VP]
        lib.orc_keep_threshold.argtypes = [ctypes.c_int, C_I32, C_VP]
        lib.orc_keep_topslab.argtypes = [C_VP, ctypes.c_int, ctypes.c_uint64, C_VP]
        lib.orc_filter.argtypes = [C_VP, ctypes.c_int, C_I64, ctypes.c_int, C_VP, ctypes.c_int, C_VP]
        lib.orc_downsample.argtypes = [C_VP, ctypes.c_int, C_I64, C_I64, C_I64, ctypes.c_int, C_VP,
                                       ctypes.c_int, C_I64, C_I64, C_I64, C_VP]
        lib.orc_atlas_pack.argtypes = [C_VP, ctypes.c_int, C_I64, C_I64, C_I64, C_I64, C_I64, C_VP]
        lib.orc_render.argtypes = [C_VP, ctypes.c_int, ctypes.c_int, C_I64, C_I64, C_I64,
                                   C_I64, C_I64, C_I64, C_VP, ctypes.c_int, ctypes.c_float,
                                   ctypes.c_double, ctypes.POINTER(View), C_VP, C_I64,
                                   C_VP, C_VP, C_VP, C_VP]
        lib.orc_ray_params.argtypes = [C_I64] * 6 + [ctypes.POINTER(View), C_I64, C_I64,
                                                     C_VP, C_VP, C_VP, C_VP, C_VP]
        lib.orc_entropy.argtypes = [C_VP, ctypes.c_int, C_VP]
        lib.orc_maxgrid.argtypes = [C_VP, ctypes.c_int, C_I64, C_I64, C_I64, ctypes.c_int, C_VP]
        lib.orc_image_histogram.argtypes = [C_VP, C_I64, C_VP]
        lib.orc_hough_circle.argtypes = [C_VP, ctypes.c_int, C_I64, C_I64, C_I64, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, C_VP, C_VP, C_VP, C_VP, C_VP, C_VP]
        lib.orc_mask_circle.argtypes = [C_VP, ctypes.c_int, C_I64, C_I64, C_I64, C_I32, C_I32, C_I32, C_VP]
        lib.orc_render_dense.argtypes = [C_VP] + [C_I64] * 6 + [C_VP, ctypes.c_int, ctypes.c_double,
                                                               ctypes.POINTER(View), C_VP, C_I64, C_VP, C_VP]
        lib.orc_render_dense_band.argtypes = [C_VP] + [C_I64] * 6 + [C_VP, ctypes.c_int, ctypes.c_double,
                                                                    ctypes.c_double, ctypes.POINTER(View), C_VP,
                                                                    C_I64, C_VP, C_VP, C_VP, C_VP]
        lib.orc_render_dense_grad.argtypes = [C_VP] + [C_I64] * 6 + [C_VP, ctypes.c_int, ctypes.c_double,
                                                                    ctypes.POINTER(View), C_VP, C_VP, C_VP,
                                                                    C_VP, C_VP]
        for f in ("orc_histogram", "orc_otsu", "orc_its", "orc_keep_threshold", "orc_keep_topslab",
                  "orc_filter", "orc_downsample", "orc_atlas_pack", "orc_render", "orc_ray_params",
                  "orc_entropy", "orc_maxgrid", "orc_render_dense", "orc_render_dense_band", "orc_render_dense_grad",
                  "orc_image_histogram", "orc_hough_circle", "orc_mask_circle"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C_VP)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments ({rc})")


def _vol(vol: np.ndarray) -> np.ndarray:
    vol = np.ascontiguousarray(vol)
    if vol.dtype not in (np.uint8, np.uint16) or vol.ndim != 3:
        raise ValueError("volume must be a 3-D uint8/uint16 array [z][y][x]")
    return vol


def histogram(vol: np.ndarray, bits: int, nbins: int, z0: int = 0, z1: int | None = None):
    vol = _vol(vol)
    nz, ny, nx = vol.shape
    z1 = nz if z1 is None else z1
    hist = np.zeros(nbins, dtype=np.uint64)
    ov = np.zeros(1, dtype=np.uint64)
    _check(_L().orc_histogram(_p(vol), vol.itemsize, nx, ny, nz, bits, z0, z1, nbins,
                              _p(hist), _p(ov)), "histogram")
    return hist, int(ov[0])


def otsu(hist: np.ndarray):
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    T = np.zeros(1, dtype=np.int32)
    s = np.zeros(1, dtype=np.float64)
    _check(_L().orc_otsu(_p(h), h.size, _p(T), _p(s)), "otsu")
    return int(T[0]), float(s[0])


def its(hist: np.ndarray, max_iter: int = 256):
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    T = np.zeros(1, dtype=np.int32)
    it = np.zeros(1, dtype=np.int32)
    cv = np.zeros(1, dtype=np.int32)
    tr = np.zeros(1, dtype=np.float64)
    _check(_L().orc_its(_p(h), h.size, max_iter, _p(T), _p(it), _p(cv), _p(tr)), "its")
    return int(T[0]), int(it[0]), bool(cv[0]), float(tr[0])


def keep_threshold(nbins: int, T: int) -> np.ndarray:
    k = np.zeros(nbins, dtype=np.uint8)
    _check(_L().orc_keep_threshold(nbins, T, _p(k)), "keep_threshold")
    return k


def keep_topslab(hist_top: np.ndarray, kmin: int = 1) -> np.ndarray:
    h = np.ascontiguousarray(hist_top, dtype=np.uint64)
    k = np.zeros(h.size, dtype=np.uint8)
    _check(_L().orc_keep_topslab(_p(h), h.size, kmin, _p(k)), "keep_topslab")
    return k


def filter_volume(vol: np.ndarray, bits: int, keep: np.ndarray) -> np.ndarray:
    vol = _vol(vol)
    keep = np.ascontiguousarray(keep, dtype=np.uint8)
    out = np.empty_like(vol)
    _check(_L().orc_filter(_p(vol), vol.itemsize, vol.size, bits, _p(keep), keep.size, _p(out)),
           "filter")
    return out


def downsample(vol: np.ndarray, bits: int, dims, keep: np.ndarray | None = None) -> np.ndarray:
    """Level of dims (mx, my, mz) from vol [z][y][x]; returns [mz][my][mx]."""
    vol = _vol(vol)
    nz, ny, nx = vol.shape
    mx, my, mz = dims
    out = np.zeros((mz, my, mx), dtype=vol.dtype)
    kp = None
    nb = 0
    if keep is not None:
        keep = np.ascontiguousarray(keep, dtype=np.uint8)
        kp = _p(keep)
        nb = keep.size
    _check(_L().orc_downsample(_p(vol), vol.itemsize, nx, ny, nz, bits, kp, nb, mx, my, mz,
                               _p(out)), "downsample")
    return out


def default_tiles(mz: int):
    """Atlas grid for mz slices: tiles_x = 2^ceil(log2 sqrt(mz)), tiles_y = ceil(mz / tiles_x)."""
    tx = 1
    while tx * tx < mz:
        tx *= 2
    return tx, -(-mz // tx)


def atlas_pack(level: np.ndarray, tiles_x: int, tiles_y: int) -> np.ndarray:
    level = _vol(level)
    mz, my, mx = level.shape
    atlas = np.zeros((tiles_y * my, tiles_x * mx), dtype=level.dtype)
    _check(_L().orc_atlas_pack(_p(level), level.itemsize, mx, my, mz, tiles_x, tiles_y,
                               _p(atlas)), "atlas_pack")
    return atlas


def slicemap(vol: np.ndarray, bits: int, level_dims, keep: np.ndarray | None = None):
    """Levels of a slicemap: level 0 from the source, level k from level k-1."""
    levels = [downsample(vol, bits, level_dims[0], keep)]
    for d in level_dims[1:]:
        levels.append(downsample(levels[-1], bits, d, None))
    return levels


def render(level: np.ndarray, bits: int, src_dims, lut: np.ndarray, az: float, el: float,
           width: int, height: int, step: float = 0.5, alpha_stop: float = 0.99,
           eps: float = 1e-4, pixels: np.ndarray | None = None):
    """FP64 render of a level; returns dict(rgba, lo, hi, nsamp) over all or listed pixels."""
    level = _vol(level)
    mz, my, mx = level.shape
    nx, ny, nz = src_dims
    lut = np.ascontiguousarray(lut, dtype=np.float32)
    v = View(az, el, width, height, step)
    if pixels is None:
        npix = width * height
        pp = None
    else:
        pixels = np.ascontiguousarray(pixels, dtype=np.int64)
        npix = pixels.size
        pp = _p(pixels)
    rgba = np.zeros((npix, 4), dtype=np.float64)
    lo = np.zeros((npix, 4), dtype=np.float64)
    hi = np.zeros((npix, 4), dtype=np.float64)
    ns = np.zeros((npix, 3), dtype=np.uint64)
    _check(_L().orc_render(_p(level), level.itemsize, bits, mx, my, mz, nx, ny, nz, _p(lut),
                           lut.shape[0], alpha_stop, eps, ctypes.byref(v), pp,
                           npix if pixels is not None else -1, _p(rgba), _p(lo), _p(hi), _p(ns)),
           "render")
    if pixels is None:
        shape = (height, width, 4)
        return dict(rgba=rgba.reshape(shape), lo=lo.reshape(shape), hi=hi.reshape(shape),
                    nsamp=ns.reshape(height, width, 3))
    return dict(rgba=rgba, lo=lo, hi=hi, nsamp=ns)


def ray_params(level_dims, src_dims, az, el, width, height, step, i, j):
    mx, my, mz = level_dims
    nx, ny, nz = src_dims
    v = View(az, el, width, height, step)
    o = np.zeros(3, np.float32)
    d = np.zeros(3, np.float32)
    tn = np.zeros(1, np.float32)
    dl = np.zeros(1, np.float32)
    n = np.zeros(1, np.int64)
    _check(_L().orc_ray_params(mx, my, mz, nx, ny, nz, ctypes.byref(v), i, j, _p(o), _p(d),
                               _p(tn), _p(dl), _p(n)), "ray_params")
    return o, d, float(tn[0]), float(dl[0]), int(n[0])


def entropy(counts: np.ndarray) -> float:
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    H = np.zeros(1, np.float64)
    _check(_L().orc_entropy(_p(c), c.size, _p(H)), "entropy")
    return float(H[0])


def maxgrid(level: np.ndarray, cell: int = 8) -> np.ndarray:
    """Per-cell maximum over [cell*c, cell*c + cell] (clamped) of a level [z][y][x]."""
    level = _vol(level)
    mz, my, mx = level.shape
    g = np.zeros((-(-mz // cell), -(-my // cell), -(-mx // cell)), np.uint16)
    _check(_L().orc_maxgrid(_p(level), level.itemsize, mx, my, mz, cell, _p(g)), "maxgrid")
    return g


def render_dense(vol: np.ndarray, src_dims, lut: np.ndarray, az: float, el: float, width: int, height: int,
                 step: float = 0.5, alpha_stop: float = 0.99, pixels: np.ndarray | None = None):
    """FP64 render of a dense intensity volume [z][y][x] -> (rgba [H][W][4] or [n][4], samples)."""
    vol = np.ascontiguousarray(vol, dtype=np.float64)
    mz, my, mx = vol.shape
    nx, ny, nz = src_dims
    lut = np.ascontiguousarray(lut, dtype=np.float64)
    v = View(az, el, width, height, step)
    if pixels is None:
        npix, pp = width * height, None
    else:
        pixels = np.ascontiguousarray(pixels, dtype=np.int64)
        npix, pp = pixels.size, _p(pixels)
    rgba = np.zeros((npix, 4), np.float64)
    ns = np.zeros(npix, np.uint64)
    _check(_L().orc_render_dense(_p(vol), mx, my, mz, nx, ny, nz, _p(lut), lut.shape[0], alpha_stop,
                                 ctypes.byref(v), pp, npix, _p(rgba), _p(ns)), "render_dense")
    if pixels is None:
        return rgba.reshape(height, width, 4), ns.reshape(height, width)
    return rgba, ns


def render_dense_band(vol: np.ndarray, src_dims, lut: np.ndarray, az: float, el: float, width: int,
                      height: int, step: float = 0.5, alpha_stop: float = 0.99, eps: float = 1e-4):
    """FP64 dense render with the early-exit band: dict(rgba, lo, hi [H][W][4], nsamp [H][W][3]);
    lo / hi stop at alpha_stop -/+ eps."""
    vol = np.ascontiguousarray(vol, dtype=np.float64)
    mz, my, mx = vol.shape
    nx, ny, nz = src_dims
    lut = np.ascontiguousarray(lut, dtype=np.float64)
    v = View(az, el, width, height, step)
    npix = width * height
    rgba, lo, hi = (np.zeros((npix, 4), np.float64) for _ in range(3))
    ns = np.zeros((npix, 3), np.uint64)
    _check(_L().orc_render_dense_band(_p(vol), mx, my, mz, nx, ny, nz, _p(lut), lut.shape[0], alpha_stop, eps,
                                      ctypes.byref(v), None, npix, _p(rgba), _p(lo), _p(hi), _p(ns)),
           "render_dense_band")
    shape = (height, width, 4)
    return dict(rgba=rgba.reshape(shape), lo=lo.reshape(shape), hi=hi.reshape(shape),
                nsamp=ns.reshape(height, width, 3))


def render_dense_grad(vol: np.ndarray, src_dims, lut: np.ndarray, az: float, el: float, width: int,
                      height: int, g_rgba: np.ndarray, step: float = 0.5, alpha_stop: float = 0.99,
                      magnitudes: bool = False):
    """Gradient of sum(g_rgba * render_dense(...)) -> (g_vol like vol, g_lut like lut), FP64.
    With magnitudes=True also the per-element sums of |terms| -> (g_vol, g_lut, mag_vol, mag_lut)."""
    vol = np.ascontiguousarray(vol, dtype=np.float64)
    mz, my, mx = vol.shape
    nx, ny, nz = src_dims
    lut = np.ascontiguousarray(lut, dtype=np.float64)
    g = np.ascontiguousarray(g_rgba, dtype=np.float64).reshape(height * width * 4)
    gv = np.zeros_like(vol)
    gl = np.zeros_like(lut)
    mv = np.zeros_like(vol) if magnitudes else None
    ml = np.zeros_like(lut) if magnitudes else None
    v = View(az, el, width, height, step)
    _check(_L().orc_render_dense_grad(_p(vol), mx, my, mz, nx, ny, nz, _p(lut), lut.shape[0], alpha_stop,
                                      ctypes.byref(v), _p(g), _p(gv), _p(gl),
                                      _p(mv) if magnitudes else None, _p(ml) if magnitudes else None),
           "render_dense_grad")
    return (gv, gl, mv, ml) if magnitudes else (gv, gl)


def image_histogram(rgba: np.ndarray) -> np.ndarray:
    """256-bin grey-level histogram of a float32 RGBA image (any leading shape)."""
    a = np.ascontiguousarray(rgba, dtype=np.float32).reshape(-1, 4)
    h = np.zeros(256, np.uint64)
    _check(_L().orc_image_histogram(_p(a), a.shape[0], _p(h)), "image_histogram")
    return h


def image_entropy(rgba: np.ndarray) -> float:
    """Eq. 2 over the image's grey-level histogram."""
    return entropy(image_histogram(rgba))


def hough_circle(slice2d: np.ndarray, thr: int, rmin: int, rmax: int, cell: int):
    """Container circle of a slice [y][x] -> dict(cx, cy, r, fit (cx, cy, r floats), acc, rhist)."""
    sl = _vol(slice2d[None])[0]
    ny, nx = sl.shape
    acc = np.zeros((-(-ny // cell), -(-nx // cell)), np.uint32)
    rh = np.zeros(rmax + 1, np.uint32)
    fit = np.zeros(3, np.float64)
    out = np.zeros(3, np.int32)
    _check(_L().orc_hough_circle(_p(sl), sl.itemsize, nx, ny, thr, rmin, rmax, cell, _p(acc), _p(rh), _p(fit),
                                 _p(out[0:1]), _p(out[1:2]), _p(out[2:3])), "hough_circle")
    return dict(cx=int(out[0]), cy=int(out[1]), r=int(out[2]), fit=fit, acc=acc, rhist=rh)


def mask_circle(vol: np.ndarray, cx: int, cy: int, r_keep: int) -> np.ndarray:
    """vol [z][y][x] with every voxel outside the circle set to 0."""
    vol = _vol(vol)
    nz, ny, nx = vol.shape
    out = np.empty_like(vol)
    _check(_L().orc_mask_circle(_p(vol), vol.itemsize, nx, ny, nz, cx, cy, r_keep, _p(out)), "mask_circle")
    return out
