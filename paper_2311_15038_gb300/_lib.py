"""ctypes view of libmctp's C ABI (include/mctp.h).  Marshalling only."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

MCTP_OK = 0
MCTP_EINVAL = -1
MCTP_EUNSUPPORTED = -2
MCTP_ESIZE = -3
MCTP_BATCH_COUNT_EVALUATED = 1
MCTP_ECUDA = -4
MCTP_ECANCELED = -6

MCTP_U8 = 1
MCTP_U16 = 2

MCTP_THR_OTSU = 0
MCTP_THR_ITS = 1
MCTP_THR_TOPSLAB = 2
MCTP_THR_EXPLICIT = 3

MCTP_MAX_LEVELS = 8
MCTP_BATCH_STATIC_SCRATCH = 8 << 20
MCTP_SERVE_BATCHED = 0
MCTP_SERVE_PER_VIEW = 1
MCTP_MAXGRID_CELL = 8

C_I32 = ctypes.c_int32
C_I64 = ctypes.c_int64
C_VP = ctypes.c_void_p


class VolumeDesc(ctypes.Structure):
    _fields_ = [("nx", C_I64), ("ny", C_I64), ("nz", C_I64), ("dtype", C_I32), ("bits", C_I32)]


class ThrParams(ctypes.Structure):
    _fields_ = [("mode", C_I32), ("explicit_T", C_I32), ("its_max_iter", C_I32), ("reserved", C_I32),
                ("topslab_kmin", ctypes.c_uint64)]


class SlicemapDesc(ctypes.Structure):
    _fields_ = [("nlevels", C_I32), ("dtype", C_I32), ("bits", C_I32), ("reserved", C_I32),
                ("src_dims", C_I64 * 3), ("dims", (C_I32 * 3) * MCTP_MAX_LEVELS),
                ("tiles_x", C_I32 * MCTP_MAX_LEVELS), ("tiles_y", C_I32 * MCTP_MAX_LEVELS),
                ("atlas", C_VP * MCTP_MAX_LEVELS), ("maxgrid", C_VP * MCTP_MAX_LEVELS),
                ("texture", ctypes.c_uint64 * MCTP_MAX_LEVELS)]


class ViewDesc(ctypes.Structure):
    _fields_ = [("azimuth_deg", ctypes.c_float), ("elevation_deg", ctypes.c_float),
                ("width", C_I32), ("height", C_I32), ("level", C_I32), ("step", ctypes.c_float)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("warp_w", C_I32), ("chunk", C_I32), ("ctas_per_sm", C_I32), ("flags", C_I32)]


class ServeParams(ctypes.Structure):
    _fields_ = [("mode", C_I32), ("max_batch_views", C_I32), ("max_inflight", C_I32), ("reserved", C_I32),
                ("tuning", BatchTuning)]


class ServeResult(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", C_I32), ("reserved", C_I32), ("image", C_VP),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_launch", ctypes.c_double),
                ("t_done", ctypes.c_double)]


EXPORTS = {
    "mctp_build_histogram": ([C_VP, ctypes.POINTER(VolumeDesc), C_I64, C_I64, C_I32, C_VP, C_VP, C_VP],
                             ctypes.c_int),
    "mctp_build_histogram_batch": ([C_VP, C_VP, C_I32, C_I32, C_VP, C_VP, C_VP], ctypes.c_int),
    "mctp_build_slicemap_batch": ([C_VP, C_VP, C_VP, C_I32, C_VP, C_I32, C_VP], ctypes.c_int),
    "mctp_atlas_texture_update_batch": ([C_VP, C_VP, C_VP, C_I32, C_VP], ctypes.c_int),
    "mctp_select_threshold": ([C_VP, C_I32, ctypes.POINTER(ThrParams), C_VP, C_VP, C_VP], ctypes.c_int),
    "mctp_select_threshold_batch": ([C_VP, C_I32, C_I32, ctypes.POINTER(ThrParams), C_VP, C_VP, C_VP],
                                    ctypes.c_int),
    "mctp_filter_threshold": ([C_VP, ctypes.POINTER(VolumeDesc), C_VP, C_I32, C_VP, C_VP], ctypes.c_int),
    "mctp_build_slicemap": ([C_VP, ctypes.POINTER(VolumeDesc), C_VP, C_I32, ctypes.POINTER(SlicemapDesc), C_VP],
                            ctypes.c_int),
    "mctp_render_views": ([ctypes.POINTER(SlicemapDesc), ctypes.POINTER(ViewDesc), C_I32, C_VP, C_I32,
                           ctypes.c_float, C_VP, C_VP, C_VP], ctypes.c_int),
    "mctp_render_batch_workspace": ([ctypes.POINTER(SlicemapDesc), C_I32, ctypes.POINTER(ViewDesc), C_VP, C_VP,
                                     C_I32, C_I32, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "mctp_render_batch": ([ctypes.POINTER(SlicemapDesc), C_I32, ctypes.POINTER(ViewDesc), C_VP, C_VP, C_I32,
                           C_VP, C_I32, C_I32, ctypes.c_float, ctypes.POINTER(BatchTuning), C_VP, C_VP, C_VP,
                           ctypes.c_size_t, C_VP], ctypes.c_int),
    "mctp_render_batch_static": ([ctypes.POINTER(SlicemapDesc), C_I32, ctypes.POINTER(ViewDesc), C_VP, C_VP, C_I32,
                                  C_VP, C_I32, C_I32, ctypes.c_float, ctypes.POINTER(BatchTuning), C_VP, C_VP, C_VP],
                                 ctypes.c_int),
    "mctp_server_create": ([ctypes.POINTER(SlicemapDesc), C_I32, C_VP, C_I32, C_I32, ctypes.c_float, C_VP,
                            ctypes.c_size_t, ctypes.POINTER(ServeParams), ctypes.POINTER(C_VP)], ctypes.c_int),
    "mctp_server_submit": ([C_VP, ctypes.POINTER(ViewDesc), C_I32, C_I32, ctypes.POINTER(ctypes.c_uint64)],
                           ctypes.c_int),
    "mctp_server_poll": ([C_VP, ctypes.POINTER(ServeResult), C_I32, ctypes.POINTER(C_I32)], ctypes.c_int),
    "mctp_server_release": ([C_VP, ctypes.c_uint64], ctypes.c_int),
    "mctp_server_cancel": ([C_VP, ctypes.c_uint64], ctypes.c_int),
    "mctp_checked_build": ([], ctypes.c_int),
    "mctp_checked_status": ([ctypes.POINTER(ctypes.c_uint32), C_I32], ctypes.c_int),
    "mctp_checked_selftest": ([C_VP], ctypes.c_int),
    "mctp_server_inject_launch_failures": ([C_VP, C_I32], ctypes.c_int),
    "mctp_server_stats": ([C_VP, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                           ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "mctp_server_destroy": ([C_VP], ctypes.c_int),
    "mctp_now": ([], ctypes.c_double),
    "mctp_render_dense": ([C_VP, C_I32, C_I32, C_I32, C_VP, ctypes.POINTER(ViewDesc), C_I32, C_VP, C_I32,
                           ctypes.c_float, C_VP, C_VP, C_VP], ctypes.c_int),
    "mctp_render_dense_backward": ([C_VP, C_I32, C_I32, C_I32, C_VP, ctypes.POINTER(ViewDesc), C_I32, C_VP, C_I32,
                                    ctypes.c_float, C_VP, C_VP, C_VP, C_VP], ctypes.c_int),
    "mctp_l2_loss": ([C_VP, C_VP, C_I64, ctypes.c_float, C_VP, C_VP, C_VP], ctypes.c_int),
    "mctp_adam_step": ([C_VP, C_VP, C_VP, C_VP, C_I64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                        ctypes.c_float, C_I32, ctypes.c_float, ctypes.c_float, C_VP], ctypes.c_int),
    "mctp_atlas_texture_create": ([ctypes.POINTER(SlicemapDesc), C_I32, ctypes.POINTER(C_VP),
                                   ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "mctp_atlas_texture_update": ([C_VP, ctypes.POINTER(SlicemapDesc), C_I32, C_VP], ctypes.c_int),
    "mctp_atlas_texture_destroy": ([C_VP], ctypes.c_int),
    "mctp_image_entropy": ([C_VP, ctypes.POINTER(ViewDesc), C_I32, C_VP, C_VP, C_VP, C_VP], ctypes.c_int),
    "mctp_container_workspace": ([C_I64, C_I64], ctypes.c_size_t),
    "mctp_find_container": ([C_VP, ctypes.POINTER(VolumeDesc), C_I64, C_I64, C_I32, C_I32, C_I32, C_VP, C_VP, C_VP,
                             ctypes.c_size_t, C_VP, C_VP, C_VP], ctypes.c_int),
    "mctp_mask_container": ([C_VP, ctypes.POINTER(VolumeDesc), C_VP, C_I32, C_VP, C_VP], ctypes.c_int),
    "mctp_default_tiles": ([C_I32, ctypes.POINTER(C_I32), ctypes.POINTER(C_I32)], ctypes.c_int),
    "mctp_atlas_bytes": ([C_I32, C_I32, C_I32, C_I32, C_I32], ctypes.c_size_t),
    "mctp_maxgrid_bytes": ([C_I32, C_I32, C_I32], ctypes.c_size_t),
    "mctp_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "mctp_version": ([], ctypes.c_int),
}

_lib = None


class MctpError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = load().mctp_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} ({code})")


def library_path() -> str:
    """The library this process uses: libmctp.so, or with MCTP_LIBRARY=checked
    in the environment the checked build (bounds-tested kernels)."""
    return _build.LIB_CHECKED if os.environ.get("MCTP_LIBRARY") == "checked" else _build.LIB


def load():
    """Load the library.  There is no fallback: a missing library is an error."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libmctp.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (args, res) in EXPORTS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def check(code: int, where: str) -> None:
    if code != MCTP_OK:
        raise MctpError(code, where)
