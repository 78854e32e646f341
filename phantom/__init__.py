"""Seeded synthetic micro-CT phantoms and transfer functions (input generators).

This module writes inputs only; it holds none of the preview method's
arithmetic, so both the CUDA library's tests and the CPU oracle may consume
what it writes.  The volume model is described in ``phantom.h``; a CPU writer
(any sub-box) and a GPU writer (whole volume) produce identical bytes.

Workloads (shaped like the paper's scans, Table II: 8-bit, ~2k x 2k slices,
an object low in the container, background in the top slices, Sec. III-D):

* ``small``  u8 256^3, seed 1001, 12 ellipsoids
* ``full``   u16 12-bit 2016 x 2016 x 1800, seed 1002, 12 ellipsoids and 300
  appendage cylinders
* ``batch``  64 u8 volumes, each axis drawn from U{384..1024}, seed 3000 + j
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_CPU_SO = os.path.join(_BUILD, "libphantom_cpu.so")
_GPU_SO = os.path.join(_BUILD, "libphantom_gpu.so")

_cpu_lib = None
_gpu_lib = None


def build(gpu: bool = True) -> None:
    """Compile the CPU writer with gcc and, if requested, the GPU writer with nvcc."""
    os.makedirs(_BUILD, exist_ok=True)
    subprocess.check_call(
        ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
         os.path.join(_HERE, "phantom_params.c"), os.path.join(_HERE, "phantom_cpu.c"),
         "-o", _CPU_SO, "-lm"])
    if gpu:
        subprocess.check_call(
            ["nvcc", "-O3", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
             "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared",
             os.path.join(_HERE, "phantom_gpu.cu"), "-o", _GPU_SO])


def _cpu():
    global _cpu_lib
    if _cpu_lib is None:
        if not os.path.exists(_CPU_SO):
            build(gpu=False)
        lib = ctypes.CDLL(_CPU_SO)
        lib.ph_make_params.argtypes = [ctypes.c_int64] * 3 + [ctypes.c_int32, ctypes.c_int32,
                                                              ctypes.c_uint64, ctypes.c_int32,
                                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
        lib.ph_make_params.restype = ctypes.c_int
        lib.ph_generate_cpu.argtypes = [ctypes.c_void_p] + [ctypes.c_int64] * 6 + [ctypes.c_void_p]
        lib.ph_generate_cpu.restype = ctypes.c_int
        lib.ph_params_size.restype = ctypes.c_int
        lib.ph_tube_info.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        lib.ph_tube_info.restype = ctypes.c_int
        _cpu_lib = lib
    return _cpu_lib


def _gpu():
    global _gpu_lib
    if _gpu_lib is None:
        if not os.path.exists(_GPU_SO):
            raise RuntimeError("GPU phantom writer not built: call phantom.build()")
        lib = ctypes.CDLL(_GPU_SO)
        lib.ph_generate_gpu.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.ph_generate_gpu.restype = ctypes.c_int
        lib.ph_params_size_gpu.restype = ctypes.c_int
        _gpu_lib = lib
    return _gpu_lib


@dataclass(frozen=True)
class VolumeSpec:
    nx: int
    ny: int
    nz: int
    bits: int = 8
    seed: int = 1001
    n_ell: int = 12
    n_cyl: int = 0
    tube: bool = False      # a cylindrical sample container around the objects

    @property
    def esize(self) -> int:
        return 1 if self.bits <= 8 else 2

    @property
    def np_dtype(self):
        return np.uint8 if self.esize == 1 else np.uint16

    @property
    def nbytes(self) -> int:
        return self.nx * self.ny * self.nz * self.esize

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


SMALL = VolumeSpec(256, 256, 256, bits=8, seed=1001, n_ell=12, n_cyl=0)
FULL = VolumeSpec(2016, 2016, 1800, bits=12, seed=1002, n_ell=12, n_cyl=300)


def batch_specs(count: int = 64, lo: int = 384, hi: int = 1024, seed: int = 3) -> list[VolumeSpec]:
    """Uneven u8 volumes for the batched workload: each axis ~ U{lo..hi}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for j in range(count):
        nx, ny, nz = (int(v) for v in rng.integers(lo, hi + 1, size=3))
        out.append(VolumeSpec(nx, ny, nz, bits=8, seed=1000 * seed + j, n_ell=12, n_cyl=0))
    return out


def serve_specs(count: int = 200, lo: int = 256, hi: int = 1024, seed: int = 5) -> list[VolumeSpec]:
    """Resident u8 cubes for the serving workload: edge ~ U{lo..hi}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for j in range(count):
        e = int(rng.integers(lo, hi + 1))
        out.append(VolumeSpec(e, e, e, bits=8, seed=1000 * seed + j, n_ell=12, n_cyl=0))
    return out


def make_params(spec: VolumeSpec) -> ctypes.Array:
    lib = _cpu()
    buf = (ctypes.c_uint8 * lib.ph_params_size())()
    rc = lib.ph_make_params(spec.nx, spec.ny, spec.nz, spec.bits, spec.esize, spec.seed,
                            spec.n_ell, spec.n_cyl, int(spec.tube), ctypes.addressof(buf))
    if rc != 0:
        raise ValueError(f"ph_make_params failed for {spec}")
    return buf


def tube_geometry(spec: VolumeSpec):
    """(axis x, axis y, inner radius, outer radius) of the container in voxel-index
    coordinates, or None for a volume without one."""
    P = make_params(spec)
    out = np.zeros(4, np.float64)
    if not _cpu().ph_tube_info(ctypes.addressof(P), out.ctypes.data_as(ctypes.c_void_p)):
        return None
    return tuple(float(v) for v in out)


def generate_cpu(spec: VolumeSpec, box=None) -> np.ndarray:
    """Voxels of ``spec`` as a [z][y][x] array; ``box`` = ((x0,x1),(y0,y1),(z0,z1)) or None."""
    P = make_params(spec)
    if box is None:
        box = ((0, spec.nx), (0, spec.ny), (0, spec.nz))
    (x0, x1), (y0, y1), (z0, z1) = box
    out = np.zeros((z1 - z0, y1 - y0, x1 - x0), dtype=spec.np_dtype)
    rc = _cpu().ph_generate_cpu(ctypes.addressof(P), x0, x1, y0, y1, z0, z1,
                                out.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError("ph_generate_cpu failed")
    return out


def generate_gpu(spec: VolumeSpec, out_tensor) -> None:
    """Fill a contiguous CUDA tensor of spec.nbytes bytes with the volume."""
    import torch
    assert out_tensor.is_cuda and out_tensor.is_contiguous()
    assert out_tensor.numel() * out_tensor.element_size() == spec.nbytes
    P = make_params(spec)
    if _gpu().ph_params_size_gpu() != len(P):
        raise RuntimeError("phantom parameter layout differs between the CPU and GPU writers")
    stream = torch.cuda.current_stream(out_tensor.device).cuda_stream
    rc = _gpu().ph_generate_gpu(ctypes.addressof(P), ctypes.c_void_p(out_tensor.data_ptr()),
                                ctypes.c_void_p(stream))
    if rc != 0:
        raise RuntimeError(f"ph_generate_gpu failed ({rc})")


def ramp_lut(n: int = 256) -> np.ndarray:
    """Grey ramp transfer function: entry i = (i/(n-1)) * (1, 1, 1, 1)."""
    v = np.arange(n, dtype=np.float64) / (n - 1)
    return np.repeat(v[:, None], 4, axis=1).astype(np.float32)


def preset_luts(n: int = 256, count: int = 8, seed: int = 5) -> list[np.ndarray]:
    """The grey ramp plus seeded piecewise-linear window / colour ramps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    luts = [ramp_lut(n)]
    x = np.arange(n, dtype=np.float64) / (n - 1)
    for _ in range(count - 1):
        lo = rng.uniform(0.05, 0.4)
        hi = rng.uniform(lo + 0.1, 1.0)
        a = np.clip((x - lo) / (hi - lo), 0.0, 1.0) * rng.uniform(0.3, 1.0)
        rgb = [np.clip(rng.uniform(0.2, 1.0) * x + rng.uniform(0.0, 0.3), 0.0, 1.0) for _ in range(3)]
        luts.append(np.stack(rgb + [a], axis=1).astype(np.float32))
    return luts
