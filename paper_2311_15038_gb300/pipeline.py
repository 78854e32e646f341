"""The preview hot path as one reusable object: histogram -> threshold keep
table -> fused filter + slicemap -> rendered views -> the most informative
view (Eq. 2), all enqueued on one CUDA stream with outputs allocated once
(arXiv 2311.15038, Table I pipelines: thresholding, slicemap conversion,
server-side rendering with the optimal image snapshot)."""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import (Slicemap, View, build_histogram, build_slicemap, find_container, image_entropy, mask_container,
               render_views, select_threshold)


@dataclass
class PreviewConfig:
    src_dims: tuple[int, int, int]          # nx, ny, nz
    bits: int
    nbins: int
    level0: tuple[int, int, int]
    nlevels: int
    views: list[View]
    mode: str = "otsu"                      # otsu | its | topslab | explicit | none
    topslab: int = 3                        # slices of the top slab (topslab mode)
    alpha_stop: float = 0.99
    explicit_T: int = 0
    container: bool = False                 # remove the sample container first (Hough circle on slice 0)
    container_thr: int = 40                 # edge threshold in 8-bit grey units
    container_margin: int = 2               # voxels kept inside the found inner wall


def turntable(n: int, size: int, level: int = 0, step: float = 0.5, elevation: float = 0.0,
              az_step: float | None = None) -> list[View]:
    """n views around the z axis: azimuth = k * az_step (default 360/n degrees)."""
    da = 360.0 / n if az_step is None else az_step
    return [View(da * k, elevation, size, size, level, step) for k in range(n)]


class PreviewPipeline:
    def __init__(self, cfg: PreviewConfig, dtype: torch.dtype, device="cuda", stream=None):
        self.cfg = cfg
        self.device = torch.device(device)
        self.stream = stream
        nb = cfg.nbins
        self.hist = torch.empty(nb, dtype=torch.uint64, device=self.device)
        self.overflow = torch.empty(1, dtype=torch.uint64, device=self.device)
        self.keep = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self.result = torch.empty(4, dtype=torch.int32, device=self.device)
        self.sm = Slicemap.allocate(cfg.src_dims, cfg.level0, cfg.nlevels, dtype, cfg.bits, self.device)
        total = sum(v.width * v.height * 4 for v in cfg.views)
        self.images = torch.empty(max(total, 4), dtype=torch.float32, device=self.device)
        self.samples = torch.empty(1, dtype=torch.uint64, device=self.device)
        self.masked = None
        if cfg.container:
            nx, ny, nz = cfg.src_dims
            self.masked = torch.empty((nz, ny, nx), dtype=dtype, device=self.device)
            self.circle = None
        nv = max(len(cfg.views), 1)
        self.image_hist = torch.empty((nv, 256), dtype=torch.uint64, device=self.device)
        self.entropy = torch.empty(nv, dtype=torch.float64, device=self.device)
        self.best = torch.empty(1, dtype=torch.int32, device=self.device)

    def run(self, vol: torch.Tensor, lut: torch.Tensor, timer=None):
        """Enqueue one pass; `timer(name)` (optional) is called between the steps."""
        c = self.cfg
        mark = timer or (lambda name: None)
        keep = None
        if c.container:
            mark("container")
            thr = c.container_thr << (c.bits - 8) if c.bits > 8 else c.container_thr
            self.circle = find_container(vol, c.bits, 0, thr, stream=self.stream)["circle"]
            vol = mask_container(vol, c.bits, self.circle, c.container_margin, self.masked, self.stream)
        mark("histogram")
        if c.mode == "topslab":
            build_histogram(vol, c.bits, c.nbins, 0, c.topslab, self.hist, self.overflow, self.stream)
        elif c.mode != "none":
            build_histogram(vol, c.bits, c.nbins, 0, None, self.hist, self.overflow, self.stream)
        mark("threshold")
        if c.mode != "none":
            select_threshold(self.hist, c.nbins, c.mode, c.explicit_T, keep=self.keep, result=self.result,
                             stream=self.stream)
            keep = self.keep
        mark("slicemap")
        build_slicemap(vol, c.bits, self.sm, keep, self.stream)
        mark("render")
        render_views(self.sm, c.views, lut, c.alpha_stop, self.images, self.samples, self.stream)
        mark("entropy")
        image_entropy(self.images, c.views, self.image_hist, self.entropy, self.best, self.stream)
        mark("end")
        return self.images, self.samples
