"""The preview hot path as one reusable object: histogram -> threshold keep
table -> fused filter + slicemap -> rendered views -> the most informative
view (Eq. 2), all enqueued on one CUDA stream with outputs allocated once
(arXiv 2311.15038, Table I pipelines: thresholding, slicemap conversion,
server-side rendering with the optimal image snapshot)."""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import _lib
from ._lib import MctpError
from . import (BatchTuning, Slicemap, View, build_histogram, build_slicemap, find_container, image_entropy,
               mask_container, render_batch, render_batch_workspace, render_views, select_threshold)


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
    renderer: str = "batch"                 # "batch": work-queue renderer (mctp_render_batch); "views": mctp_render_views
    tuning: BatchTuning | None = None       # launch shape of the work-queue renderer (None: 8 x 4 tiles, chunk 1)
    texture: bool = True                    # work-queue renderer: gather corners through atlas textures


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
        if cfg.renderer == "batch":
            # the work-queue renderer: its bitmap and slice tables live in a workspace
            # read through L1, 4 CTAs per SM, one tail; same images as render_views
            self._vsm = [0] * len(cfg.views)
            self._vlut = [0] * len(cfg.views)
            nbw = render_batch_workspace([self.sm], cfg.views, self._vsm, self._vlut, 1)
            self.workspace = torch.empty(max(nbw, 256), dtype=torch.uint8, device=self.device)
            self.tuning = cfg.tuning or BatchTuning(8, 1, 0)
            if cfg.texture:
                for k in sorted({v.level for v in cfg.views}):
                    try:
                        self.sm.make_textures([k])
                    except MctpError as e:
                        if e.code != _lib.MCTP_ESIZE:  # an atlas past the gather limit renders from loads
                            raise
        elif cfg.renderer != "views":
            raise ValueError("renderer must be 'batch' or 'views'")
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
        mark("texture")
        self.sm.update_textures(self.stream)
        mark("render")
        if c.renderer == "batch":
            render_batch([self.sm], c.views, self._vsm, self._vlut, lut, c.alpha_stop, self.tuning, self.images,
                         self.samples, self.workspace, self.stream)
        else:
            render_views(self.sm, c.views, lut, c.alpha_stop, self.images, self.samples, self.stream)
        mark("entropy")
        image_entropy(self.images, c.views, self.image_hist, self.entropy, self.best, self.stream)
        mark("end")
        return self.images, self.samples


def autotune(pipe: PreviewPipeline, lut: torch.Tensor, reps: int = 2):
    """Pick the work-queue renderer's launch shape for this pipeline's views by
    timing candidates on its current slicemap (run one pass first)."""
    from .batch import autotune_render
    if pipe.cfg.renderer != "batch":
        return None, {}
    luts = lut if lut.dim() == 3 else lut.unsqueeze(0)
    stream = pipe.stream or torch.cuda.current_stream(pipe.device)
    best, timings = autotune_render([pipe.sm], pipe.cfg.views, pipe._vsm, pipe._vlut, luts, pipe.cfg.alpha_stop,
                                    stream, reps, pipe.images, pipe.samples, pipe.workspace)
    pipe.tuning = best
    return best, timings
