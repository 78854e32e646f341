"""Many volumes through the preview path at once: per volume a histogram, a
threshold keep table and a fused filter + slicemap build; then every view of
every volume in one persistent render launch (render_batch).  The whole pass
can be captured once in a CUDA graph and replayed, so a batch costs one graph
launch on the host.  An autotuner picks the render launch shape (warp tile
shape, queue chunk, CTAs per SM) by timing candidates on the batch itself;
the shape changes speed only, never a result."""
from __future__ import annotations

import json
import os
from dataclasses import asdict, dataclass

import torch

from . import (BatchTuning, Slicemap, View, _lib, build_histogram, build_histogram_batch, build_slicemap,
               build_slicemap_batch, render_batch, render_batch_workspace, select_threshold, select_threshold_batch,
               update_textures_batch)
from ._lib import MctpError

WARP_WIDTHS = (4, 8, 16, 32)
CHUNKS = (1, 2, 4, 8, 16)
CTAS = (0, 2)


def _time_ms(fn, stream, reps: int) -> float:
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        fn()  # warm
        start.record(stream)
        for _ in range(reps):
            fn()
        end.record(stream)
    end.synchronize()
    return start.elapsed_time(end) / reps


def autotune_render(slicemaps, views, view_slicemap, view_lut, luts, alpha_stop=0.99, stream=None, reps=2,
                    out=None, samples=None, workspace=None, cache_path: str | None = None):
    """Pick the render_batch launch shape for this batch by timing.

    Coordinate search: warp tile shape at chunk 2, then the chunk at the best
    shape, then the CTA cap.  Returns (best BatchTuning, {tuning: ms}).  With
    cache_path, results are stored per batch signature (element type, level
    sizes, view count and pixels) and reused."""
    stream = stream or torch.cuda.current_stream()
    key = _signature(slicemaps, views, view_slicemap, luts)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        cache = json.load(open(cache_path))
        if key in cache:
            return BatchTuning(**cache[key]["best"]), {}
    if workspace is None:
        nb = render_batch_workspace(slicemaps, views, view_slicemap, view_lut, luts.shape[0] if luts.dim() == 3
                                    else 1)
        workspace = torch.empty(nb, dtype=torch.uint8, device=luts.device)
    total = sum(v.width * v.height * 4 for v in views)
    out = out if out is not None else torch.empty(max(total, 4), dtype=torch.float32, device=luts.device)
    samples = samples if samples is not None else torch.empty(1, dtype=torch.uint64, device=luts.device)
    timings: dict[BatchTuning, float] = {}

    def run(t: BatchTuning) -> float:
        if t not in timings:
            timings[t] = _time_ms(lambda: render_batch(slicemaps, views, view_slicemap, view_lut, luts, alpha_stop,
                                                       t, out, samples, workspace, stream), stream, reps)
        return timings[t]

    best = coordinate_search(run)
    if cache_path:
        cache[key] = dict(best=asdict(best), ms=timings[best])
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return best, timings


def coordinate_search(run) -> BatchTuning:
    """Minimise run(tuning) (ms) one parameter at a time: warp tile shape at
    chunk 2, then the chunk, then the CTA cap.  Ties keep the earlier
    candidate."""
    best = min((BatchTuning(w, 2, 0) for w in WARP_WIDTHS), key=run)
    best = min((BatchTuning(best.warp_w, c, 0) for c in CHUNKS), key=run)
    return min((BatchTuning(best.warp_w, best.chunk, k) for k in CTAS), key=run)


def _signature(slicemaps, views, view_slicemap, luts) -> str:
    dims = sorted({(sm.dims[v.level], str(sm.dtype)) for v, s in zip(views, view_slicemap)
                   for sm in [slicemaps[s]]})
    pix = sum(v.width * v.height for v in views)
    gather = all(sm.textures is not None and sm.textures[v.level] is not None
                 for v, s in zip(views, view_slicemap) for sm in [slicemaps[s]])
    return json.dumps(dict(levels=[list(d) + [t] for d, t in dims][:16], nviews=len(views), pixels=pix,
                           nlut=int(luts.shape[-2]), gather=gather))


@dataclass
class BatchItem:
    """One volume of a batch with its views."""
    volume: torch.Tensor      # [nz][ny][nx] uint8 / uint16, resident on the device
    bits: int
    views: list[View]
    lut: int = 0              # index into the batch's transfer functions


class BatchPipeline:
    """The preview path over many volumes; `run()` enqueues one pass on `stream`."""

    def __init__(self, items: list[BatchItem], level0, nlevels: int, luts: torch.Tensor, nbins: int = 256,
                 mode: str = "otsu", alpha_stop: float = 0.99, tuning: BatchTuning | None = None,
                 device="cuda", stream=None, maxgrid: bool = True, texture: bool = True):
        self.items = items
        self.device = torch.device(device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.luts = luts if luts.dim() == 3 else luts.unsqueeze(0)
        self.nbins, self.mode, self.alpha_stop = nbins, mode, alpha_stop
        self.tuning = tuning or BatchTuning()
        n = len(items)
        self.hist = torch.empty((n, nbins), dtype=torch.uint64, device=self.device)
        self.overflow = torch.empty((n, 1), dtype=torch.uint64, device=self.device)
        self.keep = torch.empty((n, nbins), dtype=torch.uint8, device=self.device)
        self.result = torch.empty((n, 4), dtype=torch.int32, device=self.device)
        self.slicemaps = []
        for it in items:
            nz, ny, nx = it.volume.shape
            self.slicemaps.append(Slicemap.allocate((nx, ny, nz), level0, nlevels, it.volume.dtype, it.bits,
                                                    self.device, maxgrid=maxgrid))
        self.views, self.view_slicemap, self.view_lut = [], [], []
        for i, it in enumerate(items):
            for v in it.views:
                self.views.append(v)
                self.view_slicemap.append(i)
                self.view_lut.append(it.lut)
        if texture:
            # atlas textures of the rendered levels; the render gathers corner quads through them
            # when every (slicemap, level) has one, else it loads from the atlases
            for i, it in enumerate(items):
                for k in sorted({v.level for v in it.views}):
                    try:
                        self.slicemaps[i].make_textures([k])
                    except MctpError as e:
                        if e.code != _lib.MCTP_ESIZE:
                            raise
        total = sum(v.width * v.height * 4 for v in self.views)
        self.images = torch.empty(max(total, 4), dtype=torch.float32, device=self.device)
        self.samples = torch.empty(1, dtype=torch.uint64, device=self.device)
        nb = render_batch_workspace(self.slicemaps, self.views, self.view_slicemap, self.view_lut,
                                    self.luts.shape[0])
        self.workspace = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self.graph = None

    def prepare(self):
        """Histograms, keep tables and slicemaps of every volume (enqueued):
        one histogram launch, one keep-table launch, the slicemap builds with
        one max-grid launch, one texture launch (volumes of one dtype and bit
        depth; otherwise volume by volume)."""
        s = self.stream
        vols = [it.volume for it in self.items]
        uniform = len({(v.dtype, it.bits) for v, it in zip(vols, self.items)}) == 1
        if not uniform:
            for i, it in enumerate(self.items):
                keep = None
                if self.mode != "none":
                    build_histogram(it.volume, it.bits, self.nbins, 0, None, self.hist[i], self.overflow[i], s)
                    select_threshold(self.hist[i], self.nbins, self.mode, keep=self.keep[i], result=self.result[i],
                                     stream=s)
                    keep = self.keep[i]
                build_slicemap(it.volume, it.bits, self.slicemaps[i], keep, s)
                self.slicemaps[i].update_textures(s)
            return
        bits = self.items[0].bits
        keep = None
        if self.mode != "none":
            build_histogram_batch(vols, bits, self.nbins, self.hist, self.overflow, s)
            select_threshold_batch(self.hist, self.mode, keep=self.keep, result=self.result, stream=s)
            keep = self.keep
        build_slicemap_batch(vols, bits, self.slicemaps, keep, s)
        update_textures_batch(self.slicemaps, s)

    def render(self):
        render_batch(self.slicemaps, self.views, self.view_slicemap, self.view_lut, self.luts, self.alpha_stop,
                     self.tuning, self.images, self.samples, self.workspace, self.stream)

    def run(self, timer=None):
        mark = timer or (lambda name: None)
        mark("prepare")
        self.prepare()
        mark("render")
        self.render()
        mark("end")
        return self.images, self.samples

    def autotune(self, reps: int = 2, cache_path: str | None = None):
        """Run the slicemap builds once, then tune the render launch shape on them."""
        with torch.cuda.stream(self.stream):
            self.prepare()
        self.tuning, timings = autotune_render(self.slicemaps, self.views, self.view_slicemap, self.view_lut,
                                               self.luts, self.alpha_stop, self.stream, reps, self.images,
                                               self.samples, self.workspace, cache_path)
        return self.tuning, timings

    def capture(self):
        """Capture one whole pass in a CUDA graph (after a warm-up pass)."""
        with torch.cuda.stream(self.stream):
            self.run()
        self.stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            self.run()
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()
        return self.images, self.samples
