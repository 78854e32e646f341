"""Benchmark of the micro-CT preview hot path (one JSON line on rank 0).

A step is one pass of the whole path over the 'full' workload: u16 12-bit
2016 x 2016 x 1800 phantom (14.6 GB, resident in HBM) -> 4096-bin histogram ->
Otsu keep table -> fused filter + slicemap levels 512^3 / 256^3 / 128^3 ->
36-view turntable at 1024 x 1024 (step 0.5, ramp transfer function, early
exit at alpha 0.99).  value = ray samples marched per second over whole
steps.  The input (14.6 GB) is larger than L2, so no flush is needed between
steps.  Multi-GPU runs are independent replicas (weak scaling).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mctp|reference]
                  [--workload full|mid|slab|small|batch|serve|fit|thresholds]

--workload batch: 64 u8 phantoms with axes ~ U{384..1024} (22 GB resident),
each through histogram, Otsu and a 256^3 slicemap, then 12 views of each at
512 x 512 in one persistent render launch, the whole pass replayed as one
CUDA graph; the line also times the plain per-volume and per-view render
launches on the same slicemaps.

--workload serve: 200 resident u8 cubes (edge ~ U{256..1024}, 71 GB) with
256^3 + 128^3 slicemaps; Poisson streams of preview requests (512^2 or
1024^2, azimuth U[0, 360), elevation U[-60, 60], one of 8 transfer
functions) at swept rates, served by the continuous-batching server and by
one render_views launch per request; p50/p99 latency and samples/s per rate.

--workload fit: a 1024^3 u8 phantom rendered from its full-resolution level
at 24 views 512^2 (azimuth 15k deg, elevation alternating +-20 deg) as FP32
targets; a 128^3 FP32 reduced volume (started from the 128^3 slicemap level)
and its 256-entry LUT are fitted by Adam through the adjoint ray march; a
step is one iteration (forward, loss, adjoint, two Adam updates).

--workload thresholds: the Otsu / ITS comparison of Fig. 5 on five u8
phantoms with a sample container, sized like Table II's datasets A-E: the
histogram, Otsu and ITS on the GPU (and the oracle's Otsu and ITS on the host),
before and after container removal.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ray samples/s + slicemap build HBM GB/s (% of peak); p50/p99 preview latency"
UNIT = "ray samples/s"
# algorithmic FP32 work of one sample: trilinear 21, normalisation 2, LUT coordinate 3, LUT
# lerps 12, compositing 9, position step 1
FP32_FLOPS_PER_SAMPLE = 48


def workload(name: str):
    import phantom
    if name == "full":
        spec = phantom.FULL
        return dict(spec=spec, bits=12, nbins=4096, level0=(512, 512, 512), nlevels=3, nviews=36, size=1024,
                    az_step=10.0, desc="full: u16 12-bit 2016x2016x1800 phantom (14.6 GB), 4096 bins, Otsu, "
                                       "levels 512^3/256^3/128^3, 36-view turntable 1024x1024, step 0.5")
    if name == "mid":
        spec = phantom.VolumeSpec(1008, 1008, 900, bits=12, seed=1002, n_ell=12, n_cyl=300)
        return dict(spec=spec, bits=12, nbins=4096, level0=(512, 512, 512), nlevels=3, nviews=36, size=1024,
                    az_step=10.0, desc="mid (profiling): u16 12-bit 1008x1008x900 phantom (1.8 GB), 4096 bins, "
                                       "Otsu, levels 512^3/256^3/128^3, 36-view turntable 1024x1024, step 0.5")
    if name == "slab":
        spec = phantom.VolumeSpec(2016, 2016, 224, bits=12, seed=1002, n_ell=12, n_cyl=300)
        return dict(spec=spec, bits=12, nbins=4096, level0=(512, 512, 64), nlevels=3, nviews=4, size=1024,
                    az_step=10.0, desc="slab (profiling): u16 12-bit 2016x2016x224 phantom (1.8 GB) with the full "
                                       "workload's footprints, 4096 bins, Otsu, levels 512x512x64/256x256x32/"
                                       "128x128x16, 4 views 1024x1024")
    if name == "thresholds":
        dims = [(1536, 1536, 1152), (1536, 1536, 1152), (2016, 2016, 2016), (2016, 2016, 1692), (1968, 1968, 1456)]
        specs = [phantom.VolumeSpec(x, y, z, bits=8, seed=6000 + i, n_ell=12, tube=True)
                 for i, (x, y, z) in enumerate(dims)]
        return dict(specs=specs, spec=specs[0], bits=8, nbins=256, level0=(256, 256, 256), nlevels=1, nviews=1,
                    size=512, az_step=0.0,
                    desc="thresholds: 5 u8 phantoms with a container, sized like Table II A-E (1536^2x1152 x2, "
                         "2016^2x2016, 2016^2x1692, 1968^2x1456; %.1f GB), 256 bins; Otsu and ITS before and "
                         "after container removal" % (sum(sp.nbytes for sp in specs) / 1e9))
    if name == "fit":
        spec = phantom.VolumeSpec(1024, 1024, 1024, bits=8, seed=1004, n_ell=12, n_cyl=0)
        return dict(spec=spec, bits=8, nbins=256, level0=(1024, 1024, 1024), nlevels=4, nviews=24, size=512,
                    az_step=15.0, elevation=20.0,
                    desc="fit: u8 1024^3 phantom (1.07 GB), Otsu, slicemap 1024^3..128^3; 24 target views 512x512 "
                         "(az 15k deg, el +-20 deg) of the 1024^3 level, LUT preset 5; fit 128^3 FP32 volume + "
                         "256x4 LUT by Adam (lr 1e-2 / 5e-3) through the adjoint march (checkpoints every 64 "
                         "samples), step 0.5 level voxel, alpha_stop 0.99")
    if name == "serve":
        specs = phantom.serve_specs(200)
        return dict(specs=specs, spec=specs[0], bits=8, nbins=256, level0=(256, 256, 256), nlevels=2, nviews=1,
                    size=512, az_step=0.0, rates=(1000.0, 2500.0, 5000.0, 7500.0, 10000.0, 12500.0, 15000.0, 20000.0),
                    requests=1500,
                    desc="serve: 200 resident u8 cubes, edge ~U{256..1024} (%.1f GB), 256 bins, Otsu, slicemap "
                         "levels 256^3/128^3, Poisson requests 512^2|1024^2, az U[0,360), el U[-60,60], LUT from "
                         "8 presets, step 0.5, level 0" % (sum(sp.nbytes for sp in specs) / 1e9))
    if name == "batch8":
        specs = phantom.batch_specs(64)[:8]
        return dict(specs=specs, spec=specs[0], bits=8, nbins=256, level0=(256, 256, 256), nlevels=1, nviews=12,
                    size=512, az_step=30.0, elevation=20.0,
                    desc="batch8 (profiling): the first 8 volumes of the batch workload (%.1f GB), otherwise "
                         "the same" % (sum(sp.nbytes for sp in specs) / 1e9))
    if name == "batch":
        specs = phantom.batch_specs(64)
        return dict(specs=specs, spec=specs[0], bits=8, nbins=256, level0=(256, 256, 256), nlevels=1, nviews=12,
                    size=512, az_step=30.0, elevation=20.0,
                    desc="batch: 64 u8 phantoms, axes ~U{384..1024} (%.1f GB), 256 bins, Otsu, one 256^3 level "
                         "each, 12 views 512x512 (az 30k deg, el 20 deg), step 0.5, ramp LUT, one persistent "
                         "render launch, CUDA graph" % (sum(sp.nbytes for sp in specs) / 1e9))
    spec = phantom.SMALL
    return dict(spec=spec, bits=8, nbins=256, level0=(128, 128, 128), nlevels=1, nviews=1, size=256,
                az_step=0.0, desc="small: u8 256^3 phantom, 256 bins, Otsu, level 128^3, 1 view 256x256")


KERNEL_SOURCES = {"histogram": ["hist.cu"], "slicemap": ["slicemap.cu", "slicemap_common.cuh"],
                  "render": ["render_batch.cu", "render_common.cuh"], "threshold": ["threshold.cu"]}


def source_sha256(files) -> str:
    """SHA-256 over the kernel's source files, in order."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2311_15038_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def measured_traffic():
    """ncu DRAM bytes per launch (profiles/traffic.json), kept only while the
    kernel's source files are unchanged since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    out = {}
    if not os.path.exists(path):
        return out
    rec = json.load(open(path))
    for kernel, files in KERNEL_SOURCES.items():
        r = rec.get(kernel)
        if not r:
            continue
        out[kernel] = r["bytes_per_launch"] if source_sha256(files) == r.get("source_sha256") else None
    return out


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)),
                    source="measured")
    return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, source="fallback")


def sm_count(device=None) -> int:
    """SMs of the GPU, queried from the device."""
    import torch
    return int(torch.cuda.get_device_properties(device if device is not None else 0).multi_processor_count)


def fp32_peak(pk, device=None):
    """Nominal FP32 rate (TFLOP/s): SMs (queried) x 128 FP32 lanes x 2 flop (FMA) x the maximum SM clock
    (from MEASURED_PEAKS.json when present); a figure from unit counts, not a measurement."""
    return sm_count(device) * 128 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12


FP32_PEAK_SOURCE = "nominal: SMs (queried) x 128 FP32 lanes x 2 flop x maximum SM clock"
FLOPS_SOURCE = ("hand count of the FP32 operations of one evaluated sample: trilinear 21, normalisation 2, "
                "LUT coordinate 3, LUT lerps 12, compositing 9, position step 1")


def render_issue_roofline(evaluated, render_s, pk, device=None):
    """Issue-rate view of the renderer, which is bound by instruction issue, not by its FP32 work: warp
    instructions per evaluated sample from an ncu count (profiles/render_counters.json, kept only while
    the kernel's sources are unchanged) x evaluated samples / render time, against SMs x 4 schedulers x
    one warp instruction per clock."""
    path = os.path.join(ROOT, "profiles", "render_counters.json")
    peak = sm_count(device) * 4 * pk["sm_max_mhz"] * 1e6
    out = dict(unit="warp instructions/s", peak=peak, peak_source="nominal: SMs x 4 schedulers x max SM clock",
               warp_inst_per_evaluated_sample=None, thread_inst_per_evaluated_sample=None, achieved=None, frac=None)
    if not os.path.exists(path):
        return out
    rec = json.load(open(path))
    if source_sha256(KERNEL_SOURCES["render"]) != rec.get("source_sha256"):
        return out
    wpe = rec["warp_inst_executed"] / rec["evaluated_samples"]
    out.update(warp_inst_per_evaluated_sample=wpe,
               thread_inst_per_evaluated_sample=rec["thread_inst_executed"] / rec["evaluated_samples"],
               lanes_per_warp_inst=rec["thread_inst_executed"] / rec["warp_inst_executed"],
               achieved=wpe * evaluated / render_s, frac=wpe * evaluated / render_s / peak,
               counters_from=rec.get("workload"))
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"])
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=reasons, samples=len(rows))


def launches_per_step(wl, nviews, ntex):
    """Kernels of this library launched by one step: histogram, threshold
    selection, the level-0 slicemap kernel (levels 1-2 fused), one 2x2x2 kernel
    per further level, one max-grid kernel per level, one texture update per
    textured level, the work-queue renderer (set-up kernel, depth-bounds
    kernel, one view-upload kernel per 128 views, the render kernel), one
    image-histogram launch per 1024 views, the entropy and best-view kernels."""
    nl = wl["nlevels"]
    return (1 + 1 + 1 + max(0, nl - 3) + nl + ntex + 3 + (nviews + 127) // 128 + (nviews + 1023) // 1024 + 2)


def batch_launches_per_step(nvol, nviews):
    """Kernels of this library launched by one pass of the batched workload:
    the histograms, the keep tables, the max grids and the texture updates of
    up to 64 volumes per launch, one level-0 kernel per volume, and the
    work-queue renderer (set-up, depth bounds, one view upload per 128 views,
    render)."""
    per64 = (nvol + 63) // 64
    return 3 * per64 + 1 + nvol + 3 + (nviews + 127) // 128


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int, device) -> float:
    """The largest value of x over all ranks (x itself on one rank): the job's
    time is the slowest replica's."""
    if ws <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank_step: float, steps: int, ws: int, seconds: float) -> float:
    """Whole-job throughput of N replicas (weak scaling): every rank processes
    the same units per step, and the job takes the slowest rank's time."""
    return units_per_rank_step * steps * ws / seconds


# --------------------------------------------------------------- CPU oracle

def host_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _pool_map(fn, items, threads):
    """fn over items on `threads` host threads (the oracle's C calls release the GIL)."""
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(fn, items))


def oracle_level0_threaded(vol_np, bits, M, keep, threads):
    """The oracle's level 0 of vol_np computed in z-slabs on host threads.
    Output slice z covers source slices [floor(z N / M), floor((z + 1) N / M));
    where z N / M is an integer a slab of g = M / gcd(N, M) output slices has
    exactly the footprints of the whole volume, so the slabs' levels stack to
    the whole level.  Returns (level, slabs)."""
    import math
    import oracle
    nz = vol_np.shape[0]
    g = M[2] // math.gcd(nz, M[2])
    nslab = M[2] // g
    src_per = nz // nslab
    slabs = _pool_map(lambda i: oracle.downsample(vol_np[i * src_per:(i + 1) * src_per], bits, (M[0], M[1], g), keep),
                      range(nslab), threads)
    return np.concatenate(slabs, axis=0), nslab


def oracle_full_step(wl, vol_np, threads=None):
    """The oracle on the full step's own data, on the host's cores: the
    histogram of the whole volume (threads over z-slabs; the slab counts add
    up exactly), Otsu, the level-0 slicemap of the whole volume (threads over
    source slabs whose footprints fill whole output slices, so each slab's
    level equals its part of the full level), the coarser levels, and one
    full view of the turntable (threads over rays).  The step's other views
    are extrapolated from that one.  Returns a cpu_baseline record."""
    import oracle
    import phantom
    threads = threads or host_threads()
    spec, bits, nbins = wl["spec"], wl["bits"], wl["nbins"]
    nz, ny, nx = vol_np.shape
    M = wl["level0"]
    t = {}
    t0 = time.perf_counter()
    zs = np.linspace(0, nz, min(threads, nz) + 1).astype(int)
    parts = _pool_map(lambda i: oracle.histogram(vol_np, bits, nbins, int(zs[i]), int(zs[i + 1])),
                      range(len(zs) - 1), threads)
    hist = sum(p[0] for p in parts)
    t["histogram"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    T, _ = oracle.otsu(hist)
    keep = oracle.keep_threshold(nbins, T)
    t["threshold"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    level0, nslab = oracle_level0_threaded(vol_np, bits, M, keep, threads)
    dims = [M]
    for _ in range(1, wl["nlevels"]):
        dims.append(tuple(d // 2 for d in dims[-1]))
    lv = level0
    for d in dims[1:]:
        lv = oracle.downsample(lv, bits, d)
    t["slicemap"] = time.perf_counter() - t0
    size = wl["size"]
    lut = phantom.ramp_lut(256)
    pix = np.arange(size * size, dtype=np.int64)
    chunks = np.array_split(pix, threads * 8)
    t0 = time.perf_counter()
    outs = _pool_map(lambda c: oracle.render(level0, bits, (spec.nx, spec.ny, spec.nz), lut, 0.0, 0.0, size, size,
                                             0.5, 0.99, 0.0, pixels=c), chunks, threads)
    t["render_one_view"] = time.perf_counter() - t0
    view_samples = float(sum(o["nsamp"][:, 1].sum() for o in outs))
    nviews = wl["nviews"]
    step_s = t["histogram"] + t["threshold"] + t["slicemap"] + nviews * t["render_one_view"]
    samples = view_samples * nviews
    return dict(value=samples / step_s, unit=UNIT, cores=threads, host_cpus=os.cpu_count(), kind="oracle",
                extrapolated=f"render: 1 of {nviews} views measured, the step's time counts it {nviews} times",
                seconds=dict(t, step=step_s), samples_one_view=int(view_samples),
                sample=f"oracle (C, {threads} threads): {nbins}-bin histogram of the whole {vol_np.nbytes / 1e9:.1f} GB "
                       f"volume, Otsu (T={T}), level 0 ({M[0]}x{M[1]}x{M[2]}) of the whole volume in {nslab} "
                       f"slabs and the coarser levels, one full {size}x{size} view (az 0) of level 0; "
                       f"{sum(t.values()):.1f} s measured")


def oracle_sample(wl, slab=None, npix=8192):
    """Time the oracle on a bounded sample of the workload and extrapolate its
    step time.  Sample: the histogram and slicemap of a 96-slice slab around
    the middle of the volume, Otsu on that histogram, and 8192 rays of one
    view aimed at the band of image rows the slab covers (so rays meet
    objects and exit early as in the full step).  Returns (seconds per full
    step, ray samples per full step, description)."""
    import oracle
    import phantom
    spec, bits, nbins = wl["spec"], wl["bits"], wl["nbins"]
    M = wl["level0"]
    nz_s = min(spec.nz, 96)
    zs = spec.nz // 2 - nz_s // 2
    if slab is None:
        slab = phantom.generate_cpu(spec, ((0, spec.nx), (0, spec.ny), (zs, zs + nz_s)))
    frac_v = nz_s / spec.nz
    t0 = time.perf_counter()
    hist, _ = oracle.histogram(slab, bits, nbins)
    t_hist = time.perf_counter() - t0
    t0 = time.perf_counter()
    T, _ = oracle.otsu(hist)
    t_otsu = time.perf_counter() - t0
    keep = oracle.keep_threshold(nbins, T)
    mz_s = max(1, int(round(M[2] * frac_v)))
    t0 = time.perf_counter()
    lv = oracle.downsample(slab, bits, (M[0], M[1], mz_s), keep)
    t_sm = time.perf_counter() - t0
    level = np.zeros((M[2], M[1], M[0]), lv.dtype)
    z0 = (M[2] - mz_s) // 2
    level[z0:z0 + mz_s] = lv
    size = wl["size"]
    L = float(np.sqrt(float(spec.nx) ** 2 + float(spec.ny) ** 2 + float(spec.nz) ** 2))
    half_rows = max(1, int(0.5 * nz_s / (L / size)))
    rng = np.random.default_rng(0)
    rows = rng.integers(size // 2 - half_rows, size // 2 + half_rows, size=npix)
    pix = rows * size + rng.integers(0, size, size=npix)
    t0 = time.perf_counter()
    ref = oracle.render(level, bits, (spec.nx, spec.ny, spec.nz), phantom.ramp_lut(256), 30.0, 0.0, size, size,
                        0.5, 0.99, 0.0, pixels=pix)
    t_r = time.perf_counter() - t0
    ns = float(ref["nsamp"][:, 1].sum())
    rays_full = wl["nviews"] * size ** 2
    samples_step = ns * rays_full / npix
    step_s = t_hist / frac_v + t_otsu + t_sm / frac_v + t_r * rays_full / npix
    text = (f"oracle (C, 1 thread): histogram + slicemap of {nz_s}/{spec.nz} slices, Otsu, {npix} rays "
            f"({int(ns)} samples) through that slab; extrapolated to one full step; "
            f"{t_hist + t_otsu + t_sm + t_r:.1f} s measured")
    return step_s, samples_step, text


def generate_host(spec, threads=None):
    """The seeded phantom written on the host's cores, slab by slab."""
    import phantom
    threads = threads or host_threads()
    vol = np.empty(spec.shape, dtype=np.uint8 if spec.esize == 1 else np.uint16)
    zs = np.linspace(0, spec.nz, min(spec.nz, 4 * threads) + 1).astype(int)

    def one(i):
        z0, z1 = int(zs[i]), int(zs[i + 1])
        if z1 > z0:
            vol[z0:z1] = phantom.generate_cpu(spec, ((0, spec.nx), (0, spec.ny), (z0, z1)))
    _pool_map(one, range(len(zs) - 1), threads)
    return vol


def run_reference(args, wl):
    """The reference arm: this build's CPU oracle (the paper has no code) on
    the same workload, every step the full step of oracle_full_step on the
    host's cores; the warm-up steps are one slab's histogram each."""
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    import phantom
    phantom.build(gpu=False)
    vol = generate_host(wl["spec"])
    for _ in range(args.warmup):
        oracle.histogram(vol[: max(1, vol.shape[0] // 64)], wl["bits"], wl["nbins"])
    recs = [oracle_full_step(wl, vol) for _ in range(args.steps)]
    rec = sorted(recs, key=lambda r: r["value"])[len(recs) // 2]
    value = rec["value"]
    step_s = rec["seconds"]["step"]
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps,
                warmup=args.warmup, ms_per_step=step_s * 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="u16/f64", data="synthetic",
                config=dict(workload=wl["desc"], l2="n/a (CPU)"),
                cpu_baseline=rec,
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- GPU

def run_gpu(args, wl):
    import torch
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    if ws > 1:
        torch.distributed.barrier()   # rank 0 built the shared in-tree libraries
    import phantom
    import paper_2311_15038_gb300 as mctp
    from paper_2311_15038_gb300 import pipeline as pl
    mctp._lib.load()

    spec = wl["spec"]
    dtype = torch.uint8 if spec.esize == 1 else torch.uint16
    vol = torch.empty(spec.shape, dtype=dtype, device=dev)
    phantom.generate_gpu(spec, vol)
    lut = torch.from_numpy(phantom.ramp_lut(256)).to(dev)
    views = pl.turntable(wl["nviews"], wl["size"], 0, 0.5, 0.0, wl["az_step"] or None)
    cfg = pl.PreviewConfig((spec.nx, spec.ny, spec.nz), wl["bits"], wl["nbins"], wl["level0"], wl["nlevels"],
                           views, "otsu", 3, 0.99)
    stream = torch.cuda.Stream(dev)
    pipe = pl.PreviewPipeline(cfg, dtype, dev, stream)

    stages = ["histogram", "threshold", "slicemap", "texture", "render", "entropy"]
    ev = {}

    def timer(name):
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        ev.setdefault(name, []).append(e)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            pipe.run(vol, lut)
    torch.cuda.synchronize(dev)
    if args.render_tuning:
        w, c, k = (int(x) for x in args.render_tuning.split(","))
        tuning = pipe.tuning = mctp.BatchTuning(w, c, k)
    else:
        tuning, _ = pl.autotune(pipe, lut)
    with torch.cuda.stream(stream):
        pipe.run(vol, lut)
    torch.cuda.synchronize(dev)
    samples_per_step = int(pipe.samples.item())
    # samples one step evaluates (the rest are skipped as empty): one counted render, untimed
    mctp.render_batch([pipe.sm], views, pipe._vsm, pipe._vlut, lut, 0.99,
                      dataclasses.replace(tuning, count_evaluated=True), pipe.images, pipe.samples, pipe.workspace,
                      stream)
    evaluated_per_step = mctp.batch_samples_evaluated(pipe.workspace)
    assert int(pipe.samples.item()) == samples_per_step

    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    step_events = []
    t_start.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            s0 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            pipe.run(vol, lut, timer)
            s1 = torch.cuda.Event(enable_timing=True)
            s1.record(stream)
            step_events.append((s0, s1))
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    elapsed = max_over_ranks(elapsed, ws, dev)
    step_ms = [a.elapsed_time(b) for a, b in step_events]
    stage_ms = {}
    for i, name in enumerate(stages):
        nxt = stages[i + 1] if i + 1 < len(stages) else "end"
        stage_ms[name] = statistics.mean(a.elapsed_time(b) for a, b in zip(ev[name], ev[nxt]))
    assert int(pipe.samples.item()) == samples_per_step

    # ---- end to end through the public API: pinned host volume in, images out
    vol_host = torch.empty(spec.shape, dtype=dtype, pin_memory=True)
    vol_host.copy_(vol)
    img_host = torch.empty(pipe.images.shape, dtype=torch.float32, pin_memory=True)
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(e2e_steps):
            vol.copy_(vol_host, non_blocking=True)
            pipe.run(vol, lut)
            img_host.copy_(pipe.images, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_s = e0.elapsed_time(e1) / 1e3 / e2e_steps
    e2e_s = max_over_ranks(e2e_s, ws, dev)

    if rank != 0:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
        return 0

    pk = peaks()
    vol_bytes = spec.nbytes
    atlas_bytes = sum(a.numel() * a.element_size() for a in pipe.sm.atlases)
    level0_bytes = pipe.sm.atlases[0].numel() * pipe.sm.atlases[0].element_size()
    image_bytes = pipe.images.numel() * 4
    # atlas textures: each rendered level's atlas read once and written once into its texture
    tex_bytes = sum(a.numel() * a.element_size() for a, t in zip(pipe.sm.atlases, pipe.sm.textures or [])
                    if t is not None)
    sm_mhz = clk.get("sm_mhz") or pk["sm_max_mhz"]
    kernels = {
        "histogram": dict(bound="hbm", bytes=vol_bytes, unit="GB/s"),
        "slicemap": dict(bound="hbm", bytes=vol_bytes + atlas_bytes, unit="GB/s"),
        "texture": dict(bound="hbm", bytes=2 * tex_bytes, unit="GB/s"),
        "render": dict(bound="alu", flops=FP32_FLOPS_PER_SAMPLE * evaluated_per_step, unit="TFLOP/s"),
        "threshold": dict(bound="alu", flops=0, unit="TFLOP/s"),
        "entropy": dict(bound="hbm", bytes=image_bytes, unit="GB/s"),
    }
    fp32 = fp32_peak(pk, dev)
    traffic = measured_traffic() if args.workload == "full" else {}
    roof = {}
    for name, k in kernels.items():
        t = stage_ms[name] / 1e3
        if k["bound"] == "hbm":
            ach = k["bytes"] / t / 1e9
            roof[name] = dict(bound="hbm", achieved=ach, peak=pk["hbm_gbs"], unit="GB/s",
                              frac=ach / pk["hbm_gbs"], ms=stage_ms[name], traffic=traffic.get(name))
        else:
            ach = k["flops"] / t / 1e12
            roof[name] = dict(bound="alu", achieved=ach, peak=fp32, unit="TFLOP/s",
                              frac=ach / fp32, ms=stage_ms[name], traffic=traffic.get(name),
                              peak_source=FP32_PEAK_SOURCE)
    roof["render"]["compulsory_hbm_gbs"] = wl["nviews"] * level0_bytes / (stage_ms["render"] / 1e3) / 1e9
    roof["render"]["flops_per_sample"] = FP32_FLOPS_PER_SAMPLE
    roof["render"]["flops_source"] = FLOPS_SOURCE
    roof["render"]["issue"] = render_issue_roofline(evaluated_per_step, stage_ms["render"] / 1e3, pk, dev)
    for name in ("histogram", "slicemap", "texture", "entropy"):
        roof[name]["peak_source"] = pk["source"] + " HBM copy bandwidth"
    dominant = max(stage_ms, key=stage_ms.get)
    value = job_rate(samples_per_step, args.steps, ws, elapsed)
    best_view = int(pipe.best.item())
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps, warmup=args.warmup,
        ms_per_step=elapsed * 1e3 / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="u16/f32", data="synthetic",
        best_view=dict(index=best_view, azimuth_deg=views[best_view].azimuth_deg,
                       entropy_bits=float(pipe.entropy[best_view].item())),
        config=dict(workload=wl["desc"], l2="inputs larger than L2 (14.6 GB volume; no flush)"
                    if vol_bytes > 200e6 else "input fits in L2 (L2-resident numbers)",
                    parallelism=f"replicas x{ws}", renderer="render_batch (work queue)",
                    tuning=dict(warp_w=tuning.warp_w, chunk=tuning.chunk, ctas_per_sm=tuning.ctas_per_sm)),
        samples_per_step=samples_per_step,
        samples_evaluated_per_step=evaluated_per_step,
        slicemap_gbs=roof["slicemap"]["achieved"], slicemap_frac_of_hbm_peak=roof["slicemap"]["frac"],
        histogram_gbs=roof["histogram"]["achieved"],
        render_samples_per_s=samples_per_step / (stage_ms["render"] / 1e3),
        render_evaluated_samples_per_s=evaluated_per_step / (stage_ms["render"] / 1e3),
        evaluated_share=evaluated_per_step / samples_per_step,
        latency_ms=dict(p50=float(np.percentile(step_ms, 50)), p99=float(np.percentile(step_ms, 99))),
        stage_ms=stage_ms,
        roofline=dict(roof[dominant], kernel=dominant),
        roofline_by_kernel=roof,
        gpu_launches=launches_per_step(wl, len(views), sum(t is not None for t in pipe.sm.textures or []))
        * args.steps,
        clocks=dict(sm_mhz=clk.get("sm_mhz"), sm_max_mhz=clk.get("sm_max_mhz"), reasons=clk.get("reasons")),
        e2e=dict(value=samples_per_step / e2e_s, unit=UNIT, h2d_bytes_per_step=vol_bytes,
                 d2h_bytes_per_step=image_bytes, ms_per_step=e2e_s * 1e3),
    )
    if not args.no_next_rows and args.workload == "full":
        line["next_rows"] = next_rows_record(dev)
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        line["cpu_baseline"] = oracle_full_step(wl, vol_host.numpy())
    del vol_host
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def next_rows_record(dev, rate: float = 4000.0, requests: int = 400):
    """Compact measurements of the batched renderer and the server beside the
    main step: the first 8 volumes of the batched workload (u8, axes
    ~U{384..1024}, 256^3 levels, 12 views 512^2 each) rendered by one batched
    launch, by one render_views launch per volume and by one per view (images
    and sample counts asserted equal); and a Poisson stream of requests
    (512^2 / 1024^2, random azimuth and elevation, 8 transfer functions) on
    those 8 slicemaps served by the continuous-batching server and by
    per-view launches, p50/p99 latency and samples/s."""
    import torch
    import phantom
    import paper_2311_15038_gb300 as mctp
    from paper_2311_15038_gb300 import batch as bt
    from paper_2311_15038_gb300 import pipeline as pl
    from paper_2311_15038_gb300 import serve as sv
    wl = workload("batch8")
    stream = torch.cuda.Stream(dev)
    vols = []
    for sp in wl["specs"]:
        v = torch.empty(sp.shape, dtype=torch.uint8, device=dev)
        phantom.generate_gpu(sp, v)
        vols.append(v)
    lut = torch.from_numpy(phantom.ramp_lut(256)).to(dev)
    views = pl.turntable(wl["nviews"], wl["size"], 0, 0.5, wl["elevation"], wl["az_step"])
    pipe = bt.BatchPipeline([bt.BatchItem(v, 8, views, 0) for v in vols], wl["level0"], wl["nlevels"], lut,
                            wl["nbins"], "otsu", 0.99, device=dev, stream=stream)
    pipe.autotune(reps=1)
    torch.cuda.synchronize(dev)
    px = wl["size"] * wl["size"] * 4
    plain = torch.empty_like(pipe.images)
    s_vol = [torch.empty(1, dtype=torch.uint64, device=dev) for _ in vols]
    s_view = [torch.empty(1, dtype=torch.uint64, device=dev) for _ in pipe.views]

    def per_volume():
        for i, sm in enumerate(pipe.slicemaps):
            mctp.render_views(sm, views, lut, 0.99, plain[i * len(views) * px:(i + 1) * len(views) * px], s_vol[i],
                              stream)

    def per_view():
        for j, v in enumerate(pipe.views):
            mctp.render_views(pipe.slicemaps[pipe.view_slicemap[j]], [v], lut, 0.99, plain[j * px:(j + 1) * px],
                              s_view[j], stream)

    def timed(fn, reps=3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            fn()
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps
    ms = dict(batched=timed(pipe.render))
    samples = int(pipe.samples.item())
    ref = pipe.images.clone()
    ms["per_volume"] = timed(per_volume)
    torch.cuda.synchronize(dev)
    equal = torch.equal(plain, ref) and sum(int(s.item()) for s in s_vol) == samples
    ms["per_view"] = timed(per_view)
    torch.cuda.synchronize(dev)
    equal = equal and torch.equal(plain, ref) and sum(int(s.item()) for s in s_view) == samples
    assert equal, "batched images differ from the per-volume / per-view launches"
    batch = dict(workload=wl["desc"], views=len(pipe.views), samples=samples, render_ms=ms,
                 samples_per_s={k: samples / (t / 1e3) for k, t in ms.items()},
                 speedup_vs_per_view=ms["per_view"] / ms["batched"], images_equal=True,
                 tuning=dict(warp_w=pipe.tuning.warp_w, chunk=pipe.tuning.chunk, ctas_per_sm=pipe.tuning.ctas_per_sm))
    # ---- serving the same slicemaps
    luts = torch.from_numpy(np.stack(phantom.preset_luts())).to(dev)
    serving = {}
    for name, cfg in (("per_view", dict(mode="per_view", max_batch_views=1, max_inflight=1)),
                      ("batched", dict(mode="batched", max_batch_views=64, max_inflight=2))):
        srv = sv.Server(pipe.slicemaps, luts, 2 << 30, **cfg)
        try:
            sv.run_trace(srv, sv.poisson_trace(2000.0, 100, len(vols), luts.shape[0], seed=98))
            trace = sv.poisson_trace(rate, requests, len(vols), luts.shape[0], seed=5)
            s0 = srv.stats()["samples"]
            done = sv.run_trace(srv, trace)
            s1 = srv.stats()["samples"]
        finally:
            srv.close()
        lat = np.array([f.t_done - a for a, f, _ in done]) * 1e3
        span = max(f.t_done for _, f, _ in done) - min(a for a, _, _ in done)
        serving[name] = dict(p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                             requests_per_s=len(done) / span, samples_per_s=(s1 - s0) / span)
    serving = dict(rate_per_s=rate, requests=requests, slicemaps=len(vols), **serving)
    del pipe, vols, plain
    torch.cuda.empty_cache()
    return dict(batched_render=batch, serving=serving)


def run_batch(args, wl):
    """The batched workload (replicas only for N > 1, like the single-volume path)."""
    import torch
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    if ws > 1:
        torch.distributed.barrier()
    import phantom
    import paper_2311_15038_gb300 as mctp
    from paper_2311_15038_gb300 import batch as bt
    from paper_2311_15038_gb300 import pipeline as pl
    mctp._lib.load()

    specs = wl["specs"]
    vols = []
    for sp in specs:
        v = torch.empty(sp.shape, dtype=torch.uint8, device=dev)
        phantom.generate_gpu(sp, v)
        vols.append(v)
    lut = torch.from_numpy(phantom.ramp_lut(256)).to(dev)
    views = pl.turntable(wl["nviews"], wl["size"], 0, 0.5, wl["elevation"], wl["az_step"])
    stream = torch.cuda.Stream(dev)
    items = [bt.BatchItem(v, 8, views, 0) for v in vols]
    pipe = bt.BatchPipeline(items, wl["level0"], wl["nlevels"], lut, wl["nbins"], "otsu", 0.99, device=dev,
                            stream=stream)
    best, tune_ms = pipe.autotune(reps=2)
    torch.cuda.synchronize(dev)

    # ---- the plain per-volume and per-view launches on the same slicemaps; the
    # batched images must equal them bit for bit
    n_views = len(pipe.views)
    total = pipe.images.numel()
    plain = torch.empty_like(pipe.images)
    plain_samples = torch.empty(1, dtype=torch.uint64, device=dev)
    per_vol_samples = [torch.empty(1, dtype=torch.uint64, device=dev) for _ in items]
    per_view_samples = [torch.empty(1, dtype=torch.uint64, device=dev) for _ in range(n_views)]
    px = wl["size"] * wl["size"] * 4

    def per_volume():
        for i, sm in enumerate(pipe.slicemaps):
            o = plain[i * len(views) * px:(i + 1) * len(views) * px]
            mctp.render_views(sm, views, lut, 0.99, o, per_vol_samples[i], stream)

    def per_view():
        for j in range(n_views):
            sm = pipe.slicemaps[pipe.view_slicemap[j]]
            mctp.render_views(sm, [pipe.views[j]], lut, 0.99, plain[j * px:(j + 1) * px], per_view_samples[j],
                              stream)

    def batched():
        pipe.render()

    def timed(fn, reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            fn()
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps / 1e3

    t_batched = timed(batched, 3)
    samples_per_step = int(pipe.samples.item())
    with torch.cuda.stream(stream):
        mctp.render_batch(pipe.slicemaps, pipe.views, pipe.view_slicemap, pipe.view_lut, pipe.luts, 0.99,
                          dataclasses.replace(pipe.tuning, count_evaluated=True), pipe.images, pipe.samples,
                          pipe.workspace, stream)
    evaluated_per_step = mctp.batch_samples_evaluated(pipe.workspace)
    ref_images = pipe.images.clone()
    t_per_volume = timed(per_volume, 3)
    torch.cuda.synchronize(dev)
    assert torch.equal(plain[:total], ref_images[:total]), "batched images differ from per-volume launches"
    assert sum(int(s.item()) for s in per_vol_samples) == samples_per_step
    t_per_view = timed(per_view, 3)
    torch.cuda.synchronize(dev)
    assert torch.equal(plain[:total], ref_images[:total]), "batched images differ from per-view launches"
    assert sum(int(s.item()) for s in per_view_samples) == samples_per_step

    # ---- stage split from one eager pass, then the graph
    ev = {}

    def timer(name):
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        ev.setdefault(name, []).append(e)

    with torch.cuda.stream(stream):
        pipe.run(timer)
    torch.cuda.synchronize(dev)
    stage_ms = dict(prepare=ev["prepare"][0].elapsed_time(ev["render"][0]),
                    render=ev["render"][0].elapsed_time(ev["end"][0]))
    pipe.capture()
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            pipe.replay()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    step_events = []
    t0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pipe.replay()
            b.record(stream)
            step_events.append((a, b))
    t1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    elapsed = t0.elapsed_time(t1) / 1e3
    assert int(pipe.samples.item()) == samples_per_step
    assert torch.equal(pipe.images, ref_images)
    elapsed = max_over_ranks(elapsed, ws, dev)
    step_ms = [a.elapsed_time(b) for a, b in step_events]

    # ---- end to end: every volume from pinned host memory, every image back
    vol_bytes = sum(sp.nbytes for sp in specs)
    hosts = []
    for v in vols:
        h = torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
        h.copy_(v)
        hosts.append(h)
    img_host = torch.empty(pipe.images.shape, dtype=torch.float32, pin_memory=True)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(e2e_steps):
            for v, h in zip(vols, hosts):
                v.copy_(h, non_blocking=True)
            pipe.replay()
            img_host.copy_(pipe.images, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_s = e0.elapsed_time(e1) / 1e3 / e2e_steps
    del hosts
    e2e_s = max_over_ranks(e2e_s, ws, dev)
    if rank != 0:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
        return 0

    pk = peaks()
    fp32 = fp32_peak(pk, dev)
    atlas_bytes = sum(sm.nbytes for sm in pipe.slicemaps)
    prep_bytes = 2 * vol_bytes + atlas_bytes   # histogram read + slicemap read + atlas writes
    render_s = stage_ms["render"] / 1e3
    ach = FP32_FLOPS_PER_SAMPLE * evaluated_per_step / render_s / 1e12
    roof = dict(bound="alu", achieved=ach, peak=fp32, unit="TFLOP/s", frac=ach / fp32, kernel="render",
                ms=stage_ms["render"], traffic=None, peak_source=FP32_PEAK_SOURCE, flops_source=FLOPS_SOURCE,
                evaluated_samples_per_s=evaluated_per_step / render_s)
    value = job_rate(samples_per_step, args.steps, ws, elapsed)
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps, warmup=args.warmup,
        ms_per_step=elapsed * 1e3 / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="u8/f32", data="synthetic",
        config=dict(workload=wl["desc"], l2="inputs larger than L2 (%.1f GB of volumes; no flush)" % (vol_bytes / 1e9),
                    parallelism=f"replicas x{ws}", tuning=dict(warp_w=best.warp_w, chunk=best.chunk,
                                                               ctas_per_sm=best.ctas_per_sm)),
        samples_per_step=samples_per_step, samples_evaluated_per_step=evaluated_per_step,
        stage_ms=stage_ms,
        prepare_gbs=prep_bytes / (stage_ms["prepare"] / 1e3) / 1e9,
        prepare_frac_of_hbm_peak=prep_bytes / (stage_ms["prepare"] / 1e3) / 1e9 / pk["hbm_gbs"],
        render_samples_per_s=dict(batched=samples_per_step / t_batched, per_volume=samples_per_step / t_per_volume,
                                  per_view=samples_per_step / t_per_view),
        render_ms=dict(batched=t_batched * 1e3, per_volume=t_per_volume * 1e3, per_view=t_per_view * 1e3),
        batched_equals_plain=True,
        autotune_ms={f"w{t.warp_w}c{t.chunk}k{t.ctas_per_sm}": ms for t, ms in tune_ms.items()},
        latency_ms=dict(p50=float(np.percentile(step_ms, 50)), p99=float(np.percentile(step_ms, 99))),
        roofline=roof,
        gpu_launches=batch_launches_per_step(len(items), n_views) * args.steps,
        clocks=dict(sm_mhz=clk.get("sm_mhz"), sm_max_mhz=clk.get("sm_max_mhz"), reasons=clk.get("reasons")),
        e2e=dict(value=samples_per_step / e2e_s, unit=UNIT, h2d_bytes_per_step=vol_bytes,
                 d2h_bytes_per_step=pipe.images.numel() * 4, ms_per_step=e2e_s * 1e3),
    )
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        sp = specs[0]
        wl0 = dict(wl, spec=sp)
        nz_s = min(sp.nz, 96)
        zs = sp.nz // 2 - nz_s // 2
        step_s, samples_step, text = oracle_sample(wl0, vols[0][zs:zs + nz_s].cpu().numpy(), npix=65536)
        line["cpu_baseline"] = dict(value=samples_step / step_s, unit=UNIT, cores=1, host_cpus=os.cpu_count(),
                                    kind="oracle", extrapolated="from a 96-slice slab and 65536 rays to the step",
                                    sample="volume 0 of the batch: " + text)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def run_thresholds(args, wl):
    """Fig. 5 analogue: threshold selection times (GPU and host oracle) and results."""
    import torch
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import phantom
    import paper_2311_15038_gb300 as mctp
    oracle.build()
    stream = torch.cuda.current_stream(dev)

    def gpu_ms(fn, reps=50):
        fn()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps

    def cpu_ms(fn, reps=200):
        t0 = time.perf_counter()
        for _ in range(reps):
            out = fn()
        return (time.perf_counter() - t0) * 1e3 / reps, out

    rows = []
    total_bytes = 0
    total_hist_s = 0.0
    for label, sp in zip("ABCDE", wl["specs"]):
        vol = torch.empty(sp.shape, dtype=torch.uint8, device=dev)
        phantom.generate_gpu(sp, vol)
        row = dict(dataset=label, dims=[sp.nx, sp.ny, sp.nz], gbytes=sp.nbytes / 1e9)
        for stage in ("raw", "container_removed"):
            if stage == "container_removed":
                n = min(sp.nx, sp.ny)
                found = mctp.find_container(vol, 8, 0, 40, n // 8, n // 2, max(4, n // 32))
                mctp.mask_container(vol, 8, found["circle"], 2, out=vol)
                row["container_circle"] = [int(v) for v in found["circle"].cpu().tolist()]
            hist = torch.empty(256, dtype=torch.uint64, device=dev)
            ov = torch.empty(1, dtype=torch.uint64, device=dev)
            h_ms = gpu_ms(lambda: mctp.build_histogram(vol, 8, 256, hist=hist, overflow=ov), reps=5)
            total_hist_s += h_ms / 1e3
            total_bytes += sp.nbytes
            keep = torch.empty(256, dtype=torch.uint8, device=dev)
            res = torch.empty(4, dtype=torch.int32, device=dev)
            otsu_ms = gpu_ms(lambda: mctp.select_threshold(hist, 256, "otsu", keep=keep, result=res))
            T_otsu = int(res[0].item())
            its_ms = gpu_ms(lambda: mctp.select_threshold(hist, 256, "its", keep=keep, result=res))
            T_its, its_iters = int(res[0].item()), int(res[1].item())
            h_np = hist.cpu().numpy()
            o_ms, (To, _) = cpu_ms(lambda: oracle.otsu(h_np))
            i_ms, (Ti, it_i, conv, _) = cpu_ms(lambda: oracle.its(h_np))
            assert To == T_otsu and Ti == T_its
            row[stage] = dict(histogram_ms=h_ms, histogram_gbs=sp.nbytes / (h_ms / 1e3) / 1e9,
                              otsu=dict(T=T_otsu, gpu_ms=otsu_ms, host_oracle_ms=o_ms),
                              its=dict(T=T_its, iterations=its_iters, gpu_ms=its_ms, host_oracle_ms=i_ms))
        rows.append(row)
        del vol
        torch.cuda.empty_cache()
    pk = peaks()
    gbs = total_bytes / total_hist_s / 1e9
    sp0 = wl["specs"][0]
    slab = phantom.generate_cpu(sp0, ((0, sp0.nx), (0, sp0.ny), (0, 256)))
    t0 = time.perf_counter()
    oracle.histogram(slab, 8, 256)
    t_orc = time.perf_counter() - t0
    line = dict(metric=METRIC, value=gbs, unit="histogram GB/s", n_gpus=1, steps=1,
                warmup=1, ms_per_step=total_hist_s * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="u8", data="synthetic", config=dict(workload=wl["desc"]), thresholds=rows,
                roofline=dict(bound="hbm", achieved=gbs, peak=pk["hbm_gbs"], unit="GB/s", frac=gbs / pk["hbm_gbs"],
                              kernel="hist_lane_kernel", traffic=None, peak_source=pk["source"]),
                cpu_baseline=dict(value=slab.nbytes / t_orc / 1e9, unit="histogram GB/s", cores=1, kind="oracle",
                                  sample=f"oracle histogram (C, 1 thread) of 256 slices of dataset A ({slab.nbytes / 1e6:.0f} MB)"),
                note="Fig. 5 analogue: Otsu sweeps all 256 bins, ITS stops once converged; times per selection")
    print(json.dumps(line), flush=True)
    return 0


def fit_oracle_baseline(fit, view, src_dims):
    """The oracle's forward render and FP64 gradient of the fitted volume on one
    128 x 128 view of the same geometry; samples of the forward per second of
    (forward + gradient), the unit of the fit workload's value."""
    import oracle
    oracle.build()
    vol = fit.vol.double().cpu().numpy()
    lut = fit.lut.double().cpu().numpy()
    w = h = 128
    t0 = time.perf_counter()
    _, ns = oracle.render_dense(vol, src_dims, lut, view.azimuth_deg, view.elevation_deg, w, h, view.step, 0.99)
    g = np.ones((h, w, 4))
    oracle.render_dense_grad(vol, src_dims, lut, view.azimuth_deg, view.elevation_deg, w, h, g, view.step, 0.99)
    dt = time.perf_counter() - t0
    return dict(value=float(ns.sum()) / dt, unit=UNIT, cores=1, kind="oracle",
                sample=f"oracle (C, 1 thread) FP64 forward + reverse-mode gradient of one 128x128 view "
                       f"({int(ns.sum())} samples) of the fitted 128^3 volume, {dt:.1f} s")


def run_fit(args, wl):
    """The differentiable workload: Adam iterations fitting a 128^3 volume and its LUT."""
    import torch
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    if ws > 1:
        torch.distributed.barrier()
    import phantom
    import paper_2311_15038_gb300 as mctp
    from paper_2311_15038_gb300 import diff
    from paper_2311_15038_gb300 import pipeline as pl
    mctp._lib.load()

    spec = wl["spec"]
    vol = torch.empty(spec.shape, dtype=torch.uint8, device=dev)
    phantom.generate_gpu(spec, vol)
    h, _ = mctp.build_histogram(vol, 8, 256)
    keep, _ = mctp.select_threshold(h, 256)
    sm = mctp.Slicemap.allocate((spec.nx, spec.ny, spec.nz), wl["level0"], wl["nlevels"], torch.uint8, 8, dev)
    mctp.build_slicemap(vol, 8, sm, keep)
    lut = torch.from_numpy(phantom.preset_luts()[5]).to(dev)
    n = wl["nviews"]
    views = [mctp.View(wl["az_step"] * k, wl["elevation"] if k % 2 == 0 else -wl["elevation"], wl["size"],
                       wl["size"], 0, 0.5) for k in range(n)]
    targets, _ = mctp.render_views(sm, views, lut, 0.99)
    # start: the coarsest level (128^3) as intensities
    k = wl["nlevels"] - 1
    mx, my, mz = sm.dims[k]
    tx, ty = sm.tiles[k]
    start = (sm.atlases[k].view(ty, my, tx, mx).permute(0, 2, 1, 3).reshape(ty * tx, my, mx)[:mz]
             .float().div_(255.0).contiguous())
    fviews = [mctp.View(v.azimuth_deg, v.elevation_deg, v.width, v.height, 0, 0.5) for v in views]
    stream = torch.cuda.Stream(dev)
    fit = diff.Fitter(start, lut, fviews, (spec.nx, spec.ny, spec.nz), targets, 0.99, 1e-2, 5e-3, stream)
    torch.cuda.synchronize(dev)
    loss0 = fit.evaluate()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            fit.step()
    torch.cuda.synchronize(dev)
    samples_fwd = int(fit.samples.item())
    # per-stage times of one iteration
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    s = stream
    with torch.cuda.stream(s):
        ev[0].record(s)
        diff.render_dense(fit.vol, fit.lut, fviews, fit.src_dims, 0.99, fit.images, fit.samples, s)
        ev[1].record(s)
        diff.l2_loss(fit.images, fit.targets, fit.scale, fit.g_img, fit.loss, s)
        ev[2].record(s)
        diff.render_dense_backward(fit.vol, fit.lut, fviews, fit.src_dims, fit.g_img, 0.99, fit.g_vol, fit.g_lut, s)
        ev[3].record(s)
        diff.adam_step(fit.vol, fit.g_vol, fit.m_vol, fit.v_vol, fit.t + 1, 0.0, lo=0.0, hi=1.0, stream=s)
        diff.adam_step(fit.lut, fit.g_lut, fit.m_lut, fit.v_lut, fit.t + 1, 0.0, lo=0.0, hi=1.0, stream=s)
        ev[4].record(s)
    torch.cuda.synchronize(dev)
    stage_ms = dict(forward=ev[0].elapsed_time(ev[1]), loss=ev[1].elapsed_time(ev[2]),
                    adjoint=ev[2].elapsed_time(ev[3]), adam=ev[3].elapsed_time(ev[4]))
    clocks = ClockSampler(local)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s)
    with torch.cuda.stream(s):
        for _ in range(args.steps):
            fit.step()
    t1.record(s)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    elapsed = t0.elapsed_time(t1) / 1e3
    # end to end: each iteration's loss read back to pinned host memory
    loss_host = torch.empty(1, dtype=torch.float32, pin_memory=True)
    e2e_steps = max(1, min(args.steps, 10))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    with torch.cuda.stream(s):
        for _ in range(e2e_steps):
            fit.step()
            loss_host.copy_(fit.loss, non_blocking=True)
    e1.record(s)
    torch.cuda.synchronize(dev)
    e2e_s = e0.elapsed_time(e1) / 1e3 / e2e_steps
    loss1 = fit.evaluate()
    elapsed = max_over_ranks(elapsed, ws, dev)

    def psnr(loss):  # loss = mean squared error over RGBA
        return float(10.0 * np.log10(1.0 / max(loss, 1e-30)))

    if rank != 0:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
        return 0
    pk = peaks()
    fp32 = fp32_peak(pk, dev)
    it_s = elapsed / args.steps
    ach = FP32_FLOPS_PER_SAMPLE * samples_fwd / (stage_ms["forward"] / 1e3) / 1e12
    line = dict(
        metric=METRIC, value=job_rate(samples_fwd, args.steps, ws, elapsed), unit=UNIT, n_gpus=ws, steps=args.steps,
        warmup=args.warmup, ms_per_step=it_s * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="f32", data="synthetic",
        config=dict(workload=wl["desc"], l2="fitted volume 8.4 MB (L2-resident); targets 100 MB",
                    parallelism=f"replicas x{ws}"),
        samples_per_step=samples_fwd,
        stage_ms=stage_ms,
        forward_samples_per_s=samples_fwd / (stage_ms["forward"] / 1e3),
        adjoint_samples_per_s=samples_fwd / (stage_ms["adjoint"] / 1e3),
        loss=dict(start=loss0, end=loss1, iterations=args.warmup + args.steps + e2e_steps, psnr_start_db=psnr(loss0),
                  psnr_end_db=psnr(loss1)),
        roofline=dict(bound="alu", achieved=ach, peak=fp32, unit="TFLOP/s", frac=ach / fp32,
                      kernel="dense_forward_kernel", traffic=None, peak_source=FP32_PEAK_SOURCE,
                      flops_source=FLOPS_SOURCE),
        cpu_baseline=fit_oracle_baseline(fit, fviews[0], (spec.nx, spec.ny, spec.nz)),
        gpu_launches=5 * args.steps,
        clocks=dict(sm_mhz=clk.get("sm_mhz"), sm_max_mhz=clk.get("sm_max_mhz"), reasons=clk.get("reasons")),
        e2e=dict(value=samples_fwd / e2e_s, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=4,
                 ms_per_step=e2e_s * 1e3, note="targets and parameters stay resident; every iteration's loss is "
                                                "copied to pinned host memory"),
    )
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def serve_oracle_baseline(sm, lut):
    """The oracle render of 32768 rays of one 512 x 512 request on a resident slicemap."""
    import oracle
    oracle.build()
    mx, my, mz = sm.dims[0]
    tx, ty = sm.tiles[0]
    level = sm.atlases[0].view(ty, my, tx, mx).permute(0, 2, 1, 3).reshape(ty * tx, my, mx)[:mz].cpu().numpy()
    rng = np.random.default_rng(0)
    pix = rng.integers(0, 512 * 512, size=32768)
    t0 = time.perf_counter()
    ref = oracle.render(level, 8, sm.src_dims, lut.cpu().numpy(), 40.0, 20.0, 512, 512, 0.5, 0.99, 0.0, pixels=pix)
    dt = time.perf_counter() - t0
    ns = float(ref["nsamp"][:, 1].sum())
    return dict(value=ns / dt, unit=UNIT, cores=1, kind="oracle",
                sample=f"oracle (C, 1 thread) render of 32768 random rays of a 512x512 view of slicemap 0 "
                       f"({int(ns)} samples, {dt:.1f} s)")


def run_serve(args, wl):
    """The serving workload: rate sweep, batched server against per-view launches."""
    import torch
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    if ws > 1:
        torch.distributed.barrier()
    import phantom
    import paper_2311_15038_gb300 as mctp
    from paper_2311_15038_gb300 import serve as sv
    mctp._lib.load()

    vols, sms = [], []
    for sp in wl["specs"]:
        v = torch.empty(sp.shape, dtype=torch.uint8, device=dev)
        phantom.generate_gpu(sp, v)
        h, _ = mctp.build_histogram(v, 8, 256)
        keep, _ = mctp.select_threshold(h, 256)
        sm = mctp.Slicemap.allocate((sp.nx, sp.ny, sp.nz), wl["level0"], wl["nlevels"], torch.uint8, 8, dev)
        mctp.build_slicemap(v, 8, sm, keep)
        sm.make_textures()  # the batched server gathers corner quads through atlas textures
        sm.update_textures()
        vols.append(v)
        sms.append(sm)
    luts = torch.from_numpy(np.stack(phantom.preset_luts())).to(dev)
    torch.cuda.synchronize(dev)
    arena = 8 << 30
    configs = {"per_view": dict(mode="per_view", max_batch_views=1, max_inflight=1),
               "batched": dict(mode="batched", max_batch_views=64, max_inflight=2)}
    results = {}
    clocks = ClockSampler(local)
    clocks.start()
    for name, cfg in configs.items():
        srv = sv.Server(sms, luts, arena, **cfg)
        try:
            warm = sv.poisson_trace(2000.0, 200, len(sms), luts.shape[0], seed=99)
            sv.run_trace(srv, warm)
            per_rate = {}
            for k, rate in enumerate(wl["rates"]):
                trace = sv.poisson_trace(rate, wl["requests"], len(sms), luts.shape[0], seed=1 + k)
                s0 = srv.stats()["samples"]
                done = sv.run_trace(srv, trace)
                s1 = srv.stats()["samples"]
                lat = np.array([f.t_done - a for a, f, _ in done]) * 1e3
                t_first = min(a for a, _, _ in done)
                t_last = max(f.t_done for _, f, _ in done)
                per_rate[rate] = dict(p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                                      samples_per_s=(s1 - s0) / (t_last - t_first),
                                      requests_per_s=len(done) / (t_last - t_first))
            st = srv.stats()
            per_rate["launches"] = st["launches"]
            per_rate["arena_high_water_bytes"] = st["arena_high_water"]
            results[name] = per_rate
        finally:
            srv.close()
    clk = clocks.stop()
    # end to end: the batched server at the top rate with every image copied to pinned host memory
    srv = sv.Server(sms, luts, arena, **configs["batched"])
    try:
        top = wl["rates"][-1]
        trace = sv.poisson_trace(top, wl["requests"], len(sms), luts.shape[0], seed=77)
        s0 = srv.stats()["samples"]
        done = sv.run_trace(srv, trace, copy_to_host=True)
        s1 = srv.stats()["samples"]
        t_first = min(a for a, _, _ in done)
        t_last = max(tc for _, _, tc in done)
        e2e_lat = np.array([tc - a for a, _, tc in done]) * 1e3
        d2h = sum(a.view.width * a.view.height * 16 for a in trace)
        e2e = dict(value=(s1 - s0) / (t_last - t_first), unit=UNIT, h2d_bytes_per_step=0,
                   d2h_bytes_per_step=d2h, p50_ms=float(np.percentile(e2e_lat, 50)),
                   p99_ms=float(np.percentile(e2e_lat, 99)), requests=len(done))
    finally:
        srv.close()
    if rank != 0:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
        return 0
    top = wl["rates"][-1]
    b, p = results["batched"][top], results["per_view"][top]
    pk = peaks()
    # share of taken samples that are evaluated (not skipped as empty), from one counted
    # batch of the top rate's first 256 requests
    probe = sv.poisson_trace(top, 256, len(sms), luts.shape[0], seed=len(wl["rates"]))
    pv = [a.view for a in probe]
    pvs = [a.slicemap for a in probe]
    pvl = [a.lut for a in probe]
    _, psamp, pws = mctp.render_batch(sms, pv, pvs, pvl, luts, 0.99, mctp.BatchTuning(count_evaluated=True))
    eval_share = mctp.batch_samples_evaluated(pws) / max(int(psamp.item()), 1)
    del pws
    line = dict(
        metric=METRIC, value=b["samples_per_s"] * ws, unit=UNIT, n_gpus=ws, steps=len(wl["rates"]),
        warmup=1, ms_per_step=None, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="u8/f32",
        data="synthetic",
        config=dict(workload=wl["desc"], l2="resident slicemaps 3.8 GB > L2; requests read them in place",
                    parallelism=f"replicas x{ws}", server=configs["batched"], baseline=configs["per_view"],
                    requests_per_rate=wl["requests"], rates_per_s=list(wl["rates"])),
        latency_ms=dict(p50=b["p50_ms"], p99=b["p99_ms"]),
        per_view_latency_ms=dict(p50=p["p50_ms"], p99=p["p99_ms"]),
        serving=results,
        roofline=dict(bound="alu", achieved=FP32_FLOPS_PER_SAMPLE * eval_share * b["samples_per_s"] / 1e12,
                      peak=fp32_peak(pk, dev), unit="TFLOP/s", peak_source=FP32_PEAK_SOURCE, flops_source=FLOPS_SOURCE,
                      frac=FP32_FLOPS_PER_SAMPLE * eval_share * b["samples_per_s"] / 1e12 / fp32_peak(pk, dev),
                      kernel="render_batch_kernel", traffic=None, evaluated_share=eval_share,
                      note="evaluated samples/s over the wall time of the top rate, so idle gaps count against it; "
                           "the evaluated share is from one counted batch of 256 requests of that rate"),
        cpu_baseline=serve_oracle_baseline(sms[0], luts[0]),
        gpu_launches=None,
        clocks=dict(sm_mhz=clk.get("sm_mhz"), sm_max_mhz=clk.get("sm_max_mhz"), reasons=clk.get("reasons")),
        e2e=e2e,
        peak_source=pk["source"],
    )
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mctp", choices=["mctp", "reference"])
    ap.add_argument("--workload", default="full",
                    choices=["full", "mid", "slab", "small", "batch", "batch8", "serve", "fit", "thresholds"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-next-rows", action="store_true",
                    help="skip the batched-render and serving sub-record of the full workload's line")
    ap.add_argument("--render-tuning", default=None, metavar="WARP_W,CHUNK,CTAS",
                    help="fixed launch shape of the work-queue renderer (default: autotuned after warm-up)")
    args = ap.parse_args()
    wl = workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, wl)
    if args.workload in ("batch", "batch8"):
        return run_batch(args, wl)
    if args.workload == "serve":
        return run_serve(args, wl)
    if args.workload == "fit":
        return run_fit(args, wl)
    if args.workload == "thresholds":
        return run_thresholds(args, wl)
    return run_gpu(args, wl)


if __name__ == "__main__":
    sys.exit(main())
