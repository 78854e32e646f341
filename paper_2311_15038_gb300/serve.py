"""Python handle of the preview server (include/mctp.h, mctp_server_*):
resident slicemaps, requests admitted by free arena memory, continuous
batching of the admitted ones into render_batch launches on several streams.
Marshalling only; the dispatcher thread and all rendering live in libmctp."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import BatchTuning, Slicemap, View, _lib, _luts3, _ptr


@dataclass(frozen=True)
class Finished:
    ticket: int
    status: int
    image_ptr: int
    t_submit: float
    t_admit: float
    t_launch: float
    t_done: float

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


def now() -> float:
    """The server's clock (seconds, monotonic)."""
    return _lib.load().mctp_now()


class Server:
    """Keeps slicemaps and transfer functions; renders submitted views.

    mode "batched": continuous batching (up to max_batch_views per launch,
    max_inflight launches on the device); mode "per_view": one render_views
    launch per request in arrival order."""

    def __init__(self, slicemaps: list[Slicemap], luts: torch.Tensor, arena_bytes: int, mode: str = "batched",
                 max_batch_views: int = 64, max_inflight: int = 2, tuning: BatchTuning | None = None,
                 alpha_stop: float = 0.99):
        self.slicemaps = slicemaps
        self.luts = _luts3(luts)
        self.arena = torch.empty(arena_bytes, dtype=torch.uint8, device=self.luts.device)
        self._sms = (_lib.SlicemapDesc * len(slicemaps))(*[sm.desc() for sm in slicemaps])
        t = (tuning or BatchTuning()).c()
        m = _lib.MCTP_SERVE_BATCHED if mode == "batched" else _lib.MCTP_SERVE_PER_VIEW
        self._params = _lib.ServeParams(m, max_batch_views, max_inflight, 0, t)
        self._h = ctypes.c_void_p()
        self._lib = _lib.load()
        _lib.check(self._lib.mctp_server_create(self._sms, len(slicemaps), _ptr(self.luts), self.luts.shape[0],
                                                self.luts.shape[1], alpha_stop, _ptr(self.arena), arena_bytes,
                                                ctypes.byref(self._params), ctypes.byref(self._h)),
                   "mctp_server_create")
        self._res = (_lib.ServeResult * 256)()
        self._views = {}

    def submit(self, view: View, slicemap: int, lut: int = 0) -> int:
        v = _lib.ViewDesc(view.azimuth_deg, view.elevation_deg, view.width, view.height, view.level, view.step)
        tk = ctypes.c_uint64()
        _lib.check(self._lib.mctp_server_submit(self._h, ctypes.byref(v), slicemap, lut, ctypes.byref(tk)),
                   "mctp_server_submit")
        self._views[tk.value] = view
        return tk.value

    def poll(self) -> list[Finished]:
        out = []
        while True:
            n = _lib.C_I32()
            _lib.check(self._lib.mctp_server_poll(self._h, self._res, len(self._res), ctypes.byref(n)),
                       "mctp_server_poll")
            for i in range(n.value):
                r = self._res[i]
                out.append(Finished(r.ticket, r.status, r.image or 0, r.t_submit, r.t_admit, r.t_launch, r.t_done))
            if n.value < len(self._res):
                return out

    def image(self, f: Finished) -> torch.Tensor:
        """Copy of a finished request's image ([H][W][4] float32 on the device)."""
        v = self._views[f.ticket]
        off = f.image_ptr - self.arena.data_ptr()
        flat = self.arena[off:off + v.width * v.height * 16].view(torch.float32)
        return flat.view(v.height, v.width, 4).clone()

    def release(self, ticket: int) -> None:
        _lib.check(self._lib.mctp_server_release(self._h, ticket), "mctp_server_release")
        self._views.pop(ticket, None)

    def cancel(self, ticket: int) -> bool:
        """Cancel a request not launched yet; True if it was (poll then reports
        it with status MCTP_ECANCELED), False if it was already launched or done."""
        rc = self._lib.mctp_server_cancel(self._h, ticket)
        if rc not in (_lib.MCTP_OK, _lib.MCTP_EINVAL):
            _lib.check(rc, "mctp_server_cancel")
        return rc == _lib.MCTP_OK

    def inject_launch_failures(self, n: int) -> None:
        """Test hook: the next n launches fail on the host as a failed kernel
        launch would (no GPU fault); their requests finish with MCTP_ECUDA."""
        _lib.check(self._lib.mctp_server_inject_launch_failures(self._h, n), "mctp_server_inject_launch_failures")

    def stats(self) -> dict:
        s, l, h = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _lib.check(self._lib.mctp_server_stats(self._h, ctypes.byref(s), ctypes.byref(l), ctypes.byref(h)),
                   "mctp_server_stats")
        return dict(samples=s.value, launches=l.value, arena_high_water=h.value)

    def close(self) -> None:
        if self._h:
            _lib.check(self._lib.mctp_server_destroy(self._h), "mctp_server_destroy")
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


@dataclass(frozen=True)
class Arrival:
    t: float          # seconds after the start of the trace
    view: View
    slicemap: int
    lut: int


def poisson_trace(rate: float, n: int, nsm: int, nluts: int, sizes=(512, 1024), elev=(-60.0, 60.0),
                  level: int = 0, step: float = 0.5, seed: int = 0) -> list[Arrival]:
    """n requests with exponential inter-arrival times (rate per second): a
    random slicemap, square view size, azimuth U[0, 360), elevation U[elev],
    transfer function."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    for i in range(n):
        size = int(sizes[int(rng.integers(len(sizes)))])
        v = View(float(rng.uniform(0.0, 360.0)), float(rng.uniform(*elev)), size, size, level, step)
        out.append(Arrival(float(t[i]), v, int(rng.integers(nsm)), int(rng.integers(nluts))))
    return out


def run_trace(srv: Server, trace: list[Arrival], copy_to_host: bool = False, timeout: float = 120.0):
    """Submit each request at its arrival time, release finished images (after
    an asynchronous copy to pinned host memory when copy_to_host), and return
    [(scheduled arrival, Finished, copy done)] in completion order."""
    start = now() + 0.005
    sched = {}
    done = []
    i = 0
    stream = torch.cuda.Stream(srv.arena.device) if copy_to_host else None
    ring = []
    if copy_to_host:
        biggest = max(a.view.width * a.view.height * 16 for a in trace)
        ring = [torch.empty(biggest, dtype=torch.uint8, pin_memory=True) for _ in range(8)]
    inflight = []   # (event, Finished, ring index)
    free_ring = list(range(len(ring)))
    waiting = []    # finished, waiting for a ring slot
    while len(done) < len(trace):
        t = now()
        while i < len(trace) and start + trace[i].t <= t:
            a = trace[i]
            sched[srv.submit(a.view, a.slicemap, a.lut)] = start + a.t
            i += 1
        for f in srv.poll():
            if f.status != 0:
                raise RuntimeError(f"request {f.ticket} failed ({f.status})")
            if copy_to_host:
                waiting.append(f)
            else:
                srv.release(f.ticket)
                done.append((sched[f.ticket], f, f.t_done))
        while waiting and free_ring:
            f = waiting.pop(0)
            k = free_ring.pop()
            v = srv._views[f.ticket]
            nb = v.width * v.height * 16
            off = f.image_ptr - srv.arena.data_ptr()
            with torch.cuda.stream(stream):
                ring[k][:nb].copy_(srv.arena[off:off + nb], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(stream)
            inflight.append((ev, f, k))
        still = []
        for ev, f, k in inflight:
            if ev.query():
                tc = now()
                srv.release(f.ticket)
                free_ring.append(k)
                done.append((sched[f.ticket], f, tc))
            else:
                still.append((ev, f, k))
        inflight = still
        if now() - start > timeout:
            raise RuntimeError("trace did not finish in time")
    return done
