"""Differentiable rendering of a reduced FP32 volume and a transfer function
(include/mctp.h: mctp_render_dense, mctp_render_dense_backward, mctp_l2_loss,
mctp_adam_step), a torch.autograd.Function over them, and a fitter that
adjusts the reduced volume and the LUT so that their renders match target
images of the full-resolution source.  Marshalling only: the forward march,
the adjoint march, the loss and the optimiser step all run in libmctp."""
from __future__ import annotations

import ctypes

import torch

from . import _cuda, _lib, _out, _ptr, _stream, view_array


def _dims(vol: torch.Tensor):
    _cuda(vol, "vol")
    if vol.dim() != 3 or vol.dtype != torch.float32:
        raise ValueError("vol must be a float32 [mz][my][mx] tensor")
    mz, my, mx = vol.shape
    return mx, my, mz


def _lut(lut: torch.Tensor) -> torch.Tensor:
    _cuda(lut, "lut")
    if lut.dtype != torch.float32 or lut.dim() != 2 or lut.shape[1] != 4:
        raise ValueError("lut must be float32 [n][4]")
    return lut


def _src(src_dims):
    return (ctypes.c_int64 * 3)(*[int(v) for v in src_dims])


def render_dense(vol: torch.Tensor, lut: torch.Tensor, views, src_dims, alpha_stop: float = 0.99,
                 out: torch.Tensor | None = None, samples: torch.Tensor | None = None, stream=None):
    """Images of the dense intensity volume -> (flat float32 RGBA, samples uint64[1])."""
    mx, my, mz = _dims(vol)
    _lut(lut)
    total = sum(v.width * v.height * 4 for v in views)
    if out is None:
        out = torch.empty(max(total, 4), dtype=torch.float32, device=vol.device)
    if samples is None:
        samples = torch.empty(1, dtype=torch.uint64, device=vol.device)
    _out(out, "out", torch.float32, total, vol.device)
    _out(samples, "samples", torch.uint64, 1, vol.device)
    _lib.check(_lib.load().mctp_render_dense(_ptr(vol), mx, my, mz, _src(src_dims), view_array(views), len(views),
                                             _ptr(lut), lut.shape[0], alpha_stop, _ptr(out), _ptr(samples),
                                             _stream(stream)), "mctp_render_dense")
    return out, samples


def render_dense_backward(vol: torch.Tensor, lut: torch.Tensor, views, src_dims, grad_rgba: torch.Tensor,
                          alpha_stop: float = 0.99, grad_vol: torch.Tensor | None = None,
                          grad_lut: torch.Tensor | None = None, stream=None):
    """(dL/dvol, dL/dlut) given dL/d(images) (the flat buffer of render_dense)."""
    mx, my, mz = _dims(vol)
    _lut(lut)
    _out(grad_rgba, "grad_rgba", torch.float32, sum(v.width * v.height * 4 for v in views), vol.device)
    if grad_vol is None:
        grad_vol = torch.empty_like(vol)
    if grad_lut is None:
        grad_lut = torch.empty_like(lut)
    _out(grad_vol, "grad_vol", torch.float32, vol.numel(), vol.device)
    _out(grad_lut, "grad_lut", torch.float32, lut.numel(), vol.device)
    _lib.check(_lib.load().mctp_render_dense_backward(_ptr(vol), mx, my, mz, _src(src_dims), view_array(views),
                                                      len(views), _ptr(lut), lut.shape[0], alpha_stop,
                                                      _ptr(grad_rgba), _ptr(grad_vol), _ptr(grad_lut),
                                                      _stream(stream)), "mctp_render_dense_backward")
    return grad_vol, grad_lut


class DenseRender(torch.autograd.Function):
    """images = DenseRender.apply(vol, lut, views, src_dims, alpha_stop); differentiable in vol and lut."""

    @staticmethod
    def forward(ctx, vol, lut, views, src_dims, alpha_stop):
        vol, lut = vol.contiguous(), lut.contiguous()
        out, _ = render_dense(vol, lut, views, src_dims, alpha_stop)
        ctx.save_for_backward(vol, lut)
        ctx.views, ctx.src_dims, ctx.alpha_stop = views, src_dims, alpha_stop
        return out

    @staticmethod
    def backward(ctx, grad_out):
        vol, lut = ctx.saved_tensors
        gv, gl = render_dense_backward(vol, lut, ctx.views, ctx.src_dims, grad_out.contiguous(), ctx.alpha_stop)
        return gv, gl, None, None, None


def l2_loss(x: torch.Tensor, target: torch.Tensor, scale: float = 1.0, grad: torch.Tensor | None = None,
            loss: torch.Tensor | None = None, stream=None):
    """(loss float32[1] = scale sum (x - t)^2, grad = 2 scale (x - t))."""
    _cuda(x, "x")
    _out(target, "target", x.dtype, x.numel(), x.device)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
    _out(loss, "loss", torch.float32, 1, x.device)
    if grad is not None:
        _out(grad, "grad", torch.float32, x.numel(), x.device)
    _lib.check(_lib.load().mctp_l2_loss(_ptr(x), _ptr(target), x.numel(), scale, _ptr(grad), _ptr(loss),
                                        _stream(stream)), "mctp_l2_loss")
    return loss, grad


def adam_step(param: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, step: int, lr: float,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, lo: float = -3.4e38, hi: float = 3.4e38,
              stream=None) -> None:
    _cuda(param, "param")
    for t, name in ((grad, "grad"), (m, "m"), (v, "v")):
        _out(t, name, param.dtype, param.numel(), param.device)
    _lib.check(_lib.load().mctp_adam_step(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), lr, beta1, beta2,
                                          eps, step, lo, hi, _stream(stream)), "mctp_adam_step")


class Fitter:
    """Adam on a reduced volume (intensities in [0, 1]) and a transfer function
    (entries in [0, 1]) so that render_dense matches target images."""

    def __init__(self, vol0: torch.Tensor, lut0: torch.Tensor, views, src_dims, targets: torch.Tensor,
                 alpha_stop: float = 0.99, lr_vol: float = 1e-2, lr_lut: float = 5e-3, stream=None):
        self.vol = vol0.clone().contiguous()
        self.lut = lut0.clone().contiguous()
        self.views, self.src_dims, self.alpha_stop = views, src_dims, alpha_stop
        self.targets = targets
        self.lr_vol, self.lr_lut = lr_vol, lr_lut
        self.stream = stream
        dev = vol0.device
        self.m_vol, self.v_vol = torch.zeros_like(self.vol), torch.zeros_like(self.vol)
        self.m_lut, self.v_lut = torch.zeros_like(self.lut), torch.zeros_like(self.lut)
        self.g_vol, self.g_lut = torch.empty_like(self.vol), torch.empty_like(self.lut)
        self.images = torch.empty_like(targets)
        self.g_img = torch.empty_like(targets)
        self.loss = torch.empty(1, dtype=torch.float32, device=dev)
        self.samples = torch.empty(1, dtype=torch.uint64, device=dev)
        self.scale = 1.0 / targets.numel()
        self.t = 0

    def step(self) -> None:
        """One iteration (enqueued): forward, loss + its gradient, adjoint, two Adam steps."""
        s = self.stream
        render_dense(self.vol, self.lut, self.views, self.src_dims, self.alpha_stop, self.images, self.samples, s)
        l2_loss(self.images, self.targets, self.scale, self.g_img, self.loss, s)
        render_dense_backward(self.vol, self.lut, self.views, self.src_dims, self.g_img, self.alpha_stop,
                              self.g_vol, self.g_lut, s)
        self.t += 1
        adam_step(self.vol, self.g_vol, self.m_vol, self.v_vol, self.t, self.lr_vol, lo=0.0, hi=1.0, stream=s)
        adam_step(self.lut, self.g_lut, self.m_lut, self.v_lut, self.t, self.lr_lut, lo=0.0, hi=1.0, stream=s)

    _STATE = ("vol", "lut", "m_vol", "v_vol", "m_lut", "v_lut")

    def state_dict(self) -> dict:
        """Everything a resumed fit needs: the reduced volume, the transfer
        function, both Adam moment pairs, the step count and the settings
        (copies on the host; the caller saves them, e.g. with torch.save).
        Waits for the fit's queued work first."""
        if self.stream is not None:
            self.stream.synchronize()
        elif self.vol.is_cuda:
            torch.cuda.synchronize(self.vol.device)
        out = {k: getattr(self, k).detach().cpu().clone() for k in self._STATE}
        out.update(t=self.t, lr_vol=self.lr_vol, lr_lut=self.lr_lut, alpha_stop=self.alpha_stop,
                   src_dims=tuple(int(v) for v in self.src_dims),
                   views=[(v.azimuth_deg, v.elevation_deg, v.width, v.height, v.level, v.step) for v in self.views])
        return out

    def load_state_dict(self, state: dict) -> None:
        """Continue a fit from state_dict(): the same views, source and shapes
        are required (checked), after which the next step() is the step the
        saved fit would have taken."""
        views = [(v.azimuth_deg, v.elevation_deg, v.width, v.height, v.level, v.step) for v in self.views]
        if [tuple(v) for v in state["views"]] != views or tuple(state["src_dims"]) != tuple(self.src_dims):
            raise ValueError("the saved fit has other views or another source volume")
        for k in self._STATE:
            dst = getattr(self, k)
            src = state[k]
            if tuple(src.shape) != tuple(dst.shape) or src.dtype != dst.dtype:
                raise ValueError(f"saved {k} has shape {tuple(src.shape)} / {src.dtype}, "
                                 f"expected {tuple(dst.shape)} / {dst.dtype}")
            dst.copy_(src.to(dst.device))
        self.t = int(state["t"])
        self.lr_vol, self.lr_lut = float(state["lr_vol"]), float(state["lr_lut"])
        self.alpha_stop = float(state["alpha_stop"])

    def evaluate(self) -> float:
        """Loss of the current parameters (synchronises)."""
        render_dense(self.vol, self.lut, self.views, self.src_dims, self.alpha_stop, self.images, self.samples,
                     self.stream)
        l2_loss(self.images, self.targets, self.scale, None, self.loss, self.stream)
        if self.stream is not None:
            self.stream.synchronize()
        return float(self.loss.item())
