"""FP32 model of the renderers' ray set-up (render_common.cuh, march_ray), for
host-side checks: the camera basis rounded once from FP64, the ray origin, the
slab test against the source box and the sample count n, each operation
rounded to single precision in the kernel's order."""
import math

import numpy as np

F = np.float32


def basis(az_deg, el_deg):
    """Camera basis as the host sets it up: FP64, rounded once to float."""
    az, el = math.radians(az_deg), math.radians(el_deg)
    b = np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)], F)
    r = np.array([-math.sin(az), math.cos(az), 0.0], F)
    u = np.array([-math.sin(el) * math.cos(az), -math.sin(el) * math.sin(az), math.cos(el)], F)
    return b, r, u


def rays(N, M, az, el, W, H, step):
    """Per pixel: ray origin, t_min and sample count n in FP32 as the kernel
    computes them (slab test against the source box), plus the view data."""
    b, r, u = basis(az, el)
    Nf = N.astype(F)
    L = F(math.sqrt(float((N.astype(np.float64) ** 2).sum())))
    c = Nf / F(2)
    delta = F(step) * F(min(N[a] / M[a] for a in range(3)))
    py, px = np.mgrid[0:H, 0:W]
    sx = ((px.astype(F) + F(0.5)) / F(W) - F(0.5)).astype(F)
    sy = (F(0.5) - (py.astype(F) + F(0.5)) / F(H)).astype(F)
    sxL, syL = (sx * L).astype(F), (sy * L).astype(F)
    o = np.stack([(c[a] + sxL * r[a] + syL * u[a] + L * b[a]).astype(F) for a in range(3)], -1)
    d = -b
    tmin = np.full(sx.shape, -np.inf, F)
    tmax = np.full(sx.shape, np.inf, F)
    miss = np.zeros(sx.shape, bool)
    for a in range(3):
        if d[a] != 0:
            inv = F(1) / d[a]
            s0 = ((F(0) - o[..., a]) * inv).astype(F)
            s1 = ((Nf[a] - o[..., a]) * inv).astype(F)
            tmin = np.maximum(tmin, np.minimum(s0, s1))
            tmax = np.minimum(tmax, np.maximum(s0, s1))
        else:
            miss |= ~((o[..., a] >= 0) & (o[..., a] <= Nf[a]))
    with np.errstate(invalid="ignore"):
        n = np.where(~miss & (tmax > tmin), np.floor(((tmax - tmin) / delta).astype(F)), 0).astype(np.int64)
    return dict(o=o, d=d, tmin=tmin, n=n, delta=delta, L=L, c=c, b=b, r=r, u=u)
