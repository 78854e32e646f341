"""Full-size parity on the 'full' workload (u16 12-bit 2016 x 2016 x 1800,
14.6 GB, 4096 bins, Otsu, levels 512^3 / 256^3 / 128^3, 36-view turntable at
1024 x 1024), run through the same pipeline object and launch configuration
as bench.py.  The histogram, threshold and all three atlases are compared
with the oracle over the whole volume (bit-exact); renders on sampled rays of
every fourth view (the oracle computes rays one by one)."""
import numpy as np
import pytest

from gpu_common import RENDER_TOL, STOP_EPS, render_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def full_config(mctp_pipeline, phantom):
    spec = phantom.FULL
    return mctp_pipeline.PreviewConfig(
        src_dims=(spec.nx, spec.ny, spec.nz), bits=12, nbins=4096, level0=(512, 512, 512), nlevels=3,
        views=mctp_pipeline.turntable(36, 1024, level=0, step=0.5, az_step=10.0), mode="otsu", alpha_stop=0.99)


def test_full_workload(capsys):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import phantom
    from paper_2311_15038_gb300 import pipeline as pl

    dev = torch.device("cuda:0")
    spec = phantom.FULL
    cfg = full_config(pl, phantom)
    vol = torch.empty(spec.shape, dtype=torch.uint16, device=dev)
    phantom.generate_gpu(spec, vol)
    # the GPU phantom writer agrees with the CPU writer (checked on bricks)
    for (x0, x1), (y0, y1), (z0, z1) in [((0, 64), (0, 48), (0, 6)), ((990, 1100), (900, 964), (800, 812)),
                                         ((1950, 2016), (1960, 2016), (1790, 1800))]:
        cpu = phantom.generate_cpu(spec, ((x0, x1), (y0, y1), (z0, z1)))
        assert np.array_equal(vol[z0:z1, y0:y1, x0:x1].cpu().numpy(), cpu)

    pipe = pl.PreviewPipeline(cfg, torch.uint16, dev)
    lut = torch.from_numpy(phantom.ramp_lut(256)).to(dev)
    flat, samples = pipe.run(vol, lut)
    torch.cuda.synchronize()

    vol_h = vol.cpu().numpy()
    del vol
    torch.cuda.empty_cache()
    h_ref, ov_ref = oracle.histogram(vol_h, 12, 4096)
    assert np.array_equal(pipe.hist.cpu().numpy(), h_ref)
    assert int(pipe.overflow.item()) == ov_ref == 0
    assert int(h_ref.sum()) == vol_h.size
    T, _ = oracle.otsu(h_ref)
    assert int(pipe.result[0].item()) == T
    keep_ref = oracle.keep_threshold(4096, T)
    assert np.array_equal(pipe.keep.cpu().numpy(), keep_ref)
    dims = [(512, 512, 512), (256, 256, 256), (128, 128, 128)]
    levels = oracle.slicemap(vol_h, 12, dims, keep_ref)
    del vol_h
    for k, lv in enumerate(levels):
        tx, ty = oracle.default_tiles(lv.shape[0])
        got = pipe.sm.atlases[k].cpu().numpy()
        ref = oracle.atlas_pack(lv, tx, ty)
        assert np.array_equal(got, ref), f"level {k}: {(got != ref).sum()} voxels differ"
        assert np.array_equal(pipe.sm.maxgrids[k].cpu().numpy(), oracle.maxgrid(lv, 8)), f"maxgrid {k}"
    # empty-space skipping is exact at full size too
    from paper_2311_15038_gb300 import render_views
    flat_full, samples_full = render_views(pipe.sm.without_maxgrid(), cfg.views, lut, 0.99)
    assert torch.equal(flat, flat_full) and int(samples.item()) == int(samples_full.item())
    del flat_full

    from paper_2311_15038_gb300 import images
    imgs = images(flat, cfg.views)
    rng = np.random.default_rng(1002)
    worst = 0.0
    for vi in range(0, 36, 4):
        v = cfg.views[vi]
        pix = np.concatenate([rng.integers(0, 1024 * 1024, size=300), 512 * 1024 + np.arange(0, 1024, 8)])
        ref = oracle.render(levels[0], 12, (spec.nx, spec.ny, spec.nz), phantom.ramp_lut(256), v.azimuth_deg,
                            v.elevation_deg, 1024, 1024, 0.5, 0.99, STOP_EPS, pixels=pix)
        got = imgs[vi].reshape(-1, 4)[torch.from_numpy(pix).to(dev)].cpu().numpy()
        err, amb = render_error(got, ref)
        worst = max(worst, float(err.max()))
        assert err.max() <= RENDER_TOL, (vi, float(err.max()))
    with capsys.disabled():
        print(f"\nfull workload: T={T}, samples={int(samples.item())}, sampled render max|err| vs FP64 = {worst:.3e}")
