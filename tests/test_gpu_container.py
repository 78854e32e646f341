"""Container removal on the GPU against the oracle: the Hough vote counts,
the radius histogram, the refined circle (bit for bit: integer steps and a
fixed-order FP32/FP64 evaluation on both sides) and the masked volume, on
phantoms with a container (u8 and 12-bit u16, square and not), drawn rings,
a slice without edges, and in place."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import phantom
    import paper_2311_15038_gb300 as mctp
    return mctp, oracle, phantom, torch.device("cuda:0")


def _check_circle(mctp, oracle, vol_np, bits, z, thr, rmin, rmax, cell, dev):
    g = torch.from_numpy(np.ascontiguousarray(vol_np)).to(dev)
    got = mctp.find_container(g, bits, z, thr, rmin, rmax, cell)
    ref = oracle.hough_circle(vol_np[z], thr, rmin, rmax, cell)
    assert np.array_equal(got["acc"].cpu().numpy().view(np.uint32), ref["acc"]), "coarse votes"
    assert np.array_equal(got["rhist"].cpu().numpy().view(np.uint32), ref["rhist"]), "radius histogram"
    assert np.array_equal(got["fit"].cpu().numpy(), ref["fit"]), (got["fit"], ref["fit"])
    c = got["circle"].cpu().numpy()
    assert (int(c[0]), int(c[1]), int(c[2])) == (ref["cx"], ref["cy"], ref["r"])
    return g, got, ref


@pytest.mark.parametrize("nx,ny,nz,bits,seed", [(128, 128, 24, 8, 1), (300, 280, 16, 8, 2), (200, 210, 12, 12, 3)])
def test_container_phantom(env, nx, ny, nz, bits, seed):
    mctp, oracle, phantom, dev = env
    spec = phantom.VolumeSpec(nx, ny, nz, bits=bits, seed=seed, n_ell=4, tube=True)
    vol = phantom.generate_cpu(spec)
    n = min(nx, ny)
    thr = 40 * (1 << (bits - 8))
    g, got, ref = _check_circle(mctp, oracle, vol, bits, 0, thr, n // 8, n // 2, max(4, n // 32), dev)
    tx, ty, r_in, _ = phantom.tube_geometry(spec)
    print(f"container {nx}x{ny}: found {ref['fit']}, phantom axis ({tx:.2f}, {ty:.2f}) inner radius {r_in:.2f}")
    # mask every slice; margin 2 leaves the wall outside
    for margin in (0, 2):
        out = mctp.mask_container(g, bits, got["circle"], margin)
        rk = ref["r"] - margin if ref["r"] >= 0 else -1
        want = oracle.mask_circle(vol, ref["cx"], ref["cy"], max(rk, 0) if ref["r"] >= 0 else -1)
        assert np.array_equal(out.cpu().numpy(), want)
    # in place, on an unaligned slab (scalar path)
    slab = g[1:].clone()[:, :, :]
    view = g[1:]
    mctp.mask_container(view, bits, got["circle"], 2, out=view)
    want = oracle.mask_circle(vol[1:], ref["cx"], ref["cy"], ref["r"] - 2)
    assert np.array_equal(view.cpu().numpy(), want)
    assert not torch.equal(slab, view)  # the container wall was removed


@pytest.mark.parametrize("n,cx0,cy0,R", [(150, 71.3, 77.8, 50.0), (257, 130.6, 121.2, 101.5)])
def test_container_drawn_ring(env, n, cx0, cy0, R):
    mctp, oracle, phantom, dev = env
    y, x = np.mgrid[0:n, 0:n]
    d = np.hypot(x - cx0, y - cy0)
    ring = np.where((d >= R) & (d <= R + 6), 200, 20).astype(np.uint8)
    vol = np.stack([ring, ring // 2])
    _check_circle(mctp, oracle, vol, 8, 0, 40, n // 8, n // 2, 8, dev)


def test_container_none_found(env):
    mctp, oracle, phantom, dev = env
    vol = np.full((3, 40, 50), 33, np.uint8)
    g, got, ref = _check_circle(mctp, oracle, vol, 8, 0, 40, 5, 20, 4, dev)
    assert ref["r"] == -1
    out = mctp.mask_container(g, 8, got["circle"], 2)
    assert torch.equal(out, g)  # nothing found: nothing removed


def test_pipeline_with_container_removal(env):
    """The preview pipeline with container removal: the circle from slice 0,
    the mask, then histogram, Otsu and the slicemap of the masked volume, all
    equal to the oracle's chain; the container changes the Otsu threshold."""
    mctp, oracle, phantom, dev = env
    from paper_2311_15038_gb300 import pipeline as pl
    spec = phantom.VolumeSpec(160, 150, 64, bits=8, seed=7, n_ell=5, tube=True)
    vol = phantom.generate_cpu(spec)
    views = [mctp.View(30.0, 10.0, 32, 32, 0, 0.5)]
    cfg = pl.PreviewConfig((160, 150, 64), 8, 256, (80, 75, 32), 1, views, "otsu", container=True)
    pipe = pl.PreviewPipeline(cfg, torch.uint8, dev)
    lut = torch.from_numpy(phantom.ramp_lut(256)).to(dev)
    pipe.run(torch.from_numpy(vol).to(dev), lut)
    torch.cuda.synchronize()
    h = oracle.hough_circle(vol[0], 40, 150 // 8, 150 // 2, max(4, 150 // 32))
    masked = oracle.mask_circle(vol, h["cx"], h["cy"], h["r"] - 2)
    assert np.array_equal(pipe.masked.cpu().numpy(), masked)
    hist, _ = oracle.histogram(masked, 8, 256)
    T = oracle.otsu(hist)[0]
    assert int(pipe.result[0].item()) == T
    T_raw = oracle.otsu(oracle.histogram(vol, 8, 256)[0])[0]
    print(f"Otsu threshold with the container {T_raw}, after removing it {T}")
    level = oracle.slicemap(masked, 8, [(80, 75, 32)], oracle.keep_threshold(256, T))[0]
    tx, ty = oracle.default_tiles(32)
    assert np.array_equal(pipe.sm.atlases[0].cpu().numpy(), oracle.atlas_pack(level, tx, ty))
