"""mctp_render_batch_static: the batched renderer on the library's fixed
device scratch instead of a caller workspace.  Two calls in a row through the
C ABI must give the images and sample counts of mctp_render_batch with a
caller workspace (bit for bit, i.e. within any tolerance) and must not change
the device's free memory.  This file is collected last so that it also runs
after every other GPU test in the same process."""
import ctypes

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
    import phantom
    import paper_2311_15038_gb300 as mctp
    return mctp, phantom, torch.device("cuda:0")


def _batch(env):
    mctp, phantom, dev = env
    V = phantom.VolumeSpec
    specs = [(V(70, 64, 58, bits=8, seed=61, n_ell=5), (35, 32, 29)),
             (V(90, 50, 66, bits=8, seed=62, n_ell=4), (45, 25, 33)),
             (V(48, 56, 40, bits=8, seed=63, n_ell=3), (48, 56, 40))]
    sms = []
    for spec, dims in specs:
        vol = torch.empty(spec.shape, dtype=torch.uint8, device=dev)
        phantom.generate_gpu(spec, vol)
        h, _ = mctp.build_histogram(vol, 8, 256)
        keep, _ = mctp.select_threshold(h, 256)
        sm = mctp.Slicemap.allocate((spec.nx, spec.ny, spec.nz), dims, 1, torch.uint8, 8, dev)
        mctp.build_slicemap(vol, 8, sm, keep)
        sms.append(sm)
    luts = torch.from_numpy(np.stack(phantom.preset_luts()[:3])).to(dev)
    rng = np.random.default_rng(17)
    views, vsm, vlut = [], [], []
    for i in range(20):
        w, hgt = [(40, 30), (17, 64), (64, 64), (1, 9)][i % 4]
        views.append(mctp.View(float(rng.uniform(-180, 180)), float(rng.uniform(-50, 50)), w, hgt, 0, 0.5))
        vsm.append(i % 3)
        vlut.append(int(rng.integers(3)))
    return sms, views, vsm, vlut, luts


def test_static_scratch_matches_workspace_call(env):
    mctp, phantom, dev = env
    from paper_2311_15038_gb300 import _lib
    sms, views, vsm, vlut, luts = _batch(env)
    ref, ref_samples, _ = mctp.render_batch(sms, views, vsm, vlut, luts, 0.99)
    torch.cuda.synchronize(dev)

    total = sum(v.width * v.height * 4 for v in views)
    out = torch.empty(total, dtype=torch.float32, device=dev)
    samples = torch.empty(1, dtype=torch.uint64, device=dev)
    a = mctp._BatchArgs(sms, views, vsm, vlut)
    tun = mctp.BatchTuning().c()
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)

    def call():
        return lib.mctp_render_batch_static(a.sms, a.nsm, a.views, a.vsm, a.vlut, a.n,
                                            ctypes.c_void_p(luts.data_ptr()), luts.shape[0], luts.shape[1], 0.99,
                                            ctypes.byref(tun), ctypes.c_void_p(out.data_ptr()),
                                            ctypes.c_void_p(samples.data_ptr()), stream)

    def check():
        err = (out - ref[:total]).abs().max().item()
        print(f"static scratch vs workspace: max |diff| = {err:.3e}, samples {int(samples.item())}")
        assert err <= 0.0
        assert torch.equal(out, ref[:total])
        assert int(samples.item()) == int(ref_samples.item())

    assert call() == 0  # first call on this device: the scratch address is looked up
    torch.cuda.synchronize(dev)
    check()  # also warms up the torch operations used around the calls below
    for _ in range(2):  # two calls in a row on the same scratch
        out.fill_(-1.0)
        samples.zero_()
        torch.cuda.synchronize(dev)
        free_before, _ = torch.cuda.mem_get_info(dev)
        assert call() == 0
        torch.cuda.synchronize(dev)
        free_after, _ = torch.cuda.mem_get_info(dev)
        assert free_after == free_before  # the call allocated no device memory
        check()
