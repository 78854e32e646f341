"""The preview server (mctp_server_*): requests submitted in bursts are
batched, admitted by free arena memory and rendered on several streams.
Every served image (and the server's sample total) must equal rendering the
request's view alone with mctp_render_views: the same result alone and in
the mix, bit for bit (so within the 2e-4 tolerance of the path)."""
import time

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
    from paper_2311_15038_gb300 import serve
    dev = torch.device("cuda:0")
    V = phantom.VolumeSpec
    specs = [(V(64, 64, 64, bits=8, seed=71, n_ell=5), [(32, 32, 32), (16, 16, 16)]),
             (V(96, 80, 72, bits=8, seed=72, n_ell=6), [(48, 40, 36)]),
             (V(50, 70, 90, bits=8, seed=73, n_ell=4), [(50, 70, 90), (25, 35, 45)])]
    sms = []
    for spec, dims in specs:
        vol = torch.empty(spec.shape, dtype=torch.uint8, device=dev)
        phantom.generate_gpu(spec, vol)
        h, _ = mctp.build_histogram(vol, 8, 256)
        keep, _ = mctp.select_threshold(h, 256)
        sm = mctp.Slicemap.allocate((spec.nx, spec.ny, spec.nz), dims[0], len(dims), torch.uint8, 8, dev)
        mctp.build_slicemap(vol, 8, sm, keep)
        sms.append(sm)
    luts = torch.from_numpy(np.stack(phantom.preset_luts())).to(dev)
    return mctp, serve, sms, luts, dev


def _requests(mctp, sms, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        s = int(rng.integers(len(sms)))
        w, h = [(48, 48), (64, 40), (17, 90), (96, 96), (1, 1)][i % 5]
        v = mctp.View(float(rng.uniform(0, 360)), float(rng.uniform(-60, 60)), w, h,
                      int(rng.integers(len(sms[s].dims))), 0.5)
        out.append((v, s, int(rng.integers(8))))
    return out


def _alone(mctp, sms, luts, req):
    v, s, l = req
    flat, smp = mctp.render_views(sms[s], [v], luts[l], 0.99)
    return flat[:v.width * v.height * 4].view(v.height, v.width, 4), int(smp.item())


def _serve_all(srv, reqs, release=True, timeout=60.0):
    tickets = {srv.submit(v, s, l): i for i, (v, s, l) in enumerate(reqs)}
    got = {}
    t0 = time.time()
    while len(got) < len(reqs):
        for f in srv.poll():
            assert f.status == 0
            got[tickets[f.ticket]] = (f, srv.image(f))
            if release:
                srv.release(f.ticket)
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(0.0005)
    return got


@pytest.mark.parametrize("mode,batch,inflight", [("batched", 16, 2), ("batched", 64, 4), ("per_view", 1, 1)])
def test_served_equals_alone(env, mode, batch, inflight):
    mctp, serve, sms, luts, dev = env
    reqs = _requests(mctp, sms, 80, seed=5)
    with serve.Server(sms, luts, 256 << 20, mode, batch, inflight) as srv:
        got = _serve_all(srv, reqs)
        st = srv.stats()
    total = 0
    for i, req in enumerate(reqs):
        ref, smp = _alone(mctp, sms, luts, req)
        total += smp
        f, img = got[i]
        assert torch.equal(img, ref), f"request {i} differs from rendering it alone"
        assert f.t_submit <= f.t_admit <= f.t_launch <= f.t_done
    assert st["samples"] == total
    if mode == "batched":
        assert st["launches"] < len(reqs)  # the burst was batched
    else:
        assert st["launches"] == len(reqs)


def test_admission_by_memory(env):
    """A 1 MiB arena whose image heap holds about six 96x96 images at a time:
    requests wait for memory that releases free, and all of them still finish
    with the right images."""
    mctp, serve, sms, luts, dev = env
    reqs = [(mctp.View(10.0 * i, 15.0, 96, 96, 0, 0.5), i % 3, i % 8) for i in range(24)]
    img = 96 * 96 * 16
    with serve.Server(sms, luts, 1 << 20, "batched", 8, 2) as srv:
        got = _serve_all(srv, reqs)
        st = srv.stats()
    assert st["arena_high_water"] <= (1 << 20)
    waited = sum(1 for f, _ in got.values() if f.t_admit > f.t_submit + 1e-4)
    assert waited > 0, "no request had to wait for memory"
    for i, req in enumerate(reqs):
        ref, _ = _alone(mctp, sms, luts, req)
        assert torch.equal(got[i][1], ref)
    assert st["arena_high_water"] >= img


def test_submit_rejects_image_larger_than_heap(env):
    mctp, serve, sms, luts, dev = env
    with serve.Server(sms, luts, 1 << 20, "batched", 8, 2) as srv:
        with pytest.raises(mctp.MctpError):
            srv.submit(mctp.View(0.0, 0.0, 512, 512, 0, 0.5), 0, 0)
        with pytest.raises(mctp.MctpError):
            srv.submit(mctp.View(0.0, 0.0, 8, 8, 5, 0.5), 0, 0)  # level out of range


def test_served_with_textures_and_depth_bounds(env):
    """Slicemaps with atlas textures: the batched server gathers corners and
    marches within each tile's depth bounds when its workspace has room for
    them (views up to 1024 x 1024), and without them for larger views; every
    image still equals rendering its view alone with loads."""
    import dataclasses
    mctp, serve, sms, luts, dev = env
    tex = [dataclasses.replace(sm, textures=None).make_textures() for sm in sms]
    for t in tex:
        t.update_textures()
    reqs = _requests(mctp, tex, 60, seed=7)
    big = [(mctp.View(30.0 + 50.0 * i, 10.0, 1100, 1100, 0, 0.5), i % len(sms), i) for i in range(2)]
    for batch, rq in ((32, reqs), (2, big)):
        with serve.Server(tex, luts, 256 << 20, "batched", batch, 2) as srv:
            got = _serve_all(srv, rq)
            st = srv.stats()
        total = 0
        for i, req in enumerate(rq):
            ref, smp = _alone(mctp, sms, luts, req)
            total += smp
            assert torch.equal(got[i][1], ref), f"request {i} of the {batch}-view server differs"
        assert st["samples"] == total


def _drain(srv, n, timeout=60.0):
    """Poll until n requests have finished; returns {ticket: Finished}."""
    got = {}
    t0 = time.time()
    while len(got) < n:
        for f in srv.poll():
            got[f.ticket] = f
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(0.0005)
    return got


def test_cancelled_requests_leave_the_queue(env):
    """Requests waiting for memory (a 3 MiB arena whose image heap holds at
    most two 256^2 images) are cancelled: they finish with MCTP_ECANCELED and no image,
    take no launch, and the requests not cancelled still equal rendering their
    views alone; a finished or unknown ticket is not cancellable."""
    mctp, serve, sms, luts, dev = env
    from paper_2311_15038_gb300 import _lib
    v = mctp.View(20.0, 10.0, 256, 256, 0, 0.5)
    reqs = [(v, i % len(sms), i % 8) for i in range(8)]
    with serve.Server(sms, luts, 3 << 20, "batched", 8, 1) as srv:
        tickets = [srv.submit(*r) for r in reqs]
        cancelled = [t for t in tickets[2:7] if srv.cancel(t)]
        assert len(cancelled) >= 3  # the first two may already be admitted or launched
        got = {}
        t0 = time.time()
        while len(got) < len(tickets):
            for f in srv.poll():
                if f.status == 0:
                    img = srv.image(f).clone()
                    srv.release(f.ticket)
                    got[f.ticket] = (f, img)
                else:
                    got[f.ticket] = (f, None)
                    srv.release(f.ticket)
            assert time.time() - t0 < 60.0
            time.sleep(0.0005)
        for t in cancelled:
            f, img = got[t]
            assert f.status == _lib.MCTP_ECANCELED and f.image_ptr == 0 and img is None
        for t, r in zip(tickets, reqs):
            if t in cancelled:
                continue
            f, img = got[t]
            assert f.status == 0
            ref, _ = _alone(mctp, sms, luts, r)
            assert torch.equal(img, ref)
        assert srv.stats()["launches"] <= len(tickets) - len(cancelled)
        assert not srv.cancel(tickets[0])        # finished and released
        assert not srv.cancel(123456789)         # unknown


def test_injected_launch_failures(env):
    """Host-side fault injection: the next two launches fail as a failed
    kernel launch would; their requests finish with MCTP_ECUDA, nothing is
    left in flight, and the server serves the following requests correctly."""
    mctp, serve, sms, luts, dev = env
    from paper_2311_15038_gb300 import _lib
    reqs = _requests(mctp, sms, 12, seed=21)
    with serve.Server(sms, luts, 64 << 20, "per_view", 1, 1) as srv:
        srv.inject_launch_failures(2)
        first = [srv.submit(*r) for r in reqs[:4]]
        done = _drain(srv, 4)
        status = [done[t].status for t in first]
        assert status.count(_lib.MCTP_ECUDA) == 2 and status.count(0) == 2
        for t in first:
            srv.release(t)
        got = _serve_all(srv, reqs[4:])
        for i, (f, img) in got.items():
            ref, _ = _alone(mctp, sms, luts, reqs[4 + i])
            assert torch.equal(img, ref)


def test_slow_producer_and_malformed_requests(env):
    """Requests that trickle in one by one (the server idles between them)
    each finish alone and correct; malformed requests (bad slicemap or LUT
    index, a level the slicemap lacks, a zero-sized view) are refused at
    submit and leave nothing behind."""
    mctp, serve, sms, luts, dev = env
    reqs = _requests(mctp, sms, 5, seed=33)
    with serve.Server(sms, luts, 64 << 20, "batched", 16, 2) as srv:
        for r in reqs:
            got = _serve_all(srv, [r])
            ref, _ = _alone(mctp, sms, luts, r)
            assert torch.equal(got[0][1], ref)
            time.sleep(0.01)
        v = mctp.View(0.0, 0.0, 32, 32, 0, 0.5)
        for bad in [(v, len(sms), 0), (v, 0, 99), (mctp.View(0.0, 0.0, 32, 32, 5, 0.5), 1, 0),
                    (mctp.View(0.0, 0.0, 0, 32, 0, 0.5), 0, 0)]:
            with pytest.raises(mctp.MctpError):
                srv.submit(*bad)
        assert srv.poll() == []
