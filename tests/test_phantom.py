"""The seeded phantom writer: deterministic, sub-boxes consistent with the
whole volume, and shaped like the scans the previews are made from (object
low in the container, surroundings alone in the top slices, Sec. III-D)."""
import numpy as np


def test_phantom_is_deterministic_and_boxes_agree(ph):
    spec = ph.VolumeSpec(61, 47, 53, bits=12, seed=77, n_ell=6, n_cyl=20)
    a = ph.generate_cpu(spec)
    b = ph.generate_cpu(spec)
    assert np.array_equal(a, b)
    box = ((13, 40), (5, 46), (20, 33))
    sub = ph.generate_cpu(spec, box)
    assert np.array_equal(sub, a[20:33, 5:46, 13:40])
    assert a.max() < 4096


def test_phantom_shape_of_workload(ph):
    v = ph.generate_cpu(ph.SMALL)
    assert v.shape == (256, 256, 256) and v.dtype == np.uint8
    top = v[:3]
    assert top.max() < 60                        # surroundings only
    assert 0.03 < (v > 60).mean() < 0.3           # an object fills part of the box
    bg = v[v < 60].astype(np.float64)
    assert abs(bg.mean() - 20) < 0.5 and abs(bg.std() - 5) < 0.5


def test_full_size_spec(ph):
    assert ph.FULL.nbytes == 2016 * 2016 * 1800 * 2
    P = ph.make_params(ph.FULL)
    assert len(P) > 0
    # a slab of the full-size volume, regenerated on the CPU
    sub = ph.generate_cpu(ph.FULL, ((1000, 1064), (900, 964), (0, 4)))
    assert sub.dtype == np.uint16 and sub.max() < 4096
    assert sub[:3].max() < 60 * 16


def test_luts(ph):
    luts = ph.preset_luts()
    assert len(luts) == 8
    for lut in luts:
        assert lut.shape == (256, 4) and lut.dtype == np.float32
        assert lut.min() >= 0 and lut.max() <= 1
    assert np.allclose(luts[0][:, 3], np.arange(256) / 255)


def test_batch_specs(ph):
    specs = ph.batch_specs()
    assert len(specs) == 64
    dims = np.array([(s.nx, s.ny, s.nz) for s in specs])
    assert dims.min() >= 384 and dims.max() <= 1024
    assert len({s.seed for s in specs}) == 64
