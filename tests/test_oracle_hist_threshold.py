"""Pins of the CPU oracle's histogram, threshold selection and filter.

Each check ties the oracle to something other than itself: numpy routines,
closed forms of Alg. 1 / Alg. 2 (Sec. III-A), the within-class variance of
Eq. 1 evaluated by brute force, and hand-derived golden values.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            out.setdefault(k.strip(), []).append(v.split())
    return out


# ---------------------------------------------------------------- histogram

@pytest.mark.parametrize("shape,bits,nbins,dtype,vmax", [
    ((5, 7, 9), 8, 256, np.uint8, 256),
    ((3, 4, 17), 8, 64, np.uint8, 256),
    ((2, 3, 5), 8, 1, np.uint8, 256),
    ((4, 6, 11), 12, 4096, np.uint16, 65536),   # values >= 4096 overflow
    ((4, 6, 11), 12, 512, np.uint16, 5000),
    ((3, 3, 3), 16, 65536, np.uint16, 65536),
])
def test_histogram_matches_bincount(orc, shape, bits, nbins, dtype, vmax):
    rng = np.random.default_rng(7)
    vol = rng.integers(0, vmax, size=shape).astype(dtype)
    hist, ov = orc.histogram(vol, bits, nbins)
    v = vol.astype(np.int64).ravel()
    valid = v < (1 << bits)
    ref = np.bincount(v[valid] >> (bits - int(np.log2(nbins))), minlength=nbins)
    assert np.array_equal(hist, ref.astype(np.uint64))
    assert ov == int((~valid).sum())
    assert int(hist.sum()) + ov == vol.size


def test_histogram_z_range(orc):
    rng = np.random.default_rng(3)
    vol = rng.integers(0, 256, size=(9, 5, 6)).astype(np.uint8)
    hist, _ = orc.histogram(vol, 8, 256, 2, 5)
    ref = np.bincount(vol[2:5].ravel(), minlength=256)
    assert np.array_equal(hist, ref.astype(np.uint64))
    empty, _ = orc.histogram(vol, 8, 256, 4, 4)
    assert int(empty.sum()) == 0


@pytest.mark.parametrize("bits,nbins", [(8, 3), (8, 512), (12, 8192), (8, 0)])
def test_histogram_rejects_bad_bins(orc, bits, nbins):
    vol = np.zeros((2, 2, 2), np.uint8 if bits <= 8 else np.uint16)
    with pytest.raises(ValueError):
        orc.histogram(vol, bits, nbins)


# ---------------------------------------------------------------------- Otsu

def _within_class_variance(hist, T):
    """Eq. 1: w0 s0^2 + w1 s1^2, from the expanded samples (two-pass variance)."""
    b = np.arange(hist.size)
    samples = np.repeat(b, hist.astype(np.int64))
    lo = samples[samples < T]
    hi = samples[samples >= T]
    if lo.size == 0 or hi.size == 0:
        return None
    n = samples.size
    return lo.size / n * lo.var() + hi.size / n * hi.var()


@pytest.mark.parametrize("seed", range(6))
def test_otsu_minimises_within_class_variance(orc, seed):
    rng = np.random.default_rng(seed)
    nbins = [16, 32, 64][seed % 3]
    hist = rng.integers(0, 50, size=nbins).astype(np.uint64)
    hist[rng.integers(0, nbins, size=nbins // 3)] = 0
    T, _ = orc.otsu(hist)
    vals = {t: _within_class_variance(hist, t) for t in range(nbins)}
    vals = {t: v for t, v in vals.items() if v is not None}
    best = min(vals.values())
    assert vals[T] <= best * (1 + 1e-12) + 1e-12
    # first minimiser (ties keep the lowest T), where the minimum is clear
    clear = [t for t, v in vals.items() if v <= best * (1 + 1e-9)]
    assert T == min(clear)


@pytest.mark.parametrize("a,b,na,nb,nbins", [(3, 11, 5, 9, 16), (0, 255, 1, 1, 256), (100, 101, 7, 2, 256)])
def test_otsu_two_deltas(orc, a, b, na, nb, nbins):
    hist = np.zeros(nbins, np.uint64)
    hist[a] = na
    hist[b] = nb
    T, sigma = orc.otsu(hist)
    # every T in (a, b] gives the same split; the first one wins
    assert T == a + 1
    n = na + nb
    assert sigma == pytest.approx(na / n * nb / n * (a - b) ** 2, rel=1e-15)


def test_otsu_golden(orc):
    g = _read_golden("otsu_its_6bins.txt")
    hist = np.array([int(x) for x in g["hist"][0]], np.uint64)
    T, sigma = orc.otsu(hist)
    assert T == int(g["otsu_T"][0][0])
    assert sigma == pytest.approx(int(g["otsu_sigma_num"][0][0]) / int(g["otsu_sigma_den"][0][0]),
                                  rel=1e-15)


def test_otsu_degenerate(orc):
    assert orc.otsu(np.zeros(8, np.uint64))[0] == 0      # empty histogram
    h = np.zeros(8, np.uint64)
    h[5] = 10
    assert orc.otsu(h)[0] == 0                            # one grey value: no split


# ----------------------------------------------------------------------- ITS

def test_its_golden(orc):
    g = _read_golden("otsu_its_6bins.txt")
    hist = np.array([int(x) for x in g["hist"][0]], np.uint64)
    T, iters, conv, T_real = orc.its(hist)
    assert conv
    assert T == int(g["its_T"][0][0])
    assert iters == int(g["its_iters"][0][0])
    assert T_real == float(g["its_T_real"][0][0])


@pytest.mark.parametrize("a,b,nbins", [(1, 12, 16), (20, 200, 256), (3, 4, 256), (30, 3000, 4096)])
def test_its_two_deltas(orc, a, b, nbins):
    hist = np.zeros(nbins, np.uint64)
    hist[a] = 13
    hist[b] = 4
    T, iters, conv, T_real = orc.its(hist)
    assert conv
    # fixed point: mu1 = a, mu2 = b, T = (a + b) / 2
    assert T_real == (a + b) / 2
    assert T == int(np.ceil((a + b) / 2))
    if a < nbins // 2 <= b:
        assert iters <= 3          # start splits the deltas: one move, one confirmation
    else:
        assert iters <= 20         # an empty side halves the distance each iteration


@pytest.mark.parametrize("sd", [9.0, 30.0])
def test_symmetric_bimodal(orc, sd):
    x = np.arange(256)
    h = np.round(1e6 * (np.exp(-0.5 * ((x - 60) / sd) ** 2) +
                        np.exp(-0.5 * ((x - 195) / sd) ** 2))).astype(np.uint64)
    assert np.array_equal(h, h[::-1])
    T, iters, conv, T_real = orc.its(h)
    # ITS: the mirror-image class means average to the centre 127.5
    assert conv and abs(T_real - 127.5) < 1e-9 and T == 128
    To, _ = orc.otsu(h)
    if sd == 30.0:
        # overlapping modes: sigma(T) = sigma(256 - T) peaks at the centre
        assert To == 128
    else:
        # separated modes: every split in the empty gap ties; the first wins
        gap = np.nonzero(h[60:196] == 0)[0]
        assert To == 60 + int(gap[0])


def test_its_empty_region_creeps_to_the_mode(orc):
    # every voxel above the start: the lower region stays empty and the
    # threshold halves its distance to the mode each iteration
    h = np.zeros(16, np.uint64)
    h[10] = 5
    T, iters, conv, T_real = orc.its(h, max_iter=256)
    assert conv and T == 10 and T_real == 10.0
    assert 40 < iters < 60
    T2, iters2, conv2, _ = orc.its(h, max_iter=5)
    assert not conv2 and iters2 == 5 and T2 == 10


def test_its_and_otsu_agree_on_separated_phantom(orc, ph):
    vol = ph.generate_cpu(ph.SMALL)
    h, _ = orc.histogram(vol, 8, 256)
    To, _ = orc.otsu(h)
    Ti, iters, conv, _ = orc.its(h)
    assert conv and iters <= 20           # "roughly ten iterations"
    assert abs(To - Ti) <= 1              # identical on well-separated data
    assert 30 < To < 80                   # between background and object modes


# --------------------------------------------------------------- keep tables

def test_keep_threshold(orc):
    k = orc.keep_threshold(16, 5)
    assert k.tolist() == [0] * 5 + [1] * 11
    assert orc.keep_threshold(4, 0).tolist() == [1, 1, 1, 1]
    assert orc.keep_threshold(4, 4).tolist() == [0, 0, 0, 0]


def test_topslab_removes_surroundings(orc):
    vol = np.zeros((8, 4, 5), np.uint8)
    rng = np.random.default_rng(0)
    vol[:] = rng.choice([5, 7], size=vol.shape)       # surroundings everywhere
    vol[5:, 1:3, 1:4] = rng.choice([100, 120, 7], size=(3, 2, 3))
    hist_top, _ = orc.histogram(vol, 8, 256, 0, 3)
    keep = orc.keep_topslab(hist_top, 1)
    assert keep[5] == 0 and keep[7] == 0 and keep[100] == 1 and keep[120] == 1
    out = orc.filter_volume(vol, 8, keep)
    assert set(np.unique(out).tolist()) <= {0, 100, 120}
    assert np.array_equal(out > 0, np.isin(vol, [100, 120]))
    keep2 = orc.keep_topslab(hist_top, 10 ** 9)
    assert keep2.all()


# -------------------------------------------------------------------- filter

@pytest.mark.parametrize("bits,nbins,dtype,vmax", [(8, 256, np.uint8, 256), (8, 32, np.uint8, 256),
                                                   (12, 4096, np.uint16, 5000), (12, 64, np.uint16, 4096)])
def test_filter_matches_numpy(orc, bits, nbins, dtype, vmax):
    rng = np.random.default_rng(11)
    vol = rng.integers(0, vmax, size=(5, 6, 7)).astype(dtype)
    keep = rng.integers(0, 2, size=nbins).astype(np.uint8)
    out = orc.filter_volume(vol, bits, keep)
    v = vol.astype(np.int64)
    shift = bits - int(np.log2(nbins))
    valid = v < (1 << bits)
    kept = np.zeros_like(valid)
    kept[valid] = keep[v[valid] >> shift] == 1
    assert np.array_equal(out, np.where(kept, vol, 0).astype(dtype))
    assert np.array_equal(orc.filter_volume(out, bits, keep), out)    # idempotent


# ------------------------------------------------------------------- entropy

def test_entropy_closed_forms(orc):
    assert orc.entropy(np.full(256, 7, np.uint64)) == pytest.approx(8.0, abs=1e-12)
    one = np.zeros(16, np.uint64)
    one[3] = 99
    assert orc.entropy(one) == 0.0
    assert orc.entropy(np.array([5, 5, 0, 0], np.uint64)) == pytest.approx(1.0, abs=1e-15)
    p = np.array([1, 2, 3, 4], np.float64) / 10
    assert orc.entropy(np.array([1, 2, 3, 4], np.uint64)) == pytest.approx(-(p * np.log2(p)).sum(), rel=1e-14)


def test_image_histogram_pins(orc):
    # grey pixels (R = G = B = k/255) have luminance k/255: bin k
    k = np.arange(256, dtype=np.float32) / np.float32(255.0)
    grey = np.stack([k, k, k, np.ones(256, np.float32)], axis=1)
    assert np.array_equal(orc.image_histogram(grey), np.ones(256, np.uint64))
    assert orc.image_entropy(grey) == pytest.approx(8.0, abs=1e-12)
    # primaries land at their luminance weights: round(0.2126*255)=54, round(0.7152*255)=182, round(0.0722*255)=18
    prim = np.array([[1, 0, 0, 1], [0, 1, 0, 1], [0, 0, 1, 1], [0, 0, 0, 0], [2.0, 2.0, 2.0, 1.0]], np.float32)
    h = orc.image_histogram(prim)
    assert h[54] == 1 and h[182] == 1 and h[18] == 1 and h[0] == 1 and h[255] == 1 and h.sum() == 5
    # a black image carries no information
    assert orc.image_entropy(np.zeros((7, 9, 4), np.float32)) == 0.0
