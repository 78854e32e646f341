"""The arithmetic facts the u8 row kernel of the slicemap build relies on,
checked with numpy's IEEE half precision (the kernel's fp16 pair operations
round the same way):

* a byte b placed in the low bits of a 16-bit lane reads as the fp16 value
  b * 2^-24, and for every integer k <= 2048 the fp16 encoding of k * 2^-24
  is the bit pattern k (subnormals and the first normal binade have the same
  spacing 2^-24), so a pair register of such sums is also two packed 16-bit
  integers;
* adding up to 8 such bytes in any order is exact (the sum stays <= 2048);
* the step test `value >= threshold` on these encodings agrees with the
  integer test, and multiplying by its 1.0 / 0.0 result keeps or drops the
  byte exactly;
* a ninth byte can round, which is why the kernel folds its pair sums into
  integer column sums every 8 source rows.
"""
import numpy as np

UNIT = np.float16(2.0 ** -24)


def test_bit_pattern_is_the_integer():
    k = np.arange(0, 2049, dtype=np.uint16)
    h = k.view(np.float16)
    assert np.array_equal(h.astype(np.float64), k.astype(np.float64) * 2.0 ** -24)
    # and the value k * 2^-24, rounded to fp16, encodes as k
    assert np.array_equal((k.astype(np.float64) * 2.0 ** -24).astype(np.float16).view(np.uint16), k)


def test_sums_of_eight_bytes_are_exact():
    rng = np.random.default_rng(1)
    b = rng.integers(0, 256, size=(20000, 8)).astype(np.uint16)
    b[:50] = 255                                    # the largest sums
    acc = np.zeros(len(b), np.float16)
    for r in range(8):
        acc = (acc + b[:, r].view(np.float16)).astype(np.float16)
    assert np.array_equal(acc.view(np.uint16), b.sum(axis=1).astype(np.uint16))


def test_step_test_and_masked_add():
    v = np.arange(256, dtype=np.uint16).view(np.float16)
    for lo in (0, 1, 37, 128, 255, 256):
        thr = np.uint16(lo).view(np.float16)
        keep = (v >= thr)
        assert np.array_equal(keep, np.arange(256) >= lo)
        prod = (v * keep.astype(np.float16)).astype(np.float16)
        assert np.array_equal(prod.view(np.uint16), np.where(np.arange(256) >= lo, np.arange(256), 0))


def test_a_ninth_byte_can_round():
    acc = np.uint16(2040).view(np.float16)
    nxt = (acc + np.uint16(255).view(np.float16)).astype(np.float16)
    assert nxt.astype(np.float64) != (2040 + 255) * 2.0 ** -24
