"""Exact-arithmetic identities the split-precision products rely on, checked on the CPU.

The split products (Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012) carry FP64 operands as
six balanced base-2^7 digits and sum digit products exactly in FP32.  The kernels rely on:

* balanced digits: for |v| <= 2^41, the 7-bit digits e_i of u = v + 64 (1 + 128 + ... + 128^5), the
  top one taking all of u above bit 35, give d_i = e_i - 64 in [-64, 64] (only the top one reaches
  64, at v = 2^41) with sum_i d_i 128^(5-i) = v;
* a digit d in [-64, 64] is exact in BF16 and FP16, and (bit pattern 0x4B400000 + d) read as FP32,
  minus 1.5 * 2^23, is d;
* a level sum of a chunk, at most 6 * 640 * 64^2 < 2^24 in magnitude, is an exact FP32 integer, and
  for |x| <= 2^22 the integer is (bits of x + 1.5 * 2^23) - 0x4B400000;
* the 64-bit recombination sum_t L_t 128^(5-t) cannot overflow for the K the library allows.
"""
import numpy as np

BIAS = 64 * ((1 << 42) - 1) // 127   # 64 * (1 + 128 + ... + 128^5)


def balanced_digits(v):
    # the five low digits are 7-bit fields of u; the top one is all of u above bit 35 (it takes the rest)
    u = v.astype(np.int64) + BIAS
    return np.stack([(u >> 35) - 64] + [((u >> (7 * (5 - i))) & 127) - 64 for i in range(1, 6)], axis=-1)


def test_balanced_digits_reconstruct_and_stay_in_range():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.integers(-(1 << 41), (1 << 41) + 1, 200000),
                        np.array([-(1 << 41), (1 << 41), 0, 1, -1, 63, 64, -64, -65])])
    d = balanced_digits(v)
    assert d.min() >= -64 and d.max() <= 64
    assert (d[:, 1:] <= 63).all()   # only the top digit reaches 64
    back = sum(d[:, i].astype(np.int64) * (1 << (7 * (5 - i))) for i in range(6))
    assert np.array_equal(back, v)


def test_digits_are_exact_in_16_bits_and_through_the_bit_pattern():
    d = np.arange(-64, 65)
    f = (np.int32(0x4B400000) + d.astype(np.int32)).view(np.float32) - np.float32(12582912.0)
    assert np.array_equal(f, d.astype(np.float32))
    assert np.array_equal(d.astype(np.float16).astype(np.int64), d)
    # BF16 keeps the top 16 bits of the FP32 word: 8 significant bits hold every |d| <= 64
    top = (d.astype(np.float32).view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32)
    assert np.array_equal(top, d.astype(np.float32))


def test_level_sums_are_exact_fp32_integers_and_convert_by_one_add():
    assert 6 * 640 * 64 * 64 < (1 << 24)
    m = 1 << 22
    x = np.arange(-m, m + 1, dtype=np.int64)
    xf = x.astype(np.float32)
    assert np.array_equal(xf.astype(np.int64), x)
    got = (xf + np.float32(12582912.0)).view(np.int32).astype(np.int64) - 0x4B400000
    assert np.array_equal(got, x)


def test_int64_recombination_has_room_for_the_allowed_k():
    # one chunk contributes |sum_t L_t 128^(5-t)| <= sum_t (t+1) * 640 * 64^2 * 128^(5-t); the library
    # allows K <= 8192 per charge group, i.e. at most 13 chunks of 640
    per_chunk = sum((t + 1) * 640 * 64 * 64 * 128 ** (5 - t) for t in range(6))
    assert 13 * per_chunk < (1 << 63)
