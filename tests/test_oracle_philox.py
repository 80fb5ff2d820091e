"""Pins for the oracle's Philox4x32-10 (the 32-bit integer generator of
Appendix B, keyed per site as the design fixes).

The pin is a black-box comparison with cuRAND's host-side Philox4_32_10
generator, which runs on the CPU.  Probing it shows that, for seed S and
stream offset o, output word i comes from block B = (o + i) // 4 with key
(lo32 S, hi32 S) and counter (lo32(B // 65536), hi32(B // 65536), B % 65536, 0),
word (o + i) % 4.  The oracle's own code is then compared against that stream
at offsets that put non-zero values in counter words 0, 1 and 2 and in both key
words.  Statistical sanity checks follow.
"""
import ctypes
import os

import numpy as np
import pytest

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so.10", "libcurand.so"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    return None


def _curand_host_stream(cr, seed, offset, n):
    gen = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert cr.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        buf = (ctypes.c_uint32 * n)()
        assert cr.curandGenerate(gen, buf, ctypes.c_size_t(n)) == 0
        return [int(v) for v in buf]
    finally:
        cr.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 1, 0x2503146880000001, 0xFFFFFFFFFFFFFFFF,
                                  0x123456789ABCDEF0])
@pytest.mark.parametrize("offset", [0, 4 * 65535, (1 << 34) + 8, (1 << 50) + 12,
                                    3 * (1 << 52) + 65536 * 4 * 7 + 40])
def test_philox_matches_curand_host_generator(orc, seed, offset):
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not present")
    n = 64
    got = _curand_host_stream(cr, seed, offset, n)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    want = []
    for i in range(0, n, 4):
        B = (offset + i) // 4
        q, th = divmod(B, 65536)
        want += orc.philox4x32_10([q & 0xFFFFFFFF, q >> 32, th, 0], key)
    assert got == want


def test_site_random_selects_word_of_counter(orc):
    """site_random(j) is word j & 3 of Philox at counter j >> 2."""
    seed = 0x2503146880000004
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in [0, 1, 2, 3, 4, 7, 1 << 33, (1 << 36) + 3, (1 << 39) - 1]:
        q = j >> 2
        block = orc.philox4x32_10([q & 0xFFFFFFFF, q >> 32, 17, 1], key)
        assert orc.site_random(seed, j, 17, 1) == block[j & 3]


def test_philox_bit_balance_and_byte_histogram(orc):
    """Each output bit is set half the time; low bytes are uniform (chi^2)."""
    words = []
    seed = 12345
    for q in range(4096):
        words += orc.philox4x32_10([q, 0, 3, 1], [seed, 0])
    w = np.array(words, dtype=np.uint64)
    n = w.size
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint64)) & 1).sum(axis=0)
    assert np.all(np.abs(bits - n / 2) < 5 * np.sqrt(n / 4))
    hist = np.bincount((w & 0xFF).astype(np.int64), minlength=256)
    chi2 = ((hist - n / 256) ** 2 / (n / 256)).sum()
    # 255 degrees of freedom: mean 255, sd ~22.6
    assert 150 < chi2 < 380


def test_philox_counter_words_all_matter(orc):
    """Changing any one counter or key word changes every output word."""
    base_c, base_k = [11, 22, 33, 44], [55, 66]
    ref = orc.philox4x32_10(base_c, base_k)
    for i in range(4):
        c = list(base_c)
        c[i] ^= 1
        out = orc.philox4x32_10(c, base_k)
        assert all(a != b for a, b in zip(out, ref))
    for i in range(2):
        k = list(base_k)
        k[i] ^= 1
        out = orc.philox4x32_10(base_c, k)
        assert all(a != b for a, b in zip(out, ref))
