"""Pins for the oracle's correlation function along the axes (Eq. (2)):
agreement with a library FFT autocorrelation (Wiener-Khinchin), the identity
S_x(1) + S_y(1) = B with the bond sum behind E (Eq. (3)), S(0) = Q, the
reflection symmetry S(r) = S(L - r), and closed forms on constructed lattices."""
import numpy as np
import pytest


def _fft_autocorr(s, axis):
    f = np.fft.fft(s.astype(np.float64), axis=axis)
    return np.rint(np.fft.ifft(f * np.conj(f), axis=axis).real.sum(axis=1 - axis)).astype(np.int64)


@pytest.mark.parametrize("L,vals", [(16, (-1, 1)), (24, (-1, 0, 1)), (64, (-1, 1))])
def test_correlation_matches_fft_autocorrelation(orc, L, vals):
    rng = np.random.default_rng(L)
    s = rng.choice(vals, size=(L, L)).astype(np.int8)
    r = np.arange(L)
    sx, sy = orc.correlation(s, r)
    # s[y, x]: the x direction is axis 1, y is axis 0
    assert np.array_equal(sx, _fft_autocorr(s, 1))
    assert np.array_equal(sy, _fft_autocorr(s, 0))
    assert np.array_equal(sx[1:], sx[1:][::-1]) and np.array_equal(sy[1:], sy[1:][::-1])


def test_correlation_identities_with_measure(orc):
    for model in (0, 1):
        s = orc.init_random(48, model, 3)
        orc.run(s, model, 3, 0, [0.5] * 5)
        B, M, Q, _, _ = orc.measure(s)
        sx, sy = orc.correlation(s, [0, 1])
        assert sx[0] == Q and sy[0] == Q
        assert sx[1] + sy[1] == B


def test_correlation_constructed_lattices(orc):
    L = 32
    y, x = np.indices((L, L))
    neel = (1 - 2 * ((x + y) & 1)).astype(np.int8)
    r = np.arange(L)
    sx, sy = orc.correlation(neel, r)
    want = (L * L) * (1 - 2 * (r & 1))
    assert np.array_equal(sx, want) and np.array_equal(sy, want)
    stripes = (1 - 2 * (x & 1)).astype(np.int8)          # alternate along x only
    sx, sy = orc.correlation(stripes, r)
    assert np.array_equal(sx, want) and np.all(sy == L * L)
