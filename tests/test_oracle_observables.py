"""Pins for the oracle's observables: the bond sum behind E (Eqs. (2)-(3)),
M and Q, the row/column sums, and the second-moment correlation length
xi_2 of Appendix B.

Pins: constructed lattices whose sums are known in closed form, invariants
(sum R = sum C = M), the energy of a single defect, and for xi_2 the closed
form of a single Fourier mode plus agreement with a library FFT.
"""
import math

import numpy as np
import pytest


def _lattice(f, L):
    y, x = np.indices((L, L))
    return np.ascontiguousarray(f(x, y).astype(np.int8))


@pytest.mark.parametrize("L", [4, 6, 64])
def test_measure_constructed_lattices(orc, L):
    N = L * L
    up = _lattice(lambda x, y: np.ones_like(x), L)
    B, M, Q, R, C = orc.measure(up)
    assert (B, M, Q) == (2 * N, N, N) and np.all(R == L) and np.all(C == L)
    neel = _lattice(lambda x, y: 1 - 2 * ((x + y) & 1), L)
    B, M, Q, R, C = orc.measure(neel)
    assert (B, M, Q) == (-2 * N, 0, N) and np.all(R == 0) and np.all(C == 0)
    # vertical stripes: horizontal bonds anti-aligned, vertical bonds aligned
    stripes = _lattice(lambda x, y: 1 - 2 * (x & 1), L)
    B, M, Q, R, C = orc.measure(stripes)
    assert (B, M, Q) == (0, 0, N)
    assert np.all(R == 0) and np.array_equal(C, L * (1 - 2 * (np.arange(L) & 1)))
    # horizontal stripes of +1 / 0 (Blume-Capel vacancies on odd rows)
    vac = _lattice(lambda x, y: 1 - (y & 1), L)
    B, M, Q, R, C = orc.measure(vac)
    assert (B, M, Q) == (N // 2, N // 2, N // 2)
    assert np.array_equal(R, L * (1 - (np.arange(L) & 1))) and np.all(C == L // 2)


def test_measure_single_defect(orc):
    L = 16
    s = np.ones((L, L), dtype=np.int8)
    s[3, 5] = -1
    B, M, Q, R, C = orc.measure(s)
    assert (B, M, Q) == (2 * L * L - 8, L * L - 2, L * L)
    assert R[3] == L - 2 and C[5] == L - 2 and R.sum() == M and C.sum() == M
    s[3, 5] = 0
    B, M, Q, R, C = orc.measure(s)
    assert (B, M, Q) == (2 * L * L - 4, L * L - 1, L * L - 1)


def test_measure_invariants_random(orc):
    rng = np.random.default_rng(5)
    for L in (8, 30, 64):
        s = rng.integers(-1, 2, size=(L, L)).astype(np.int8)
        B, M, Q, R, C = orc.measure(s)
        assert R.sum() == M and C.sum() == M and Q == int((s != 0).sum())
        # translation invariance of B, M, Q; transposition swaps R and C
        B2, M2, Q2, R2, C2 = orc.measure(np.ascontiguousarray(np.roll(s, (3, 5), (0, 1))))
        assert (B2, M2, Q2) == (B, M, Q)
        B3, M3, Q3, R3, C3 = orc.measure(np.ascontiguousarray(s.T))
        assert (B3, M3, Q3) == (B, M, Q) and np.array_equal(R3, C) and np.array_equal(C3, R)


def test_xi2_single_mode_closed_form(orc):
    """L = 4, sums a + b cos(2 pi x / 4): M = 4a, |M(k)| = 2b, so
    xi_2 = sqrt(4 a^2 / b^2 - 1) / (2 sin(pi / 4))."""
    for a, b in [(3, 1), (5, 2), (10, 7)]:
        C = np.array([a + b, a, a - b, a], dtype=np.int32)
        R = C.copy()
        M = 4 * a
        want = math.sqrt(4 * a * a / (b * b) - 1) / (2 * math.sin(math.pi / 4))
        assert abs(orc.xi2([M], R[None], C[None]) - want) <= 1e-14 * want


def test_xi2_matches_library_fft(orc):
    rng = np.random.default_rng(1)
    for L in (8, 64, 1024, 1000):
        n = 7
        R = rng.integers(-L, L + 1, size=(n, L)).astype(np.int32) + 3 * L // 4
        C = rng.integers(-L, L + 1, size=(n, L)).astype(np.int32) + 3 * L // 4
        M = R.sum(axis=1).astype(np.int64)
        s0 = np.mean(M.astype(np.float64) ** 2)
        sk = np.mean(0.5 * (np.abs(np.fft.fft(C, axis=1)[:, 1]) ** 2 +
                            np.abs(np.fft.fft(R, axis=1)[:, 1]) ** 2))
        want = math.sqrt(s0 / sk - 1) / (2 * math.sin(math.pi / L))
        got = orc.xi2(M, R, C)
        assert abs(got - want) <= 1e-9 * want, (L, got, want)


def test_xi2_degenerate_cases(orc):
    L = 16
    # uniform sums: no k_min component, xi infinite
    R = np.full((1, L), 4, dtype=np.int32)
    assert orc.xi2([4 * L], R, R) == math.inf
    # M = 0 with fluctuations: <S0> <= <Sk>, undefined
    R = np.zeros((1, L), dtype=np.int32)
    R[0, 0], R[0, 1] = 5, -5
    assert math.isnan(orc.xi2([0], R, R))
    # ensemble average: a replica with M = 0 lowers <S0> only
    Rp = np.array([[2] * L], dtype=np.int32)
    Rp[0, 0] += 3
    x1 = orc.xi2([int(Rp.sum())], Rp, Rp)
    x2 = orc.xi2([int(Rp.sum()), int(Rp.sum())], np.vstack([Rp, Rp]), np.vstack([Rp, Rp]))
    assert x1 == x2
