"""Host analysis of the critical-temperature study (paper_2503_14688_b300.tc),
pinned on exactly solvable inputs:

  * reweighting: samples drawn from the exact Boltzmann distribution of the
    Ising L = 4 torus at beta0 (all 2^16 states enumerated), reweighted to
    beta1, reproduce the exact U4 and xi_2 at beta1;
  * the crossing of U4 with a target, on the same samples, equals the
    crossing of the exact U4(beta) curve;
  * observables at beta0 equal the plain averages, xi_2 equal to the
    library's isg_xi2 on the same integers;
  * the constant fit is the weighted mean.
"""
import math

import numpy as np
import pytest

import exact
from paper_2503_14688_b300 import tc

L = 4


def _states():
    n = L * L
    codes = np.arange(2 ** n, dtype=np.int64)
    sp = 2 * exact._spins_from_codes(codes, n, 2) - 1          # (states, 16)
    B = exact._bond_sum(sp, L).astype(np.float64)
    g = sp.reshape(-1, L, L)
    M = sp.sum(axis=1).astype(np.float64)
    R = g.sum(axis=2).astype(np.float64)                        # row sums R[y]
    C = g.sum(axis=1).astype(np.float64)                        # column sums C[x]
    ph = np.exp(2j * np.pi * np.arange(L) / L)
    Sk = 0.5 * (np.abs(C @ ph) ** 2 + np.abs(R @ ph) ** 2)
    return B, M, R, C, Sk


def _exact(beta, B, M, Sk):
    w = np.exp(beta * (B - B.max()))
    w /= w.sum()
    m2, m4, sk = w @ M ** 2, w @ M ** 4, w @ Sk
    xi = math.sqrt(m2 / sk - 1) / (2 * math.sin(math.pi / L))
    return m4 / m2 ** 2, xi / L


def _samples(beta0, n, seed=3):
    B, M, R, C, Sk = _states()
    w = np.exp(beta0 * (B - B.max()))
    idx = np.random.default_rng(seed).choice(B.size, size=n, p=w / w.sum())
    return tc.Samples(L, beta0, B[idx].reshape(8, -1), M[idx].reshape(8, -1),
                      Sk[idx].reshape(8, -1)), (B, M, R, C, Sk), idx


def test_reweighting_reproduces_exact_averages():
    s, (B, M, R, C, Sk), _ = _samples(0.40, 800_000)
    for beta1 in (0.36, 0.40, 0.44):
        u4, xi = tc.observables(s, beta1)
        u4x, xix = _exact(beta1, B, M, Sk)
        assert u4 == pytest.approx(u4x, abs=4e-3)
        assert xi == pytest.approx(xix, abs=4e-3)


def test_plain_averages_at_beta0_and_xi2_of_the_library():
    import paper_2503_14688_b300 as P

    s, (B, M, R, C, Sk), idx = _samples(0.40, 4000, seed=5)
    u4, xi = tc.observables(s, 0.40)
    m = s.M.reshape(-1)
    assert u4 == pytest.approx((m ** 4).mean() / (m ** 2).mean() ** 2, rel=1e-12)
    want = P.xi2(M[idx].astype(np.int64), R[idx].astype(np.int32), C[idx].astype(np.int32)) / L
    assert xi == pytest.approx(want, rel=1e-9)


def test_crossing_matches_exact_curve():
    from scipy.optimize import brentq

    B, M, R, C, Sk = _states()
    target = 1.4
    beta_x = brentq(lambda b: _exact(b, B, M, Sk)[0] - target, 0.2, 0.8, xtol=1e-12)
    s, _, _ = _samples(beta_x + 0.01, 800_000, seed=9)
    got = tc.crossing(s, "u4", span=0.05, target=target)
    assert got == pytest.approx(beta_x, abs=2e-3)


def test_constant_fit_is_weighted_mean():
    m, e, c = tc.constant_fit([1.0, 2.0, 4.0], [1.0, 0.5, 2.0])
    w = np.array([1.0, 4.0, 0.25])
    want = float((w * np.array([1.0, 2.0, 4.0])).sum() / w.sum())
    assert m == pytest.approx(want, rel=1e-14)
    assert e == pytest.approx(1 / math.sqrt(w.sum()), rel=1e-14)
    assert c == pytest.approx(float((w * (np.array([1.0, 2.0, 4.0]) - want) ** 2).sum()) / 2)
