"""Pins for the oracle's Metropolis acceptance (Introduction: the update is
Metropolis; Appendix B: 32-bit integer random numbers).

* thresholds against the closed form min(1, e^{-beta dE}) within the rounding
  bound of the integer grid, and the beta = 0 / beta = infinity limits;
* measured acceptance frequencies of the checkerboard sweep against
  e^{-beta dE}, class by class, for both models.  Colour-0 sites are updated
  in the first half of a sweep while their colour-1 neighbours are frozen, so
  their energy class is known from the lattice before the sweep and their
  acceptance from the lattice after it.
"""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("bits", [31, 32])
@pytest.mark.parametrize("beta", [0.05, 0.44068679350977147, 1 / 1.6938, 1.0, 3.0])
def test_threshold_closed_form(orc, bits, beta):
    for dE in [0.5, 1.0, 2.0, 3.0, 4.0, 6.0, 8.0, 7.25]:
        thr = orc.threshold(beta, dE, bits)
        p = math.exp(-beta * dE)
        assert abs(thr / 2.0 ** bits - p) <= 2.0 ** -(bits + 1) * (1 + 1e-12)
        assert 0 <= thr <= 2 ** bits


@pytest.mark.parametrize("bits", [31, 32])
def test_threshold_limits(orc, bits):
    # beta = 0: every move accepted; dE <= 0 always accepted
    assert orc.threshold(0.0, 8.0, bits) == 2 ** bits
    assert orc.threshold(0.7, 0.0, bits) == 2 ** bits
    assert orc.threshold(0.7, -4.0, bits) == 2 ** bits
    # beta = infinity (T -> 0): no uphill move accepted
    assert orc.threshold(math.inf, 4.0, bits) == 0
    # monotone in dE
    thr = [orc.threshold(0.5, dE, bits) for dE in range(1, 9)]
    assert all(a >= b for a, b in zip(thr, thr[1:]))


def _colour0_mask(L):
    y, x = np.indices((L, L))
    return ((x + y) & 1) == 0


def _nbr_sum(s):
    return (np.roll(s, 1, 0) + np.roll(s, -1, 0) + np.roll(s, 1, 1) + np.roll(s, -1, 1)).astype(np.int64)


def test_ising_acceptance_frequencies(orc):
    L, beta, seed = 64, 0.3, 0x2503146880000001
    s = orc.init_random(L, orc.ISING, seed)
    c0 = _colour0_mask(L)
    acc = {}
    for t in range(300):
        before = s.copy()
        orc.run(s, orc.ISING, seed, t, [beta])
        dE = 2 * before.astype(np.int64) * _nbr_sum(before)
        flipped = before != s
        for e in (-8, -4, 0, 4, 8):
            sel = c0 & (dE == e)
            a, n = acc.get(e, (0, 0))
            acc[e] = (a + int(flipped[sel].sum()), n + int(sel.sum()))
    for e, (a, n) in acc.items():
        assert n > 1000
        p = 1.0 if e <= 0 else math.exp(-beta * e)
        if p == 1.0:
            assert a == n
        else:
            assert abs(a / n - p) < 4.5 * math.sqrt(p * (1 - p) / n), (e, a, n, p)


@pytest.mark.parametrize("beta,delta", [(1 / 1.6938, 0.0), (0.8, 0.5)])
def test_blume_capel_acceptance_frequencies(orc, beta, delta):
    """P(s -> s' | s, h) = 1/2 min(1, e^{-beta dE}) for each of the two proposals."""
    L, seed = 64, 0x2503146880000002
    s = orc.init_random(L, orc.BLUME_CAPEL, seed)
    c0 = _colour0_mask(L)
    counts = {}
    for t in range(300):
        before = s.copy()
        orc.run(s, orc.BLUME_CAPEL, seed, t, [beta], delta=delta)
        h = _nbr_sum(before)
        for sv in (-1, 0, 1):
            for hv in range(-4, 5):
                sel = c0 & (before == sv) & (h == hv)
                n = int(sel.sum())
                if n == 0:
                    continue
                after = s[sel]
                for s2 in (-1, 0, 1):
                    if s2 == sv:
                        continue
                    key = (sv, hv, s2)
                    a0, n0 = counts.get(key, (0, 0))
                    counts[key] = (a0 + int((after == s2).sum()), n0 + n)
    checked = 0
    for (sv, hv, s2), (a, n) in counts.items():
        if n < 2000:
            continue
        dE = -(s2 - sv) * hv + delta * (s2 * s2 - sv * sv)
        p = 0.5 * min(1.0, math.exp(-beta * dE))
        assert abs(a / n - p) < 4.5 * math.sqrt(p * (1 - p) / n) + 1e-12, (sv, hv, s2, a, n, p)
        checked += 1
    assert checked >= 20


def test_bc_proposal_rule(orc):
    """s' is the (b+1)-th smallest of the two values other than s."""
    for sv in (-1, 0, 1):
        others = sorted(v for v in (-1, 0, 1) if v != sv)
        assert [orc.bc_proposal(sv, b) for b in (0, 1)] == others


def test_hot_start_statistics(orc):
    """T = infinity start: Ising +-1 with 1/2 each; Blume-Capel 1/3 each."""
    L = 512
    s = orc.init_random(L, orc.ISING, 7)
    n = L * L
    assert set(np.unique(s)) == {-1, 1}
    assert abs((s == 1).mean() - 0.5) < 4 * math.sqrt(0.25 / n)
    b = orc.init_random(L, orc.BLUME_CAPEL, 7)
    for v in (-1, 0, 1):
        assert abs((b == v).mean() - 1 / 3) < 4 * math.sqrt(2 / 9 / n)
    # nearest-neighbour correlation of a T = infinity state vanishes
    B, M, Q, _, _ = orc.measure(s)
    assert abs(B) < 4 * math.sqrt(2 * n)
    # a different seed gives a different lattice; the same seed the same one
    assert not np.array_equal(s, orc.init_random(L, orc.ISING, 8))
    assert np.array_equal(s, orc.init_random(L, orc.ISING, 7))
