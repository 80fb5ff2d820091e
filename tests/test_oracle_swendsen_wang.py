"""Pins for the oracle's Swendsen-Wang iteration (Appendix B: cluster updates
of the s = +-1 spins, combined with Metropolis sweeps for Blume-Capel).

* the bond threshold against its closed form and limits;
* the clusters against networkx's connected components of the active-bond
  graph, the bonds drawn here from the (cuRAND-pinned) Philox4x32-10 with the
  keying the oracle documents; labels = smallest site index; the flip of each
  cluster against its root's coin; vacancies untouched;
* beta = 0 (no bond: every +-1 site alone) and beta -> infinity (every
  aligned pair bonded: clusters = geometric domains);
* stationarity: long chains reproduce exact enumeration: Ising L = 4 under
  Swendsen-Wang alone, Blume-Capel L = 4 under Metropolis sweep + Swendsen-
  Wang steps (the Swendsen-Wang part alone cannot change s^2).
"""
import math

import networkx as nx
import numpy as np
import pytest

import exact
from conftest import binned_mean_sem

BETA_C = math.log(1 + math.sqrt(2)) / 2
Z_MAX = 4.5


def _word(orc, seed, i, k, w3):
    q = i >> 2
    out = orc.philox4x32_10([q & 0xFFFFFFFF, q >> 32, k, w3], [seed & 0xFFFFFFFF, seed >> 32])
    return int(out[i & 3])


def _expected(orc, s, seed, k, beta):
    """Clusters and the flipped lattice, from networkx components of the
    active bonds."""
    L = s.shape[0]
    thr = orc.sw_threshold(beta)
    g = nx.Graph()
    g.add_nodes_from(range(L * L))
    for y in range(L):
        for x in range(L):
            i = y * L + x
            if s[y, x] == 0:
                continue
            for d, (yy, xx) in enumerate(((y, (x + 1) % L), ((y + 1) % L, x))):
                if s[yy, xx] == s[y, x] and _word(orc, seed, i, k, 4 + d) < thr:
                    g.add_edge(i, yy * L + xx)
    labels = np.empty(L * L, dtype=np.int64)
    flipped = s.copy().reshape(-1)
    n = 0
    for comp in nx.connected_components(g):
        r = min(comp)
        for i in comp:
            labels[i] = r
        if s.reshape(-1)[r] != 0:
            n += 1
            if _word(orc, seed, r, k, 6) >= 2 ** 31:
                for i in comp:
                    flipped[i] = -flipped[i]
    return labels.reshape(L, L), flipped.reshape(L, L), n


def test_bond_threshold_closed_form(orc):
    assert orc.sw_threshold(0.0) == 0
    assert orc.sw_threshold(40.0) == 2 ** 32
    for beta in (1e-6, 0.1, BETA_C, 0.7, 2.0):
        thr = orc.sw_threshold(beta)
        assert abs(thr / 2 ** 32 - (1 - math.exp(-2 * beta))) <= 2 ** -33 * (1 + 1e-9)


@pytest.mark.parametrize("model,L,beta", [(0, 8, 0.3), (0, 12, BETA_C), (0, 10, 0.8),
                                          (1, 8, 0.6), (1, 12, 1 / 1.6938), (1, 6, 1.5)])
def test_clusters_and_flips_against_networkx(orc, model, L, beta):
    seed = 0x2503146880000000 + 77 * L + model
    s = orc.init_random(L, model, seed)
    for k in range(4):
        before = s.copy()
        want_labels, want_s, want_n = _expected(orc, before, seed, k, beta)
        labels, n = orc.swendsen_wang(s, seed, k, beta)
        assert np.array_equal(labels, want_labels), k
        assert n == want_n
        assert np.array_equal(s, want_s), k
        assert np.array_equal(before == 0, s == 0)          # vacancies stay
        # interleave Metropolis sweeps so the next iteration sees a new state
        orc.run(s, model, seed, k, [beta])


def test_beta_zero_and_infinity(orc):
    seed, L = 0x2503146880000091, 10
    s = orc.init_random(L, 1, seed)
    labels, n = orc.swendsen_wang(s.copy(), seed, 0, 0.0)
    assert np.array_equal(labels.reshape(-1), np.arange(L * L))
    assert n == int(np.count_nonzero(s))
    # p = 1: every aligned +-1 pair bonded, clusters = domains of equal spins
    g = nx.Graph()
    g.add_nodes_from(range(L * L))
    for y in range(L):
        for x in range(L):
            for yy, xx in ((y, (x + 1) % L), ((y + 1) % L, x)):
                if s[y, x] != 0 and s[yy, xx] == s[y, x]:
                    g.add_edge(y * L + x, yy * L + xx)
    labels, n = orc.swendsen_wang(s.copy(), seed, 0, 40.0)
    for comp in nx.connected_components(g):
        assert {int(labels.reshape(-1)[i]) for i in comp} == {min(comp)}
    # a uniform Ising lattice is one cluster: all spins flip or none
    u = np.ones((8, 8), dtype=np.int8)
    flips = set()
    for k in range(8):
        v = u.copy()
        _, n = orc.swendsen_wang(v, seed, k, 40.0)
        assert n == 1 and abs(int(v.sum())) == 64
        flips.add(int(v[0, 0]))
    assert flips == {-1, 1}


def _check(name, series, want):
    mean, sem = binned_mean_sem(series)
    z = (mean - want) / sem
    assert abs(z) < Z_MAX, f"{name}: {mean:.6f} +- {sem:.6f}, exact {want:.6f}, z={z:.2f}"


@pytest.mark.parametrize("beta", [0.2, BETA_C, 0.6])
def test_ising_L4_swendsen_wang_matches_enumeration(orc, beta):
    L, n, seed = 4, 60_000, 0x2503146880000095
    s = orc.init_random(L, 0, seed)
    e, m = np.empty(n), np.empty(n)
    for k in range(n + 200):
        orc.swendsen_wang(s, seed, k, beta)
        if k >= 200:
            B, M = orc.measure(s)[:2]
            e[k - 200], m[k - 200] = -B / 16, M / 16
    ex = exact.enumerate_ising(L, beta)
    _check("e", e, ex["e"])
    _check("|m|", np.abs(m), ex["absm"])
    _check("m^2", m ** 2, ex["m2"])
    _check("m^4", m ** 4, ex["m4"])


@pytest.mark.parametrize("T,delta", [(1.6938, 0.0), (1.0, 0.5)])
def test_blume_capel_L4_sweep_plus_sw_matches_enumeration(orc, T, delta):
    L, n, seed, beta = 4, 40_000, 0x2503146880000096, 1 / T
    s = orc.init_random(L, 1, seed)
    e, m, q = np.empty(n), np.empty(n), np.empty(n)
    for k in range(n + 200):
        orc.run(s, 1, seed, k, [beta], delta=delta)
        orc.swendsen_wang(s, seed, k, beta)
        if k >= 200:
            B, M, Q = orc.measure(s)[:3]
            e[k - 200], m[k - 200], q[k - 200] = (-B + delta * Q) / 16, M / 16, Q / 16
    ex = exact.enumerate_blume_capel(L, beta, delta)
    _check("e", e, ex["e"])
    _check("|m|", np.abs(m), ex["absm"])
    _check("m^2", m ** 2, ex["m2"])
    _check("q", q, ex["q"])
