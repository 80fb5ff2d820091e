"""Pins for the oracle's dynamics from exact equilibrium results.

A correct Metropolis chain (Introduction; Table I) has the Boltzmann
distribution of Eq. (1) as its stationary law, so long-run means of the
oracle must agree, within their binned statistical error, with:

* brute-force enumeration: Ising L = 4 (2^16 states), Blume-Capel L = 3
  (3^9 states, sequential visiting order since L is odd) and L = 4 (3^16
  states, the true checkerboard);
* Kaufman's exact finite-L energy of the Ising torus at beta_c, whose
  L -> infinity limit is the paper's E_eq(T_c) = -sqrt(2) (Results);
* Onsager's energy and Yang's magnetisation off criticality at L = 128,
  where finite-size corrections are exponentially small.
"""
import math

import numpy as np
import pytest

import exact
from conftest import binned_mean_sem

BETA_C = math.log(1 + math.sqrt(2)) / 2
Z_MAX = 4.5


def _check(name, got_series, want):
    mean, sem = binned_mean_sem(got_series)
    z = (mean - want) / sem
    assert abs(z) < Z_MAX, f"{name}: oracle {mean:.6f} +- {sem:.6f}, exact {want:.6f}, z={z:.2f}"


def test_enumeration_helpers_agree():
    """The row-by-row Blume-Capel sum equals a direct sum over 3^9 states."""
    L, beta, delta = 3, 0.7, 0.3
    codes = np.arange(3 ** 9)
    sp = exact._spins_from_codes(codes, 9, 3) - 1
    B = exact._bond_sum(sp, L)
    Q = (sp * sp).sum(axis=1)
    w = np.exp(beta * B - beta * delta * Q)
    e_direct = float((w * (-B + delta * Q)).sum() / w.sum() / 9)
    assert abs(exact.enumerate_blume_capel(3, beta, delta)["e"] - e_direct) < 1e-12
    # beta = 0: each site uniform on {-1,0,1}
    assert abs(exact.enumerate_blume_capel(3, 0.0, 0.0)["q"] - 2 / 3) < 1e-12


def test_kaufman_matches_enumeration_and_limit():
    for beta in (0.2, BETA_C, 0.6):
        assert abs(exact.kaufman_energy(4, beta) - exact.enumerate_ising(4, beta)["e"]) < 1e-12
    # L -> infinity at beta_c: the paper's -sqrt 2, approached as c1/L
    e256, e1024 = exact.kaufman_energy(256, BETA_C), exact.kaufman_energy(1024, BETA_C)
    assert abs(e1024 + math.sqrt(2)) < 1e-3
    assert abs((e256 + math.sqrt(2)) * 256 - (e1024 + math.sqrt(2)) * 1024) < 1e-3
    for beta in (0.3, 0.6):
        assert abs(exact.kaufman_energy(128, beta) - exact.onsager_energy(beta)) < 1e-12


@pytest.mark.parametrize("beta", [0.2, BETA_C, 0.6])
def test_ising_L4_matches_enumeration(orc, beta):
    L, n = 4, 400_000
    s = orc.init_random(L, orc.ISING, 0x2503146880000011)
    orc.run(s, orc.ISING, 0x2503146880000011, 0, [beta] * 1000)
    bmq, _, _ = orc.run(s, orc.ISING, 0x2503146880000011, 1000, [beta] * n,
                        record_every=1, with_rows=False)
    ex = exact.enumerate_ising(L, beta)
    N = L * L
    _check("e", -bmq[:, 0] / N, ex["e"])
    _check("|m|", np.abs(bmq[:, 1]) / N, ex["absm"])
    _check("m^2", (bmq[:, 1] / N) ** 2, ex["m2"])
    _check("m^4", (bmq[:, 1] / N) ** 4, ex["m4"])


@pytest.mark.parametrize("T,delta", [(1.0, 0.0), (1.6938, 0.0), (3.0, 0.0), (1.0, 0.5),
                                     (1.6938, 0.5)])
def test_blume_capel_L3_matches_enumeration(orc, T, delta):
    L, n, beta = 3, 400_000, 1 / T
    seed = 0x2503146880000012
    s = orc.init_random(L, orc.BLUME_CAPEL, seed)
    orc.run(s, orc.BLUME_CAPEL, seed, 0, [beta] * 1000, delta=delta)
    bmq, _, _ = orc.run(s, orc.BLUME_CAPEL, seed, 1000, [beta] * n, delta=delta,
                        record_every=1, with_rows=False)
    ex = exact.enumerate_blume_capel(L, beta, delta)
    N = L * L
    _check("e", (-bmq[:, 0] + delta * bmq[:, 2]) / N, ex["e"])
    _check("|m|", np.abs(bmq[:, 1]) / N, ex["absm"])
    _check("m^2", (bmq[:, 1] / N) ** 2, ex["m2"])
    _check("q", bmq[:, 2] / N, ex["q"])


@pytest.mark.parametrize("T,delta", [(1.6938, 0.0), (1.0, 0.5)])
def test_blume_capel_L4_matches_enumeration(orc, T, delta):
    L, n, beta = 4, 300_000, 1 / T
    seed = 0x2503146880000013
    s = orc.init_random(L, orc.BLUME_CAPEL, seed)
    orc.run(s, orc.BLUME_CAPEL, seed, 0, [beta] * 1000, delta=delta)
    bmq, _, _ = orc.run(s, orc.BLUME_CAPEL, seed, 1000, [beta] * n, delta=delta,
                        record_every=1, with_rows=False)
    ex = exact.enumerate_blume_capel(L, beta, delta)
    N = L * L
    _check("e", (-bmq[:, 0] + delta * bmq[:, 2]) / N, ex["e"])
    _check("|m|", np.abs(bmq[:, 1]) / N, ex["absm"])
    _check("m^2", (bmq[:, 1] / N) ** 2, ex["m2"])
    _check("q", bmq[:, 2] / N, ex["q"])


def test_ising_L32_energy_at_beta_c_matches_kaufman(orc):
    """Finite-L exact energy at T_c (-> -sqrt 2 + c1/L, Results)."""
    L, n = 32, 100_000
    seed = 0x2503146880000014
    s = np.ones((L, L), dtype=np.int8)
    orc.run(s, orc.ISING, seed, 0, [BETA_C] * 5000, nthreads=4)
    bmq, _, _ = orc.run(s, orc.ISING, seed, 5000, [BETA_C] * n, record_every=1,
                        with_rows=False, nthreads=4)
    _check("e(beta_c)", -bmq[:, 0] / (L * L), exact.kaufman_energy(L, BETA_C))


@pytest.mark.parametrize("beta,cold", [(0.3, False), (0.6, True)])
def test_ising_L128_onsager_and_yang(orc, beta, cold):
    L, n = 128, 3000
    seed = 0x2503146880000015
    s = np.ones((L, L), dtype=np.int8) if cold else orc.init_random(L, orc.ISING, seed)
    orc.run(s, orc.ISING, seed, 0, [beta] * 500, nthreads=4)
    bmq, _, _ = orc.run(s, orc.ISING, seed, 500, [beta] * n, record_every=1,
                        with_rows=False, nthreads=4)
    N = L * L
    _check("e", -bmq[:, 0] / N, exact.onsager_energy(beta))
    if cold:
        _check("|m|", np.abs(bmq[:, 1]) / N, exact.yang_magnetisation(beta))
