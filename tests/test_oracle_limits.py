"""Pins for the oracle from the deterministic limits of the dynamics.

* beta = 0 (T = infinity): every Ising move is accepted, so one sweep negates
  every spin exactly.
* beta = infinity (T -> 0): only dE <= 0 moves are accepted, so the energy of
  Eq. (1) never increases; the ground state is a fixed point and a single
  defect in it heals within one sweep.
* Global spin flip (Ising): Eq. (1) is even in s and the random words are keyed
  by site, not by spin, so the trajectory from -s is exactly the negated one.
* A changed seed or sweep index changes the trajectory; the same ones repeat it.
* Threads: rows of one colour are independent for even L, so splitting them
  among threads gives the identical result.
"""
import math

import numpy as np
import pytest


def test_beta_zero_sweep_negates_ising(orc):
    s = orc.init_random(64, orc.ISING, 3)
    s0 = s.copy()
    orc.run(s, orc.ISING, 3, 0, [0.0])
    assert np.array_equal(s, -s0)
    B0, M0, *_ = orc.measure(s0)
    B1, M1, *_ = orc.measure(s)
    assert M1 == -M0 and B1 == B0


@pytest.mark.parametrize("model,delta", [(0, 0.0), (1, 0.0), (1, 0.7)])
def test_beta_infinity_energy_never_increases(orc, model, delta):
    L = 64
    s = orc.init_random(L, model, 11)
    bmq, _, _ = orc.run(s, model, 11, 0, [math.inf] * 60, delta=delta, record_every=1,
                        with_rows=False)
    energy = -bmq[:, 0] + delta * bmq[:, 2]
    assert np.all(np.diff(energy) <= 1e-9)
    assert energy[-1] < energy[0]


@pytest.mark.parametrize("model", [0, 1])
def test_ground_state_fixed_and_defect_heals(orc, model):
    L = 32
    s = np.ones((L, L), dtype=np.int8)
    orc.run(s, model, 5, 0, [math.inf] * 3)
    assert np.all(s == 1)
    for (x, y) in [(4, 6), (5, 6)]:  # one defect on each colour
        s = np.ones((L, L), dtype=np.int8)
        s[y, x] = -1
        # Ising: the defect flips back at its own half-sweep.  Blume-Capel: the
        # move -1 -> 0 or -1 -> +1 is downhill, and 0 -> +1 is too, so the
        # defect is gone after each of its proposals has picked +1 once.
        sweeps = 1 if model == 0 else 40
        orc.run(s, model, 5, 0, [math.inf] * sweeps)
        assert np.all(s == 1), (x, y)


def test_global_spin_flip_symmetry_ising(orc):
    L, seed = 64, 99
    a = orc.init_random(L, orc.ISING, seed)
    b = (-a).astype(np.int8)
    betas = [0.44068679350977147] * 25
    ra = orc.run(a, orc.ISING, seed, 0, betas, record_every=1)
    rb = orc.run(b, orc.ISING, seed, 0, betas, record_every=1)
    assert np.array_equal(b, -a)
    assert np.array_equal(ra[0][:, 0], rb[0][:, 0])      # B even
    assert np.array_equal(ra[0][:, 1], -rb[0][:, 1])     # M odd
    assert np.array_equal(ra[1], -rb[1]) and np.array_equal(ra[2], -rb[2])


@pytest.mark.parametrize("model", [0, 1])
def test_keying_seed_and_sweep_index(orc, model):
    L = 64
    base = orc.init_random(L, model, 1)
    outs = {}
    for seed, t0 in [(1, 0), (1, 0), (2, 0), (1, 5)]:
        s = base.copy()
        orc.run(s, model, seed, t0, [0.5] * 3)
        outs.setdefault((seed, t0), []).append(s)
    assert np.array_equal(*outs[(1, 0)])
    assert not np.array_equal(outs[(1, 0)][0], outs[(2, 0)][0])
    assert not np.array_equal(outs[(1, 0)][0], outs[(1, 5)][0])


@pytest.mark.parametrize("model", [0, 1])
def test_split_runs_equal_one_run(orc, model):
    """n1 sweeps then n2 sweeps (t0 = n1) equal n1+n2 sweeps in one call."""
    L = 64
    a = orc.init_random(L, model, 21)
    b = a.copy()
    betas = np.linspace(0.3, 0.7, 20)
    orc.run(a, model, 21, 0, betas)
    orc.run(b, model, 21, 0, betas[:7])
    orc.run(b, model, 21, 7, betas[7:])
    assert np.array_equal(a, b)


@pytest.mark.parametrize("model", [0, 1])
def test_threads_do_not_change_result(orc, model):
    L = 128
    a = orc.init_random(L, model, 4)
    b = a.copy()
    orc.run(a, model, 4, 0, [0.45] * 10, nthreads=1)
    orc.run(b, model, 4, 0, [0.45] * 10, nthreads=4)
    assert np.array_equal(a, b)
