"""The GPU Swendsen-Wang iteration (isg_swendsen_wang; Appendix B) against
the oracle, and its physics.

Parity: cluster labels (smallest site index) and spins equal the oracle's
after every iteration, interleaved with Metropolis sweeps, for both models,
several temperatures (beta = 0 and the always-bond limit included) and sizes
up to L = 1024; the iteration count survives a checkpoint.

Physics: the elementary Monte Carlo step of Appendix B (10 Metropolis
sweeps + one Swendsen-Wang iteration) at the paper's T_c of Blume-Capel,
and pure Swendsen-Wang for Ising at beta_c, reproduce the universal
U4* = 1.1679229 and (xi_2/L)* = 0.9050488 at L = 128.
"""
import math
import os

import numpy as np
import pytest

from paper_2503_14688_b300 import workloads as wl

pytestmark = pytest.mark.gpu

U4_STAR = 1.1679229
XI_STAR = 0.9050488292


@pytest.fixture(scope="module")
def isg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2503_14688_b300 import build

    build.build()
    import paper_2503_14688_b300 as P

    return P


CASES = [(0, 64, 0.3, 0.0), (0, 128, wl.BETA_C_ISING, 0.0), (0, 64, 0.8, 0.0),
         (1, 64, 1 / 1.6938, 0.0), (1, 128, 1 / wl.T_C_BLUME_CAPEL, 0.3), (1, 64, 1.5, 0.0),
         (0, 64, 0.0, 0.0), (1, 64, 40.0, 0.0)]


@pytest.mark.parametrize("model,L,beta,delta", CASES)
def test_labels_and_spins_match_oracle(isg, orc, model, L, beta, delta):
    seed = wl.BASE_SEED + 500 + 7 * L + model
    lat = isg.Lattice(L, model, seed=seed, delta=delta)
    lat.init_random()
    s = orc.init_random(L, model, seed)
    mb = max(beta, 0.1) if beta < 40 else 2.0  # Metropolis beta between iterations
    for k in range(6):
        lat.sweep(2, beta=mb)
        orc.run(s, model, seed, 2 * k, [mb, mb], delta=delta)
        lat.swendsen_wang(beta)
        labels, _ = orc.swendsen_wang(s, seed, k, beta)
        assert np.array_equal(lat.sw_labels(), labels.astype(np.int32)), k
        assert np.array_equal(lat.get(), s), k
    assert lat.sw_iterations == 6
    lat.close()


@pytest.mark.parametrize("model", [0, 1])
def test_large_lattice_matches_oracle(isg, orc, model):
    L, seed = 1024, wl.BASE_SEED + 611 + model
    beta = wl.BETA_C_ISING if model == 0 else 1 / wl.T_C_BLUME_CAPEL
    lat = isg.Lattice(L, model, seed=seed)
    lat.init_random()
    s = orc.init_random(L, model, seed)
    threads = os.cpu_count() or 1
    for k in range(3):
        lat.sweep(5, beta=beta)
        orc.run(s, model, seed, 5 * k, [beta] * 5, nthreads=threads)
        lat.swendsen_wang(beta)
        labels, _ = orc.swendsen_wang(s, seed, k, beta)
        assert np.array_equal(lat.sw_labels(), labels.astype(np.int32)), k
        assert np.array_equal(lat.get(), s), k
    lat.close()


def test_uniform_lattice_is_one_cluster(isg):
    lat = isg.Lattice(64, 0, seed=3)
    lat.init_uniform(1)
    seen = set()
    for _ in range(10):
        lat.swendsen_wang(40.0)
        assert np.all(lat.sw_labels() == 0)
        g = lat.get()
        assert abs(int(g.astype(np.int64).sum())) == 64 * 64
        seen.add(int(g[0, 0]))
    assert seen == {-1, 1}
    lat.close()


def test_errors_and_checkpoint(isg, tmp_path):
    lat = isg.Lattice(64, 1, seed=9)
    lat.init_random()
    with pytest.raises(isg.IsgError) as e:
        lat.sw_labels()
    assert e.value.status == -1
    for bad in (-0.1, float("nan"), float("inf")):
        with pytest.raises(isg.IsgError):
            lat.swendsen_wang(bad)
    assert lat.sw_iterations == 0
    lat.sweep(3, beta=0.6)
    lat.swendsen_wang(0.6, n=2)
    path = str(tmp_path / "sw.isg")
    lat.save(path)
    lat.sweep(3, beta=0.6)
    lat.swendsen_wang(0.6)
    want = lat.get()
    lat.close()
    again = isg.Lattice.load(path)
    assert again.sw_iterations == 2
    again.sweep(3, beta=0.6)
    again.swendsen_wang(0.6)
    assert np.array_equal(again.get(), want)
    again.init_random()
    assert again.sw_iterations == 0
    again.close()
    big = isg.Lattice(65536, 0, seed=1)
    with pytest.raises(isg.IsgError) as e:
        big.swendsen_wang(0.4)
    assert e.value.status == -1
    big.close()


def _u4_xi(isg, Ms, Rs, Cs, L):
    M = np.asarray(Ms, dtype=np.float64)
    u4 = (M ** 4).mean() / (M ** 2).mean() ** 2
    xi = isg.xi2(np.asarray(Ms), np.asarray(Rs), np.asarray(Cs)) / L
    return u4, xi


def _blocks(isg, Ms, Rs, Cs, L, nb=16):
    n = len(Ms) // nb * nb
    vals = []
    for b in range(nb):
        keep = np.ones(n, bool)
        keep[b * n // nb:(b + 1) * n // nb] = False
        vals.append(_u4_xi(isg, np.asarray(Ms)[:n][keep], np.asarray(Rs)[:n][keep],
                           np.asarray(Cs)[:n][keep], L))
    vals = np.array(vals)
    return np.sqrt((nb - 1) * ((vals - vals.mean(axis=0)) ** 2).mean(axis=0))


@pytest.mark.parametrize("model,sweeps", [(1, 10), (0, 0)])
def test_emcs_reproduces_universal_values(isg, model, sweeps):
    L, n_lat, therm, meas = 128, 8, 50, 800
    beta = 1 / wl.T_C_BLUME_CAPEL if model == 1 else wl.BETA_C_ISING
    Ms, Rs, Cs = [], [], []
    for r in range(n_lat):
        lat = isg.Lattice(L, model, seed=wl.BASE_SEED + 7100 + r, record_capacity=meas + 1)
        lat.init_random()
        lat.emcs(therm, beta, sweeps=sweeps)
        lat.emcs(meas, beta, sweeps=sweeps, record_every=1)
        for o in lat.read_records():
            Ms.append(o.M)
            Rs.append(o.R)
            Cs.append(o.C)
        lat.close()
    u4, xi = _u4_xi(isg, Ms, Rs, Cs, L)
    du4, dxi = _blocks(isg, Ms, Rs, Cs, L)
    assert abs(u4 - U4_STAR) < 4 * du4 + 0.003, (u4, du4)
    assert abs(xi - XI_STAR) < 4 * dxi + 0.006, (xi, dxi)
    assert du4 < 0.03 and dxi < 0.03
