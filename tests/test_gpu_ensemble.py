"""GPU parity of the replica ensemble (isg_ensemble_*): every replica must
evolve bit for bit like a lattice swept alone with the same seed (itself
checked against the oracle in test_gpu_parity.py), and a subset is compared
with the oracle directly.  Sizes cover the shared-memory path (Ising
L <= 1280, Blume-Capel L <= 896) and the global-memory path beyond it; the
ensemble-mean xi_2 of the records is compared with the oracle's."""
import math

import numpy as np
import pytest

from paper_2503_14688_b300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def isg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2503_14688_b300 import build

    build.build()
    import paper_2503_14688_b300 as P

    return P


def _alone(isg, L, model, seed, betas, record_every, delta=0.0):
    lat = isg.Lattice(L, model, seed=seed, delta=delta, record_capacity=len(betas) + 1)
    lat.init_random()
    lat.sweep(len(betas), betas=betas, record_every=record_every)
    recs = lat.read_records()
    s = lat.get()
    lat.close()
    return recs, s


def _same_obs(a, b):
    assert (a.sweep, a.B, a.M, a.Q) == (b.sweep, b.B, b.M, b.Q)
    assert np.array_equal(a.R, b.R) and np.array_equal(a.C, b.C)


def test_mixed_ensemble_matches_lattices_alone(isg, orc):
    Ls = [64, 128, 192, 256, 320, 512, 1024, 1280, 1536, 64, 256, 1024]
    models = [0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1]  # BC 1024 takes the global path
    seeds = [wl.BASE_SEED + 600 + r for r in range(len(Ls))]
    delta, n, k = 0.25, 24, 4
    betas = np.linspace(0.35, 0.55, n)
    ens = isg.Ensemble(Ls, seeds, models=models, delta=delta, record_capacity=8)
    ens.init_random()
    ens.sweep(10, betas=betas[:10], record_every=5)
    ens.sweep(n - 10, betas=betas[10:], record_every=k)  # second call: graph update path
    rows = ens.read_records()
    assert len(rows) == 2 + (n - 10) // k
    for r, (L, m, sd) in enumerate(zip(Ls, models, seeds)):
        recs1, s = _alone(isg, L, m, sd, betas[:10], 5, delta)
        lat = isg.Lattice(L, m, seed=sd, delta=delta, record_capacity=16)
        lat.set(s, t=10)
        lat.sweep(n - 10, betas=betas[10:], record_every=k)
        recs = recs1 + lat.read_records()
        final = lat.get()
        lat.close()
        assert len(recs) == len(rows)
        for i, row in enumerate(rows):
            _same_obs(row[r], recs[i])
        assert np.array_equal(ens.get(r), final), (L, m)
    # a few replicas straight against the oracle
    for r in (0, 2, 9):
        s = orc.init_random(Ls[r], models[r], seeds[r])
        bmq, R, C = orc.run(s, models[r], seeds[r], 0, betas, delta=delta)
        assert np.array_equal(ens.get(r), s)


def test_blume_capel_never_accepted_moves_in_ensemble(isg):
    """Per-sweep tables where some Blume-Capel moves can never be accepted
    (beta = 10, inf) between ordinary ones: shared-memory replicas equal the
    lattices swept alone."""
    Ls, delta = [64, 256, 512], 1.9
    seeds = [wl.BASE_SEED + 650 + r for r in range(len(Ls))]
    betas = np.array([0.6, 10.0, 0.6, np.inf, 0.8, 3.0] * 4)
    ens = isg.Ensemble(Ls, seeds, models=[1] * len(Ls), delta=delta, record_capacity=8)
    ens.init_random()
    ens.sweep(len(betas), betas=betas, record_every=6)
    rows = ens.read_records()
    for r, (L, sd) in enumerate(zip(Ls, seeds)):
        recs, s = _alone(isg, L, 1, sd, betas, 6, delta)
        for k, rec in enumerate(recs):
            _same_obs(rows[k][r], rec)
        assert np.array_equal(ens.get(r), s)
    ens.close()


def test_multi_lattice_launches_with_odd_word_counts(isg):
    """Global-path groups whose rows hold an odd number of words (Ising
    L = 1344, Blume-Capel L = 960: one word per thread) and a Blume-Capel
    group with a never-accepted move (beta = 10 at Delta = 1.9) equal the
    lattices alone."""
    Ls = [1344, 1344, 1344, 960, 960, 960]
    models = [0, 0, 0, 1, 1, 1]
    seeds = [wl.BASE_SEED + 760 + r for r in range(len(Ls))]
    betas = np.array([0.4, 0.45, 10.0, 0.6, 0.5, 0.7, 10.0, 0.44, 0.55, 0.62])
    ens = isg.Ensemble(Ls, seeds, models=models, delta=1.9, record_capacity=4)
    ens.init_random()
    ens.sweep(len(betas), betas=betas, record_every=5)
    rows = ens.read_records()
    for r, (L, m, sd) in enumerate(zip(Ls, models, seeds)):
        recs, s = _alone(isg, L, m, sd, betas, 5, delta=1.9)
        for k, rec in enumerate(recs):
            _same_obs(rows[k][r], rec)
        assert np.array_equal(ens.get(r), s), (L, m)
    ens.close()


def test_long_call_over_large_replicas_runs_without_a_graph(isg):
    """Replicas too large for shared memory (Blume-Capel L = 1024) take one
    multi-lattice launch per half-sweep; a call with more than 2048 of them
    is queued on the stream instead of captured.  Its replicas and records
    equal lattices alone, and a following short (captured) call continues
    them."""
    n_rep, n = 8, 1100  # 2 x 1100 multi-lattice launches
    Ls = [1024] * n_rep
    seeds = [wl.BASE_SEED + 700 + r for r in range(n_rep)]
    betas = np.full(n + 20, 1 / wl.T_C_BLUME_CAPEL)
    ens = isg.Ensemble(Ls, seeds, models=[1] * n_rep, delta=0.0, record_capacity=120)
    ens.init_random()
    ens.sweep(n, betas=betas[:n], record_every=10)
    ens.sweep(20, betas=betas[n:], record_every=10)
    rows = ens.read_records()
    assert len(rows) == 112
    for r in (0, 5):
        recs, s = _alone(isg, 1024, 1, seeds[r], betas, 10)
        for k in (0, 55, 109, 110, 111):
            _same_obs(rows[k][r], recs[k])
        assert np.array_equal(ens.get(r), s)
    ens.close()


def test_ensemble_workload_subset_and_xi2(isg, orc):
    """The replica-ensemble workload (uneven mix of L in {64..1024}, hot start
    quenched to beta_c), 64 replicas covering all sizes, 300 sweeps recorded
    every 100: bit-exact against lattices alone; the ensemble-mean xi_2 of the
    L = 64 replicas equals the oracle's, computed from the oracle's own runs."""
    Ls = wl.ensemble_sizes(64)
    Ls[:5] = [64, 128, 256, 512, 1024]
    seeds = [wl.BASE_SEED + 3 + r for r in range(64)]
    n, k = 300, 100
    ens = isg.Ensemble(Ls, seeds, record_capacity=4)
    assert ens.autotune(2)["threads_per_cta"] in (256, 512, 1024)
    ens.init_random()
    ens.sweep(n, beta=wl.BETA_C_ISING, record_every=k)
    rows = ens.read_records()
    assert len(rows) == n // k
    for r in range(0, 64, 7):
        recs, s = _alone(isg, int(Ls[r]), 0, seeds[r], [wl.BETA_C_ISING] * n, k)
        for i, row in enumerate(rows):
            _same_obs(row[r], recs[i])
        assert np.array_equal(ens.get(r), s)
    idx = [r for r in range(64) if Ls[r] == 64]
    assert len(idx) >= 3
    M, R, C = [], [], []
    for r in idx:
        s = orc.init_random(64, 0, seeds[r])
        bmq, Rr, Cr = orc.run(s, 0, seeds[r], 0, [wl.BETA_C_ISING] * n, record_every=k)
        M.append(bmq[-1, 1])
        R.append(Rr[-1])
        C.append(Cr[-1])
        assert np.array_equal(ens.get(r), s)
    want = orc.xi2(M, np.array(R), np.array(C))
    got = isg.xi2([rows[-1][r].M for r in idx], np.array([rows[-1][r].R for r in idx]),
                  np.array([rows[-1][r].C for r in idx]))
    assert (math.isnan(got) and math.isnan(want)) or abs(got - want) <= 1e-12 * abs(want)


def test_ensemble_errors(isg):
    with pytest.raises(isg.IsgError):
        isg.Ensemble([100], [1])
    ens = isg.Ensemble([64, 128], [1, 2], record_capacity=1)
    ens.init_random()
    with pytest.raises(isg.IsgError) as e:
        ens.sweep(4, beta=0.4, record_every=2)  # two rows, room for one
    assert e.value.status == -5
    with pytest.raises(isg.IsgError):
        ens.sweep(1, beta=-1.0)


def test_every_launch_shape_gives_the_same_replicas(isg):
    """The launch shape (CTA size, half-CTA teams, sweeps per launch, the
    multi-lattice words per thread and band rows) never changes a result:
    every shape below, including launches cut in the middle of a record
    period (rounded up) and forced multi-lattice shapes, gives each replica
    exactly the run of the lattice alone; the autotuner's choice is the
    fastest candidate of each part."""
    Ls = [64, 320, 1024, 256, 2048, 1536, 2048]
    models = [0, 1, 0, 1, 0, 0, 1]
    seeds = [wl.BASE_SEED + 700 + r for r in range(len(Ls))]
    n, k = 30, 5
    betas = [0.44 + 0.002 * i for i in range(n)]
    alone = []
    for L, m, sd in zip(Ls, models, seeds):
        lat = isg.Lattice(L, m, seed=sd, record_capacity=n // k)
        lat.init_random()
        lat.sweep(n, betas=np.asarray(betas), record_every=k)
        alone.append((lat.read_records(), lat.get()))
        lat.close()
    shapes = [dict(threads_per_cta=256, half_teams=0, sweeps_per_launch=7, multi_words=1, multi_band=16),
              dict(threads_per_cta=1024, half_teams=1, sweeps_per_launch=0, multi_words=4, multi_band=64),
              dict(threads_per_cta=512, half_teams=1, sweeps_per_launch=13, multi_words=2, multi_band=32),
              dict(threads_per_cta=1024, half_teams=0, sweeps_per_launch=1, multi_words=0, multi_band=0)]
    for shape in shapes:
        ens = isg.Ensemble(Ls, seeds, models=models, record_capacity=n // k)
        ens.set_tuning(**shape)
        assert ens.tuning() == shape
        ens.init_random()
        ens.sweep(n, betas=betas, record_every=k)
        rows = ens.read_records()
        assert len(rows) == n // k
        for r, (recs, s) in enumerate(alone):
            for i, row in enumerate(rows):
                _same_obs(row[r], recs[i])
            assert np.array_equal(ens.get(r), s), (shape, r)
        ens.close()
    ens = isg.Ensemble(Ls, seeds, models=models)
    ens.init_random()
    best, cands = ens.autotune(4, with_candidates=True)
    part0 = [c for c in cands if c["part"] == 0]
    part1 = [c for c in cands if c["part"] == 1]
    assert len(part0) == 12 and len(part1) == 16
    f0 = min(part0, key=lambda c: c["ms"])
    f1 = min(part1, key=lambda c: c["ms"])
    assert (best["threads_per_cta"], best["half_teams"], best["sweeps_per_launch"]) == \
        (f0["threads_per_cta"], f0["half_teams"], f0["sweeps_per_launch"])
    assert (best["multi_words"], best["multi_band"]) == (f1["multi_words"], f1["multi_band"])
    with pytest.raises(isg.IsgError):
        ens.set_tuning(threads_per_cta=300)
    ens.close()
