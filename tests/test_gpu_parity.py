"""GPU parity: the CUDA path through the C ABI against the oracle, element by
element, on the same seeded inputs.  Integer work (spins, B, M, Q, row and
column sums) must agree bit for bit at every recorded sweep; the FP64 xi_2
computed from them must agree to 1e-12 relative (here: exactly, since both
sides evaluate the same operation sequence on equal integers).
"""
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


def _compare_records(gpu_recs, bmq, R, C):
    assert len(gpu_recs) == len(bmq)
    for i, r in enumerate(gpu_recs):
        assert (r.B, r.M, r.Q) == tuple(int(v) for v in bmq[i]), (i, r.sweep)
        assert np.array_equal(r.R, R[i]), ("row sums", i)
        assert np.array_equal(r.C, C[i]), ("col sums", i)


def _pair(isg, orc, model, L, seed, hot=True, delta=0.0, start=None):
    lat = isg.Lattice(L, model, seed=seed, delta=delta, record_capacity=64)
    if start is not None:
        lat.set(start)
        s = start.copy()
    elif hot:
        lat.init_random()
        s = orc.init_random(L, model, seed)
    else:
        lat.init_uniform(1)
        s = np.ones((L, L), dtype=np.int8)
    return lat, s


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("L", [64, 128, 192, 256, 320, 1024])
def test_hot_start_matches_oracle(isg, orc, model, L):
    seed = wl.BASE_SEED + 100 + L
    lat = isg.Lattice(L, model, seed=seed)
    lat.init_random()
    assert np.array_equal(lat.get(), orc.init_random(L, model, seed))


@pytest.mark.parametrize("model", [0, 1])
def test_set_get_and_windows(isg, model):
    L = 192
    rng = np.random.default_rng(7)
    vals = (-1, 1) if model == 0 else (-1, 0, 1)
    s = rng.choice(vals, size=(L, L)).astype(np.int8)
    lat = isg.Lattice(L, model, seed=1)
    lat.set(s, t=17)
    assert lat.sweep_index == 17
    assert np.array_equal(lat.get(), s)
    for (y0, x0, h, w) in [(0, 0, 5, 7), (190, 185, 9, 11), (3, 100, 64, 1), (0, 0, L, L)]:
        want = np.roll(np.roll(s, -y0, 0), -x0, 1)[:h, :w]
        assert np.array_equal(lat.get_rect(y0, x0, h, w), want)
    bad = s.copy()
    bad[5, 5] = 2
    with pytest.raises(isg.IsgError):
        lat.set(bad)


def test_ising_L256_quench_every_sweep(isg, orc):
    """Ising L=256, hot start, beta_c, 100 sweeps: lattice and sums every sweep."""
    w = wl.ising_quench_small()
    lat, s = _pair(isg, orc, w.model, w.L, w.seed)
    betas = [w.beta] * w.sweeps
    bmq, R, C = orc.run(s, w.model, w.seed, 0, betas, record_every=1)
    recs = []
    for chunk in range(0, w.sweeps, 50):
        lat.sweep(50, beta=w.beta, record_every=1)
        recs += lat.read_records()
    assert [r.sweep for r in recs] == list(range(1, w.sweeps + 1))
    _compare_records(recs, bmq, R, C)
    assert np.array_equal(lat.get(), s)
    # xi_2 of the (one-replica) record set, sweep by sweep
    for i in (0, 9, 49, 99):
        a = isg.xi2([recs[i].M], recs[i].R[None], recs[i].C[None])
        b = orc.xi2([bmq[i, 1]], R[i][None], C[i][None])
        assert (math.isnan(a) and math.isnan(b)) or a == b


@pytest.mark.parametrize("L", [64, 128, 192, 320, 512])
@pytest.mark.parametrize("model", [0, 1])
def test_small_lattices_every_sweep(isg, orc, model, L):
    """Word widths 1, 2, 3, 5, 8 per row: every thread/word layout case."""
    seed = wl.BASE_SEED + 200 + L + model
    beta = wl.BETA_C_ISING if model == 0 else 1 / wl.T_C_BLUME_CAPEL
    lat, s = _pair(isg, orc, model, L, seed)
    bmq, R, C = orc.run(s, model, seed, 0, [beta] * 20, record_every=1)
    lat.sweep(20, beta=beta, record_every=1)
    _compare_records(lat.read_records(), bmq, R, C)
    assert np.array_equal(lat.get(), s)


def test_blume_capel_L1024_every_sweep(isg, orc):
    """Blume-Capel Delta=0, T=1.6938, L=1024, 1000 sweeps, sums every sweep."""
    w = wl.blume_capel_parity()
    lat, s = _pair(isg, orc, w.model, w.L, w.seed)
    bmq, R, C = orc.run(s, w.model, w.seed, 0, [w.beta] * w.sweeps, record_every=1,
                        nthreads=orc.default_threads())
    recs = []
    for _ in range(0, w.sweeps, 50):
        lat.sweep(50, beta=w.beta, record_every=1)
        recs += lat.read_records()
    _compare_records(recs, bmq, R, C)
    assert np.array_equal(lat.get(), s)


@pytest.mark.parametrize("delta,T", [(0.5, 1.0), (-0.7, 2.0), (1.9, 0.6)])
def test_blume_capel_crystal_field(isg, orc, delta, T):
    L, seed = 256, wl.BASE_SEED + 300
    lat, s = _pair(isg, orc, 1, L, seed, delta=delta)
    bmq, R, C = orc.run(s, 1, seed, 0, [1 / T] * 40, delta=delta, record_every=1)
    lat.sweep(40, beta=1 / T, record_every=1)
    _compare_records(lat.read_records(), bmq, R, C)
    assert np.array_equal(lat.get(), s)


def test_blume_capel_moves_never_accepted(isg, orc):
    """Blume-Capel at beta so large that some thresholds round to 0 (the move
    is never taken): the kernels switch to the (u >> 1) < thr31 compare for
    those sweeps.  beta(t) alternates between such sweeps, beta = inf and
    ordinary ones, so both compare forms follow each other on one lattice."""
    L, seed, delta = 192, wl.BASE_SEED + 310, 1.9
    lat, s = _pair(isg, orc, 1, L, seed, delta=delta)
    betas = [0.6, 10.0, 0.6, math.inf, 0.8, 3.0] * 5
    bmq, R, C = orc.run(s, 1, seed, 0, betas, delta=delta, record_every=1)
    lat.sweep(len(betas), betas=betas, record_every=1)
    _compare_records(lat.read_records(), bmq, R, C)
    assert np.array_equal(lat.get(), s)


@pytest.mark.parametrize("model", [0, 1])
def test_schedule_and_per_sweep_betas(isg, orc, model):
    """Pre-cooling bath (Table II): T1 until t_switch, then T2; and beta(t) arrays."""
    L, seed, n = 256, wl.BASE_SEED + 400 + model, 60
    t_start, beta = wl.precooling_schedule(model, t_switch=23)
    betas = [beta[0] if t < 23 else beta[1] for t in range(n)]
    lat, s = _pair(isg, orc, model, L, seed)
    bmq, R, C = orc.run(s, model, seed, 0, betas, record_every=3)
    lat.sweep_schedule(n, t_start, beta, record_every=3)
    _compare_records(lat.read_records(), bmq, R, C)
    assert np.array_equal(lat.get(), s)
    # arbitrary beta(t) passed per sweep, continuing from t = 60
    more = np.linspace(0.2, 0.9, 15)
    orc.run(s, model, seed, n, more)
    lat.sweep(15, betas=more)
    assert np.array_equal(lat.get(), s)
    assert lat.sweep_index == n + 15


def test_limits_on_gpu(isg, orc):
    """beta = 0 negates an Ising lattice per sweep; beta = inf never raises E."""
    L = 256
    lat = isg.Lattice(L, 0, seed=9, record_capacity=32)
    lat.init_random()
    s0 = lat.get()
    lat.sweep(1, beta=0.0)
    assert np.array_equal(lat.get(), -s0)
    lat.sweep(30, beta=math.inf, record_every=1)
    e = [-r.B for r in lat.read_records()]
    assert all(b <= a for a, b in zip(e, e[1:]))


def test_measure_and_half_sweeps(isg, orc):
    L, seed = 512, wl.BASE_SEED + 500
    lat, s = _pair(isg, orc, 0, L, seed)
    B, M, Q, R, C = orc.measure(s)
    o = lat.measure()
    assert (o.B, o.M, o.Q) == (B, M, Q) and np.array_equal(o.R, R) and np.array_equal(o.C, C)
    # two half-sweeps = one sweep
    lat.half_sweep(0, 0.5)
    lat.half_sweep(1, 0.5)
    orc.run(s, 0, seed, 0, [0.5])
    assert lat.sweep_index == 1 and np.array_equal(lat.get(), s)


def test_record_ring_limits(isg):
    lat = isg.Lattice(64, 0, seed=1, record_capacity=4)
    lat.init_random()
    lat.sweep(4, beta=0.4, record_every=1)
    with pytest.raises(isg.IsgError) as e:
        lat.sweep(1, beta=0.4, record_every=1)
    assert e.value.status == -5  # ISG_ERR_BUSY
    assert len(lat.read_records(2)) == 2
    lat.sweep(2, beta=0.4, record_every=1)
    recs = lat.read_records()
    assert [r.sweep for r in recs] == [3, 4, 5, 6]


def test_invalid_arguments_gpu(isg):
    lat = isg.Lattice(64, 0, seed=1)
    lat.init_random()
    for bad in (-0.1, float("nan")):
        with pytest.raises(isg.IsgError):
            lat.sweep(1, beta=bad)
    with pytest.raises(isg.IsgError):
        lat.half_sweep(2, 0.4)
    with pytest.raises(isg.IsgError):
        lat.init_uniform(0)  # 0 is not an Ising spin


@pytest.mark.parametrize("model", [0, 1])
def test_checkpoint_resume_is_bit_exact(isg, tmp_path, model):
    """n1 sweeps, save, load, n2 sweeps == n1 + n2 sweeps straight."""
    L, seed = 320, wl.BASE_SEED + 700 + model
    beta = 0.45 if model == 0 else 0.6
    straight = isg.Lattice(L, model, seed=seed, delta=0.2, record_capacity=8)
    straight.init_random()
    straight.sweep(13, beta=beta)
    straight.sweep(9, beta=beta, record_every=3)
    want = straight.read_records()
    a = isg.Lattice(L, model, seed=seed, delta=0.2)
    a.init_random()
    a.sweep(13, beta=beta)
    path = str(tmp_path / "ckpt.isg")
    a.save(path)
    a.close()
    b = isg.Lattice.load(path, record_capacity=8)
    assert b.sweep_index == 13 and b.L == L
    b.sweep(9, beta=beta, record_every=3)
    got = b.read_records()
    assert [(r.sweep, r.B, r.M, r.Q) for r in got] == [(r.sweep, r.B, r.M, r.Q) for r in want]
    assert np.array_equal(b.get(), straight.get())


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("L", [64, 192, 256, 1024])
def test_correlation_matches_oracle(isg, orc, model, L):
    """Axis correlation sums (Eq. (2)) on an evolved lattice, all parities of
    r, the wrap-around distances and r = 0, bit-exact."""
    seed = wl.BASE_SEED + 800 + L + model
    lat, s = _pair(isg, orc, model, L, seed, delta=0.3)
    beta = 0.44 if model == 0 else 0.6
    lat.sweep(7, beta=beta)
    orc.run(s, model, seed, 0, [beta] * 7, delta=0.3)
    r = sorted(set([0, 1, 2, 3, 5, 31, 32, 33, 63, L // 2 - 1, L // 2, L // 2 + 1, L - 1]) &
               set(range(L)))
    gx, gy = lat.correlation(r)
    ox, oy = orc.correlation(s, r)
    assert np.array_equal(gx, ox) and np.array_equal(gy, oy)
    o = lat.measure()
    assert gx[r.index(1)] + gy[r.index(1)] == o.B and gx[0] == o.Q


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("L", [2112, 16384])
def test_correlation_matches_oracle_with_many_bands(isg, orc, model, L):
    """The correlation pass where a launch has many row bands (1-row bands
    at L = 2112, 16-row bands of four 4-row steps at L = 16384), so that
    the vertical partner row wraps inside bands for most distances (the
    band is walked in two segments there) and segments start on rows of
    either parity; seeded lattices with a bias, since the sums of a hot
    start are near zero."""
    rng = np.random.default_rng(wl.BASE_SEED + 820 + L + model)
    if model == 0:
        s = np.where(rng.random((L, L)) < 0.6, 1, -1).astype(np.int8)
    else:
        s = rng.choice(np.array([-1, 0, 1], dtype=np.int8), size=(L, L), p=[0.25, 0.25, 0.5])
    lat = isg.Lattice(L, model, seed=1)
    try:
        lat.set(s)
        r = sorted(set([0, 1, 2, 3, 5, 7, 64, 65, 1001, L // 2 - 1, L // 2, L // 2 + 1, L - 3, L - 1]))
        gx, gy = lat.correlation(r)
    finally:
        lat.close()
    ox, oy = orc.correlation(s, r)
    assert np.array_equal(gx, ox) and np.array_equal(gy, oy)
