"""GPU tests of the request server (isg_server_*): continuous batching must
not bend the dynamics.  Each request's final lattice, final observables and
periodic records must equal those of the same request run alone through
isg_sweep_schedule, bit for bit, whatever ran beside it; admission must
respect the memory budget; requests arriving while others run are admitted
and finish."""
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


def _alone(isg, model, L, seed, n, t_start, beta, delta, record_every):
    lat = isg.Lattice(L, model, seed=seed, delta=delta, record_capacity=max(1, n))
    lat.init_random()
    lat.sweep_schedule(n, t_start, beta, record_every=record_every)
    recs = lat.read_records()
    fin = lat.measure()
    s = lat.get()
    lat.close()
    return s, fin, recs


def test_results_same_alone_and_in_the_mix(isg):
    chunk = 20
    srv = isg.Server(hbm_budget=8 << 30, max_active=6, chunk_sweeps=chunk)
    rng = np.random.default_rng(5)
    reqs = []
    # every valid side, not only powers of two: 64, 192, 320 arrive while
    # others (shared-memory batch and own-stream lattices) run
    specs = [(0, 256), (1, 256), (0, 512), (0, 1024), (1, 512), (0, 2048), (1, 1024), (0, 64),
             (1, 192), (0, 320), (1, 768), (0, 1280), (0, 512), (1, 320), (0, 192), (1, 64)]
    for i, (model, L) in enumerate(specs):
        Tc = wl.T_C_ISING if model == 0 else wl.T_C_BLUME_CAPEL
        n = int(rng.integers(30, 90))
        t_start, beta = wl.stepped_bath(Tc, n, steps=4)
        delta = 0.3 if model == 1 else 0.0
        rec = 10 if i % 3 == 0 else 0
        rid = srv.submit(model, L, wl.BASE_SEED + 5 + i, n, t_start, beta, delta=delta,
                         record_every=rec, keep=True, arrival_time=0.002 * i)
        reqs.append((rid, model, L, wl.BASE_SEED + 5 + i, n, t_start, beta, delta, rec))
    peak = 0
    while True:
        active, queued = srv.step()
        peak = max(peak, active)
        assert active <= 6
        if active == 0 and queued == 0:
            break
    srv.drain()
    assert peak >= 2  # work really overlapped
    for (rid, model, L, seed, n, t_start, beta, delta, rec) in reqs:
        res = srv.poll(rid)
        assert res.state == 2 and res.sweeps_done == n
        assert res.t_arrival <= res.t_admit <= res.t_done
        s, fin, recs = _alone(isg, model, L, seed, n, t_start, beta, delta, rec)
        assert (res.B, res.M, res.Q) == (fin.B, fin.M, fin.Q), (model, L)
        assert np.array_equal(srv.get_lattice(rid), s), (model, L)
        got = srv.read_records(rid)
        assert len(got) == len(recs)
        for a, b in zip(got, recs):
            assert (a.sweep, a.B, a.M, a.Q) == (b.sweep, b.B, b.M, b.Q)
            assert np.array_equal(a.R, b.R) and np.array_equal(a.C, b.C)
        srv.release(rid)
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()


def test_admission_respects_budget(isg):
    one = isg.Lattice.nbytes(0, 2048) + (32 + 8 * 2048)
    srv = isg.Server(hbm_budget=int(2.5 * one), max_active=8, chunk_sweeps=10)
    ids = [srv.submit(0, 2048, 100 + i, 25, [0], [0.44]) for i in range(5)]
    while True:
        active, queued = srv.step()
        assert srv.stats()["bytes_in_use"] <= 2.5 * one
        assert active <= 2
        if active == 0 and queued == 0:
            break
    for rid in ids:
        assert srv.poll(rid).state == 2
    assert srv.stats()["flips_done"] == 5 * 2048 * 2048 * 25
    srv.close()


def test_server_rejects_bad_requests(isg):
    srv = isg.Server(hbm_budget=1 << 30, max_active=2, chunk_sweeps=10)
    with pytest.raises(isg.IsgError):
        srv.submit(0, 100, 1, 10, [0], [0.4])          # not a multiple of 64
    with pytest.raises(isg.IsgError):
        srv.submit(0, 256, 1, 10, [5], [0.4])          # schedule must start at 0
    with pytest.raises(isg.IsgError):
        srv.submit(0, 256, 1, 10, [0], [0.4], record_every=3)  # does not divide the chunk
    with pytest.raises(isg.IsgError) as e:
        srv.submit(0, 1 << 17, 1, 10, [0], [0.4])      # 2 GiB: never fits the budget
    assert e.value.status == -2
    srv.close()
