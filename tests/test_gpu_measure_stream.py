"""The record pass at sides whose rows split into whole 256-word segments
(L a multiple of 16384), where it streams the rows into shared memory with
bulk copies (k_measure_stream).  B, M, Q, R and C (Eqs. (2)-(3)) must equal
the oracle's on seeded lattices with one and two segments per row -- the
side words of a segment's edges come from the row's other end there -- and
the register-walk record of the same lattice held as row slabs with four
segments per row (inner segments, halos from the neighbour segments).  A
wait that runs out (ISG_INJECT_WAIT: one block is promised 16 bytes that
never come) must fail that record with ISG_ERR_DEVICE_TIMEOUT -- through the
lattice calls, a served request's final record and the allocation-free
entry point -- the next record must be right, and no device fault is
involved."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BETA = {0: 0.44068679350977147, 1: 1 / 1.69355839821214427017}


@pytest.fixture(scope="module")
def isg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2503_14688_b300 import build

    build.build()
    import paper_2503_14688_b300 as P

    yield P
    P.lattice.inject_fault(3, 0)


def _lattice(model, L, seed):
    """Seeded spins with a bias, so that every sum is far from zero."""
    rng = np.random.default_rng(seed)
    if model == 0:
        return np.where(rng.random((L, L)) < 0.62, 1, -1).astype(np.int8)
    return rng.choice(np.array([-1, 0, 1], dtype=np.int8), size=(L, L), p=[0.25, 0.2, 0.55])


def _same(a, b):
    assert (a.B, a.M, a.Q) == (b.B, b.M, b.Q)
    assert np.array_equal(a.R, b.R) and np.array_equal(a.C, b.C)


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("L", [16384, 32768])
def test_streamed_record_equals_the_oracle(isg, orc, model, L):
    s = _lattice(model, L, 0x2503146880000000 + 90 + L + model)
    lat = isg.Lattice(L, model, seed=1)
    try:
        lat.set(s, t=7)
        o = lat.measure()
    finally:
        lat.close()
    B, M, Q, R, C = orc.measure(s)
    assert o.sweep == 7
    assert (o.B, o.M, o.Q) == (B, M, Q)
    assert np.array_equal(o.R, R) and np.array_equal(o.C, C)


@pytest.mark.parametrize("model", [0, 1])
def test_streamed_record_equals_the_slab_record_with_inner_segments(isg, model):
    from paper_2503_14688_b300 import decomposition as dd

    L, P, n, seed = 65536, 2, 2, 0x2503146880000000 + 95 + model
    lat = isg.Lattice(L, model, seed=seed, record_capacity=4)
    slabs = {r: dd.Slab(model, L, y0, rows, seed) for r, (y0, rows) in enumerate(dd.partition(L, P))}
    try:
        lat.init_random()
        lat.sweep(n, beta=BETA[model], record_every=1)
        whole = lat.read_records()
        for sl in slabs.values():
            sl.init_random()
        run = dd.Decomposition(slabs, dd.LocalExchange(P))
        parts = run.sweep(n, beta=BETA[model], record_every=1)
        assert len(whole) == len(parts) == n
        for a, b in zip(whole, parts):
            assert a.sweep == b.sweep
            _same(a, b)
    finally:
        lat.close()
        for sl in slabs.values():
            sl.close()


@pytest.mark.parametrize("model", [0, 1])
def test_a_wait_that_runs_out_fails_only_its_record(isg, model):
    from paper_2503_14688_b300 import _abi

    L = 16384
    s = _lattice(model, L, 0x2503146880000000 + 99 + model)
    lat = isg.Lattice(L, model, seed=2, record_capacity=4)
    try:
        lat.set(s)
        good = lat.measure()
        isg.lattice.inject_fault(3, 1)
        with pytest.raises(_abi.IsgError) as e:
            lat.measure()
        assert e.value.status == -4  # ISG_ERR_DEVICE_TIMEOUT
        _same(lat.measure(), good)
        # in the record ring: the failed record is dropped, the next one kept
        isg.lattice.inject_fault(3, 1)
        lat.record()
        lat.record()
        with pytest.raises(_abi.IsgError) as e:
            lat.read_records()
        assert e.value.status == -4
        rest = lat.read_records()
        assert len(rest) == 1
        _same(rest[0], good)
        assert np.array_equal(lat.get(), s)
    finally:
        isg.lattice.inject_fault(3, 0)
        lat.close()


def test_a_failed_final_record_fails_only_its_request(isg):
    """A served request of L = 16384 runs on its own stream and ends with a
    streamed record pass; when that pass's waits run out the request ends
    ISG_REQ_FAILED with ISG_ERR_DEVICE_TIMEOUT, and the next one is done."""
    srv = isg.Server(hbm_budget=2 << 30, max_active=2, chunk_sweeps=10)
    try:
        isg.lattice.inject_fault(3, 1)
        bad = srv.submit(0, 16384, 11, 10, [0], [0.44])
        srv.drain()
        r = srv.poll(bad)
        assert r.state == 5 and r.error == -4
        good = srv.submit(0, 16384, 12, 10, [0], [0.44], keep=True)
        srv.drain()
        r = srv.poll(good)
        assert r.state == 2 and r.sweeps_done == 10
        lat = isg.Lattice(16384, 0, seed=12)
        lat.init_random()
        lat.sweep(10, beta=0.44)
        o = lat.measure()
        lat.close()
        assert (r.B, r.M, r.Q) == (o.B, o.M, o.Q)
        srv.release(good)
    finally:
        isg.lattice.inject_fault(3, 0)
        srv.close()


def test_a_wait_that_runs_out_in_the_noalloc_pass(isg):
    """isg_measure_planes_noalloc at L = 16384 takes the streamed pass: a
    wait that runs out is reported as ISG_ERR_DEVICE_TIMEOUT and the next
    call is right."""
    import torch

    from paper_2503_14688_b300 import _abi

    L = 16384
    buf = torch.empty(isg.Lattice.nbytes(0, L), dtype=torch.uint8, device="cuda")
    lat = isg.Lattice(L, 0, seed=13, device_buf=buf)
    try:
        lat.init_random()
        want = lat.measure()
        isg.lattice.inject_fault(3, 1)
        with pytest.raises(_abi.IsgError) as e:
            isg.measure_planes_noalloc(0, L, buf)
        assert e.value.status == -4
        _same(isg.measure_planes_noalloc(0, L, buf), want)
    finally:
        isg.lattice.inject_fault(3, 0)
        lat.close()
