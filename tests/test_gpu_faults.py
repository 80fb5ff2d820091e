"""Failure handling on the host: allocation failures, launch failures,
request cancellation and deadlines.  Every failure here is made on the host
(isg_debug_inject skips an allocation or a launch and reports the error);
no test faults, traps or hangs the GPU.  What must hold: the call reports the
error (ISG_ERR_OOM / ISG_ERR_CUDA), nothing it allocated stays allocated,
the library stays usable, and in the server one request's failure,
cancellation or expiry leaves every other request bit for bit as it would be
alone."""
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

    yield P
    P.lattice.inject_fault(1, 0)
    P.lattice.inject_fault(2, 0)


def _free():
    import torch

    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_lattice_create_fails_cleanly_at_each_allocation(isg):
    from paper_2503_14688_b300 import _abi

    free0 = _free()
    for k in (1, 2, 3):
        isg.lattice.inject_fault(_abi.ISG_INJECT_ALLOC, k)
        with pytest.raises(isg.IsgError) as e:
            isg.Lattice(1024, 0, seed=1)
        assert e.value.status == _abi.ISG_ERR_OOM
        assert _free() == free0
    isg.lattice.inject_fault(_abi.ISG_INJECT_ALLOC, 0)
    lat = isg.Lattice(1024, 0, seed=1)
    lat.close()
    assert _free() == free0


def test_ensemble_create_fails_cleanly(isg):
    from paper_2503_14688_b300 import _abi

    free0 = _free()
    Ls = [64, 256, 2048]
    for k in range(1, 8):
        isg.lattice.inject_fault(_abi.ISG_INJECT_ALLOC, k)
        try:
            ens = isg.Ensemble(Ls, [1, 2, 3], models=[0, 1, 0])
        except isg.IsgError as e:
            assert e.status == _abi.ISG_ERR_OOM
        else:  # fewer allocations than k: nothing was injected
            ens.close()
        assert _free() == free0
    isg.lattice.inject_fault(_abi.ISG_INJECT_ALLOC, 0)


def test_failed_launch_reports_cuda_error_and_the_library_recovers(isg):
    from paper_2503_14688_b300 import _abi

    lat = isg.Lattice(512, 1, seed=7)
    lat.init_random()
    isg.lattice.inject_fault(_abi.ISG_INJECT_LAUNCH, 3)
    with pytest.raises(isg.IsgError) as e:
        lat.sweep(4, beta=0.6)
    assert e.value.status == _abi.ISG_ERR_CUDA
    # after an error the spins are undefined: start again, as a fresh lattice
    lat.init_random()
    lat.sweep(4, beta=0.6)
    ref = isg.Lattice(512, 1, seed=7)
    ref.init_random()
    ref.sweep(4, beta=0.6)
    assert np.array_equal(lat.get(), ref.get())
    lat.close()
    ref.close()


def _alone(isg, model, L, seed, n, t_start, beta):
    lat = isg.Lattice(L, model, seed=seed)
    lat.init_random()
    lat.sweep_schedule(n, t_start, beta)
    fin = lat.measure()
    s = lat.get()
    lat.close()
    return s, fin


def _req(i, model, L, n):
    Tc = wl.T_C_ISING if model == 0 else wl.T_C_BLUME_CAPEL
    t_start, beta = wl.stepped_bath(Tc, n, steps=4)
    return dict(model=model, L=L, seed=wl.BASE_SEED + 900 + i, n=n, t_start=t_start, beta=beta)


def _submit(srv, r, **kw):
    return srv.submit(r["model"], r["L"], r["seed"], r["n"], r["t_start"], r["beta"], keep=True, **kw)


def _check_alone(isg, srv, rid, r):
    res = srv.poll(rid)
    assert res.state == 2 and res.error == 0
    s, fin = _alone(isg, r["model"], r["L"], r["seed"], r["n"], r["t_start"], r["beta"])
    assert (res.B, res.M, res.Q) == (fin.B, fin.M, fin.Q)
    assert np.array_equal(srv.get_lattice(rid), s)
    srv.release(rid)


def test_server_admission_failure_fails_one_request(isg):
    from paper_2503_14688_b300 import _abi

    srv = isg.Server(hbm_budget=4 << 30, max_active=4, chunk_sweeps=20)
    reqs = [_req(0, 0, 2048, 60), _req(1, 1, 1024, 60), _req(2, 0, 512, 60)]
    # each admission allocates the planes, then the records: the 3rd device
    # allocation from here is the second request's planes
    isg.lattice.inject_fault(_abi.ISG_INJECT_ALLOC, 3)
    ids = [_submit(srv, r) for r in reqs]
    srv.drain()
    bad = srv.poll(ids[1])
    assert bad.state == _abi.ISG_REQ_FAILED and bad.error == _abi.ISG_ERR_OOM
    for k in (0, 2):
        _check_alone(isg, srv, ids[k], reqs[k])
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()


def test_server_batch_launch_failure_fails_its_requests_only(isg):
    from paper_2503_14688_b300 import _abi

    srv = isg.Server(hbm_budget=4 << 30, max_active=8, chunk_sweeps=20)
    first = [_req(10 + i, i % 2, 256, 40) for i in range(3)]  # shared-memory batch
    isg.lattice.inject_fault(_abi.ISG_INJECT_LAUNCH, 1)      # its first launch fails
    ids = [_submit(srv, r) for r in first]
    srv.step()
    for rid in ids:
        res = srv.poll(rid)
        assert res.state == _abi.ISG_REQ_FAILED and res.error == _abi.ISG_ERR_CUDA
    assert srv.stats()["bytes_in_use"] == 0
    later = [_req(20, 0, 320, 40), _req(21, 1, 192, 40)]
    lids = [_submit(srv, r) for r in later]
    srv.drain()
    for rid, r in zip(lids, later):
        _check_alone(isg, srv, rid, r)
    srv.close()


def test_server_cancel_queued_and_running(isg):
    from paper_2503_14688_b300 import _abi

    srv = isg.Server(hbm_budget=4 << 30, max_active=1, chunk_sweeps=10)
    long_r = _req(30, 0, 2048, 3000)
    waiting = _req(31, 1, 512, 50)
    after = _req(32, 1, 256, 50)
    a = _submit(srv, long_r)
    b = _submit(srv, waiting)
    srv.step()
    srv.step()
    assert srv.poll(a).state == _abi.ISG_REQ_RUNNING and srv.poll(b).state == _abi.ISG_REQ_QUEUED
    srv.cancel(b)                       # queued: never admitted
    rb = srv.poll(b)
    assert rb.state == _abi.ISG_REQ_CANCELLED and rb.t_admit < 0
    srv.cancel(a)                       # running: stops after its queued chunk
    assert srv.poll(a).state == _abi.ISG_REQ_CANCELLED
    assert srv.stats()["bytes_in_use"] == 0
    with pytest.raises(isg.IsgError):
        srv.cancel(a)                   # already out of the schedule
    c = _submit(srv, after)
    srv.drain()
    _check_alone(isg, srv, c, after)
    assert srv.stats()["flips_done"] == after["L"] ** 2 * after["n"]
    srv.close()


def test_server_deadline_expires_a_request(isg):
    from paper_2503_14688_b300 import _abi

    srv = isg.Server(hbm_budget=8 << 30, max_active=4, chunk_sweeps=20)
    slow = _req(40, 0, 8192, 4000)   # about 0.2 s of device work
    quick = _req(41, 1, 512, 40)
    a = _submit(srv, slow, deadline=srv.clock() + 0.02)
    b = _submit(srv, quick)
    srv.drain()
    ra = srv.poll(a)
    assert ra.state == _abi.ISG_REQ_EXPIRED and ra.t_done >= 0.02
    _check_alone(isg, srv, b, quick)
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()
