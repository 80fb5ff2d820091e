"""Row-slab domain decomposition on the GPU (Introduction; Table I: one
lattice on many GPUs).  The slabs' union must equal the lattice swept whole
(isg_sweep) bit for bit after every record, and the merged records must equal
the whole lattice's -- which the parity tests pin to the oracle -- and, at
L = 256, the oracle's directly.  Slabs run in one process (several slabs on
the one GPU, halos copied device to device) and as two gloo processes that
each own one slab on the same GPU and exchange their edge rows through host
memory.  No kernel ever waits on another process: the exchange happens on
the host between launches."""
import os
import socket

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

    return P


def _whole(isg, model, L, seed, delta, betas, every):
    lat = isg.Lattice(L, model, seed=seed, delta=delta, record_capacity=len(betas) // every + 1)
    lat.init_random()
    lat.sweep(len(betas), betas=np.asarray(betas), record_every=every)
    recs = lat.read_records()
    s = lat.get()
    lat.close()
    return s, recs


def _same_records(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert (x.sweep, x.B, x.M, x.Q) == (y.sweep, y.B, y.M, y.Q)
        assert np.array_equal(x.R, y.R) and np.array_equal(x.C, y.C)


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("L,P", [(256, 1), (256, 2), (1024, 4), (2048, 3)])
def test_slabs_in_one_process_equal_the_whole_lattice(isg, model, L, P):
    from paper_2503_14688_b300 import decomposition as dd

    seed, n, every = 0x2503146880000000 + 60 + L + P, 50, 10
    delta = 0.0 if model == 0 else 0.2
    betas = [BETA[model] * (0.95 + 0.002 * i) for i in range(n)]
    parts = dd.partition(L, P)
    slabs = {r: dd.Slab(model, L, y0, rows, seed, delta) for r, (y0, rows) in enumerate(parts)}
    for s in slabs.values():
        s.init_random()
    run = dd.Decomposition(slabs, dd.LocalExchange(P))
    recs = run.sweep(n, betas=betas, record_every=every)
    union = np.concatenate([run.get()[r] for r in range(P)])
    whole, wrecs = _whole(isg, model, L, seed, delta, betas, every)
    assert np.array_equal(union, whole)
    _same_records(recs, wrecs)
    for s in slabs.values():
        assert s.sweep_count == n
        s.close()


@pytest.mark.parametrize("model", [0, 1])
def test_slabs_equal_the_oracle(isg, orc, model):
    from paper_2503_14688_b300 import decomposition as dd

    L, P, n, every, seed = 256, 4, 20, 5, 0x2503146880000000 + 70 + model
    betas = [BETA[model]] * n
    parts = dd.partition(L, P)
    slabs = {r: dd.Slab(model, L, y0, rows, seed) for r, (y0, rows) in enumerate(parts)}
    for s in slabs.values():
        s.init_random()
    # the hot start of the owned rows is the lattice's hot start
    s0 = orc.init_random(L, model, seed)
    for r, (y0, rows) in enumerate(parts):
        assert np.array_equal(slabs[r].get(), s0[y0:y0 + rows])
    run = dd.Decomposition(slabs, dd.LocalExchange(P))
    recs = run.sweep(n, betas=betas, record_every=every)
    bmq, R, C = orc.run(s0, model, seed, 0, betas, record_every=every)
    assert np.array_equal(np.concatenate([run.get()[r] for r in range(P)]), s0)
    for i, r in enumerate(recs):
        assert (r.B, r.M, r.Q) == tuple(int(v) for v in bmq[i])
        assert np.array_equal(r.R, R[i]) and np.array_equal(r.C, C[i])
    for s in slabs.values():
        s.close()


def test_slab_set_get_and_invalid_arguments(isg):
    from paper_2503_14688_b300 import decomposition as dd
    from paper_2503_14688_b300 import _abi

    rng = np.random.default_rng(3)
    s = dd.Slab(1, 128, 32, 48, seed=5)
    v = rng.integers(-1, 2, size=(48, 128)).astype(np.int8)
    s.set(v, t=7)
    assert np.array_equal(s.get(), v) and s.sweep_count == 7
    v[3, 5] = 2
    with pytest.raises(_abi.IsgError):
        s.set(v)
    s.close()
    for y0, rows in [(8, 16), (0, 24), (0, 0), (112, 32)]:
        with pytest.raises(_abi.IsgError):
            dd.Slab(0, 128, y0, rows)


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, model, L, n, every, seed, out_dir):
    import torch
    import torch.distributed as dist

    from paper_2503_14688_b300 import decomposition as dd

    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        parts = dd.partition(L, world)
        y0, rows = parts[rank]
        slab = dd.Slab(model, L, y0, rows, seed, host_edges=True)
        slab.init_random()
        xc = dd.DistExchange(rank, world, [r for _, r in parts], device="cpu")
        run = dd.Decomposition({rank: slab}, xc)
        recs = run.sweep(n, beta=BETA[model], record_every=every)
        np.save(os.path.join(out_dir, f"rows{rank}.npy"), slab.get())
        if rank == 0:
            np.save(os.path.join(out_dir, "bmq.npy"),
                    np.array([[r.sweep, r.B, r.M, r.Q] for r in recs], dtype=np.int64))
            np.save(os.path.join(out_dir, "R.npy"), np.stack([r.R for r in recs]))
            np.save(os.path.join(out_dir, "C.npy"), np.stack([r.C for r in recs]))
        slab.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("model", [0, 1])
def test_two_gloo_processes_equal_the_whole_lattice(isg, orc, tmp_path, model):
    import torch.multiprocessing as mp

    L, n, every, seed, world = 512, 50, 10, 0x2503146880000000 + 80 + model, 2
    mp.start_processes(_rank_main, args=(world, _free_port(), model, L, n, every, seed,
                                         str(tmp_path)),
                       nprocs=world, join=True, start_method="spawn")
    union = np.concatenate([np.load(tmp_path / f"rows{r}.npy") for r in range(world)])
    whole, wrecs = _whole(isg, model, L, seed, 0.0, [BETA[model]] * n, every)
    assert np.array_equal(union, whole)
    bmq = np.load(tmp_path / "bmq.npy")
    assert np.array_equal(bmq, [[r.sweep, r.B, r.M, r.Q] for r in wrecs])
    assert np.array_equal(np.load(tmp_path / "R.npy"), np.stack([r.R for r in wrecs]))
    assert np.array_equal(np.load(tmp_path / "C.npy"), np.stack([r.C for r in wrecs]))
