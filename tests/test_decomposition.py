"""Host logic of the row-slab domain decomposition (Introduction: one lattice
on many GPUs), on the CPU: the package's driver (partition, halo exchange,
record merge) run over oracle-backed slabs must reproduce the whole-lattice
oracle bit for bit -- in one process (LocalExchange) and across world_size 2
and 3 gloo processes (DistExchange, point-to-point halo rows)."""
import os
import socket

import numpy as np
import pytest

import oracle
from oracle_slab_engine import OracleSlab
from paper_2503_14688_b300 import decomposition as dd

BETA = {0: 0.44068679350977147, 1: 1 / 1.69355839821214427017}


def test_partition_covers_the_lattice_in_quanta():
    for L, P in [(64, 1), (64, 4), (256, 3), (1024, 7), (1 << 20, 64)]:
        parts = dd.partition(L, P)
        assert len(parts) == P
        assert parts[0][0] == 0 and sum(r for _, r in parts) == L
        assert all(y0 % 16 == 0 and r % 16 == 0 and r >= 16 for y0, r in parts)
        assert all(parts[k + 1][0] == parts[k][0] + parts[k][1] for k in range(P - 1))
        assert max(r for _, r in parts) - min(r for _, r in parts) <= 16
    with pytest.raises(ValueError):
        dd.partition(64, 5)


def _reference(model, L, seed, betas, delta, every):
    s = oracle.init_random(L, model, seed)
    bmq, R, C = oracle.run(s, model, seed, 0, betas, delta=delta, record_every=every)
    return s, bmq, R, C


def _check(recs, union, ref, every):
    s, bmq, R, C = ref
    assert np.array_equal(union, s)
    assert len(recs) == len(bmq)
    for i, r in enumerate(recs):
        assert r.sweep == (i + 1) * every
        assert (r.B, r.M, r.Q) == tuple(int(v) for v in bmq[i])
        assert np.array_equal(r.R, R[i]) and np.array_equal(r.C, C[i])


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("P", [1, 2, 3])
def test_local_slabs_reproduce_the_oracle(model, P):
    L, n, every, seed = 96, 8, 2, 0x2503146880000000 + 40 + P
    delta = 0.4 if model == 1 else 0.0
    betas = [BETA[model] * (0.9 + 0.05 * i) for i in range(n)]
    parts = dd.partition(L, P)
    slabs = {r: OracleSlab(model, L, y0, rows, seed, delta) for r, (y0, rows) in enumerate(parts)}
    run = dd.Decomposition(slabs, dd.LocalExchange(P))
    recs = run.sweep(n, betas=betas, record_every=every)
    union = np.concatenate([run.get()[r] for r in range(P)])
    _check(recs, union, _reference(model, L, seed, betas, delta, every), every)


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, model, L, n, every, seed, delta, out_dir):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        parts = dd.partition(L, world)
        y0, rows = parts[rank]
        betas = [BETA[model] * (0.9 + 0.05 * i) for i in range(n)]
        slab = OracleSlab(model, L, y0, rows, seed, delta)
        xc = dd.DistExchange(rank, world, [r for _, r in parts], device="cpu")
        run = dd.Decomposition({rank: slab}, xc)
        recs = run.sweep(n, betas=betas, record_every=every)
        np.save(os.path.join(out_dir, f"rows{rank}.npy"), slab.get())
        if rank == 0:
            np.save(os.path.join(out_dir, "bmq.npy"),
                    np.array([[r.sweep, r.B, r.M, r.Q] for r in recs], dtype=np.int64))
            np.save(os.path.join(out_dir, "R.npy"), np.stack([r.R for r in recs]))
            np.save(os.path.join(out_dir, "C.npy"), np.stack([r.C for r in recs]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,model", [(2, 0), (2, 1), (3, 0)])
def test_gloo_ranks_reproduce_the_oracle(tmp_path, world, model):
    import torch.multiprocessing as mp

    L, n, every, seed = 96, 6, 3, 0x2503146880000000 + 50 + world
    delta = 0.25 if model == 1 else 0.0
    mp.start_processes(_rank_main, args=(world, _free_port(), model, L, n, every, seed, delta,
                                         str(tmp_path)),
                       nprocs=world, join=True, start_method="spawn")
    union = np.concatenate([np.load(tmp_path / f"rows{r}.npy") for r in range(world)])
    bmq = np.load(tmp_path / "bmq.npy")
    ref = _reference(model, L, seed, [BETA[model] * (0.9 + 0.05 * i) for i in range(n)], delta,
                     every)
    s, rbmq, R, C = ref
    assert np.array_equal(union, s)
    assert np.array_equal(bmq[:, 0], [(i + 1) * every for i in range(len(bmq))])
    assert np.array_equal(bmq[:, 1:], rbmq)
    assert np.array_equal(np.load(tmp_path / "R.npy"), R)
    assert np.array_equal(np.load(tmp_path / "C.npy"), C)
