"""Parity of the served workload in the configuration the benchmark times:
48 requests of the served stream (Ising or Blume-Capel, L = 2^8 .. 2^14,
10^3 .. 10^4 sweeps under a ten-step bath from 1.5 T_c to 1.01 T_c), all
admitted at once into a server with 48 slots, 100-sweep chunks and a 96 GiB
budget.  Every request's final spins and observables equal the same request
run alone; the smallest requests of each model also equal the oracle run
with the same per-sweep temperatures.
"""
import os

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


def _betas(n, t_start, beta):
    """Per-sweep beta of a piecewise-constant schedule (sweep t uses the last
    piece with t_start <= t)."""
    out = np.empty(n)
    for k, (t0, b) in enumerate(zip(t_start, beta)):
        t1 = t_start[k + 1] if k + 1 < len(t_start) else n
        out[t0:t1] = b
    return out


def test_served_workload_alone_equals_in_the_mix(isg, orc):
    reqs = wl.served_requests(48)
    srv = isg.Server(hbm_budget=96 << 30, max_active=48, chunk_sweeps=100)
    ids = [srv.submit(r["model"], r["L"], r["seed"], r["sweeps"], r["t_start"], r["beta"],
                      keep=True, arrival_time=0.0) for r in reqs]
    srv.drain()
    small = {}
    for r in sorted(range(len(reqs)), key=lambda i: reqs[i]["L"] ** 2 * reqs[i]["sweeps"]):
        small.setdefault(reqs[r]["model"], [])
        if len(small[reqs[r]["model"]]) < 2:
            small[reqs[r]["model"]].append(r)
    threads = os.cpu_count() or 1
    for i, (rid, q) in enumerate(zip(ids, reqs)):
        res = srv.poll(rid)
        assert res.state == 2 and res.sweeps_done == q["sweeps"]
        got = srv.get_lattice(rid)
        lat = isg.Lattice(q["L"], q["model"], seed=q["seed"])
        lat.init_random()
        lat.sweep_schedule(q["sweeps"], q["t_start"], q["beta"])
        fin = lat.measure()
        assert (res.B, res.M, res.Q) == (fin.B, fin.M, fin.Q), (q["model"], q["L"])
        assert np.array_equal(got, lat.get()), (q["model"], q["L"])
        lat.close()
        if i in small.get(q["model"], []):
            s = orc.init_random(q["L"], q["model"], q["seed"])
            orc.run(s, q["model"], q["seed"], 0, _betas(q["sweeps"], q["t_start"], q["beta"]),
                    nthreads=threads)
            assert np.array_equal(got, s), ("oracle", q["model"], q["L"])
        srv.release(rid)
    assert sum(len(v) for v in small.values()) == 4
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()
