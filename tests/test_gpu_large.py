"""Parity at the full sizes of the large quench, in the launch configuration
the benchmark times: Ising L = 2^20 (2^40 spins, 128 GiB) and Blume-Capel
L = 2^19 (64 GiB), hot start, quench to T_c, records every 10 sweeps;
checked after 10 and after 100 sweeps.

The whole oracle cannot hold these lattices, so the spins are checked on
sampled windows: the oracle evolves a window with global keys and a fixed
outer ring, exact on the light-cone interior (distance > 2n from the ring
after n sweeps), which must equal the GPU lattice bit for bit.  The recorded
sums are checked against host recomputation from the GPU's own spins on
sampled rows and columns, and by sum R = sum C = M.
"""
import numpy as np
import pytest

from paper_2503_14688_b300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def isg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    free, _ = torch.cuda.mem_get_info()
    if free < 140 * 2**30:
        pytest.skip("needs about 140 GiB of free device memory")
    from paper_2503_14688_b300 import build

    build.build()
    import paper_2503_14688_b300 as P

    return P


@pytest.mark.parametrize("which", ["ising", "blume_capel"])
def test_full_size_light_cone_and_sums(isg, orc, which):
    """The large-quench workload as the benchmark runs it (records every 10
    sweeps), checked at t = 10 and t = 100 on four oracle windows each and
    on the recorded sums."""
    w = wl.ising_large() if which == "ising" else wl.blume_capel_large()
    core = 128
    L = w.L
    lat = isg.Lattice(L, w.model, seed=w.seed, delta=w.delta, record_capacity=16)
    try:
        lat.init_random()
        rng = np.random.default_rng(17)
        done = 0
        for n in (10, 100):
            lat.sweep(n - done, beta=w.beta, record_every=10)
            done = n
            rec = lat.read_records()[-1]
            assert rec.sweep == n
            corners = [(int(a), int(b)) for a, b in rng.integers(0, L, size=(3, 2))]
            corners.append((L - core // 2, L - core // 2))  # straddles both periodic seams
            m = 2 * n + 2
            for (y0, x0) in corners:
                h = core + 2 * m
                wy, wx = (y0 - m) % L, (x0 - m) % L
                win = orc.window_init(h, h, wy, wx, L, w.model, w.seed)
                orc.window_run(win, wy, wx, L, w.model, w.seed, 0, [w.beta] * n, delta=w.delta)
                got = lat.get_rect(y0, x0, core, core)
                assert np.array_equal(got, win[m:m + core, m:m + core]), (n, y0, x0)
            # recorded sums against the GPU's own spins, recomputed on the host
            assert int(rec.R.astype(np.int64).sum()) == rec.M
            assert int(rec.C.astype(np.int64).sum()) == rec.M
            assert abs(rec.B) <= 2 * L * L and rec.Q <= L * L and abs(rec.M) <= rec.Q
            for y in rng.integers(0, L, size=3):
                row = lat.get_rect(int(y), 0, 1, L)
                assert int(row.astype(np.int64).sum()) == int(rec.R[y])
            for x in rng.integers(0, L, size=3):
                col = lat.get_rect(0, int(x), L, 1)
                assert int(col.astype(np.int64).sum()) == int(rec.C[x])
        # the axis correlation sums at full size: S(0) = Q, Sx(1) + Sy(1) = B
        sx, sy = lat.correlation([0, 1, 2, 1000])
        assert sx[0] == rec.Q and sy[0] == rec.Q
        assert sx[1] + sy[1] == rec.B
        # isg_measure on the same state equals the record
        o = lat.measure()
        assert (o.B, o.M, o.Q) == (rec.B, rec.M, rec.Q)
        assert np.array_equal(o.R, rec.R) and np.array_equal(o.C, rec.C)
    finally:
        lat.close()
