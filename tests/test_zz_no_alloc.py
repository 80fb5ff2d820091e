"""isg_measure_planes_noalloc against isg_measure.

The no-allocation entry point exists for callers that cannot obtain device
memory at the moment they measure (all device memory owned by their own pool
allocator, or loops that cannot afford the device-wide synchronisation of
cudaMalloc/cudaFree).  It must give exactly what isg_measure gives -- these
are integer sums, so the tolerance is bit-exact, as in every other parity
test here -- on consecutive calls that reuse its one static scratch array.

It is also checked against the oracle (the plain CPU sweep and observables)
on a lattice the oracle swept, at the largest accepted side L = 2^18 (where
the record fills the static array exactly and the measure kernel runs many
row bands with atomics into it), on the default stream, with the row/column
sums skipped, and for the property behind its name: device memory stays
unchanged over a loop of calls.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

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


def _lattice_on_tensor(isg, model, L, seed, stream):
    import torch

    nbytes = isg.Lattice.nbytes(model, L)
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    lat = isg.Lattice(L, model, seed=seed, delta=0.3 if model == 1 else 0.0, stream=stream,
                      device_buf=buf)
    lat.init_random()
    return lat, buf


def _same(a, b):
    assert (a.B, a.M, a.Q) == (b.B, b.M, b.Q)
    assert np.array_equal(a.R, b.R) and np.array_equal(a.C, b.C)


def test_noalloc_measure_matches_isg_measure(isg):
    import torch

    stream = torch.cuda.Stream()
    ising, ibuf = _lattice_on_tensor(isg, isg.ISING, 512, 11, stream)
    bc, bbuf = _lattice_on_tensor(isg, isg.BLUME_CAPEL, 256, 12, stream)
    ising.sweep(7, beta=0.44)
    bc.sweep(5, beta=0.6)
    # two calls in a row on the shared scratch array (different sizes)
    a1 = isg.measure_planes_noalloc(isg.ISING, 512, ibuf, stream=stream, sweep=7)
    a2 = isg.measure_planes_noalloc(isg.BLUME_CAPEL, 256, bbuf, stream=stream, sweep=5)
    _same(a1, ising.measure())
    _same(a2, bc.measure())
    assert (a1.sweep, a2.sweep) == (7, 5)
    # and again after the lattices changed: nothing left over from before
    ising.sweep(3, beta=0.44)
    b1 = isg.measure_planes_noalloc(isg.ISING, 512, ibuf, stream=stream)
    b2 = isg.measure_planes_noalloc(isg.ISING, 512, ibuf, stream=stream)
    ref = ising.measure()
    _same(b1, ref)
    _same(b2, ref)
    assert (b1.B, b1.M) != (a1.B, a1.M)


def test_noalloc_rejects_sizes_beyond_its_limit(isg):
    import torch

    from paper_2503_14688_b300 import _abi

    lib = isg.lib()
    buf = torch.empty(256, dtype=torch.uint8, device="cuda")
    o = _abi.isg_obs()
    L = _abi.ISG_NOALLOC_MAX_L * 2
    st = lib.isg_measure_planes_noalloc(isg.ISING, L, buf.data_ptr(), None, 0, ctypes.byref(o))
    assert st == _abi.ISG_ERR_INVALID
    assert b"static scratch limit" in lib.isg_last_error()
    st = lib.isg_measure_planes_noalloc(isg.ISING, 100, buf.data_ptr(), None, 0, ctypes.byref(o))
    assert st == _abi.ISG_ERR_INVALID


def test_noalloc_matches_the_oracle(isg):
    """Planes swept on the GPU from the oracle's start give the oracle's
    observables (L = 256, both models, 20 sweeps at the workloads' betas)."""
    import torch

    import oracle
    from paper_2503_14688_b300 import workloads as wl

    stream = torch.cuda.Stream()
    for model, beta, delta in [(isg.ISING, wl.BETA_C_ISING, 0.0),
                               (isg.BLUME_CAPEL, 1.0 / wl.T_C_BLUME_CAPEL, 0.0)]:
        L, n, seed = 256, 20, wl.BASE_SEED + 77
        buf = torch.empty(isg.Lattice.nbytes(model, L), dtype=torch.uint8, device="cuda")
        lat = isg.Lattice(L, model, seed=seed, delta=delta, stream=stream, device_buf=buf)
        lat.init_random()
        lat.sweep(n, beta=beta)
        got = isg.measure_planes_noalloc(model, L, buf, stream=stream, sweep=n)
        s = oracle.init_random(L, model, seed)
        oracle.run(s, model, seed, 0, [beta] * n, delta=delta)
        B, M, Q, R, C = oracle.measure(s)
        assert (got.B, got.M, got.Q) == (int(B), int(M), int(Q))
        assert np.array_equal(got.R, R) and np.array_equal(got.C, C)
        lat.close()


def test_noalloc_at_its_largest_side_on_the_default_stream(isg):
    """L = ISG_NOALLOC_MAX_L = 2^18 (an 8 GiB Ising lattice): the record
    fills the static array exactly; two calls in a row on the default stream
    equal isg_measure, and a call with both sums skipped copies only the
    scalars."""
    import torch

    from paper_2503_14688_b300 import _abi

    L = _abi.ISG_NOALLOC_MAX_L
    model = isg.ISING
    buf = torch.empty(isg.Lattice.nbytes(model, L), dtype=torch.uint8, device="cuda")
    lat = isg.Lattice(L, model, seed=0x5EED18, device_buf=buf)  # default stream
    lat.init_random()
    lat.sweep(2, beta=0.44)
    ref = lat.measure()
    a = isg.measure_planes_noalloc(model, L, buf, sweep=2)
    b = isg.measure_planes_noalloc(model, L, buf, sweep=2)
    _same(a, ref)
    _same(b, ref)
    lib = isg.lib()
    o = _abi.isg_obs()  # row_sums = col_sums = NULL
    assert lib.isg_measure_planes_noalloc(model, L, buf.data_ptr(), None, 9, ctypes.byref(o)) == 0
    assert (o.sweep, o.B, o.M, o.Q) == (9, ref.B, ref.M, ref.Q)
    lat.close()
    del buf
    torch.cuda.empty_cache()


def test_noalloc_leaves_device_memory_unchanged(isg):
    """After one warm-up call, 100 calls at two sides leave the free device
    memory exactly as it was: the call allocates nothing."""
    import torch

    stream = torch.cuda.Stream()
    lats = [_lattice_on_tensor(isg, isg.ISING, 1024, 21, stream),
            _lattice_on_tensor(isg, isg.BLUME_CAPEL, 512, 22, stream)]
    for lat, buf in lats:
        lat.sweep(2, beta=0.5)
        isg.measure_planes_noalloc(lat.model, lat.L, buf, stream=stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for i in range(50):
        for lat, buf in lats:
            isg.measure_planes_noalloc(lat.model, lat.L, buf, stream=stream, sweep=i)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for lat, _ in lats:
        lat.close()
