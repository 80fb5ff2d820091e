"""isg_measure_planes_noalloc against isg_measure.

The no-allocation entry point exists for callers that cannot obtain device
memory at the moment they measure (all device memory owned by their own pool
allocator, or loops that cannot afford the device-wide synchronisation of
cudaMalloc/cudaFree).  It must give exactly what isg_measure gives -- these
are integer sums, so the tolerance is bit-exact, as in every other parity
test here -- on consecutive calls that reuse its one static scratch array.

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
