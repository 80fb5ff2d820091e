"""Pins of the oracle's row-slab functions (domain decomposition, Introduction:
one lattice spread over many GPUs, each holding a part of it).

The slab functions are pinned to the whole-lattice oracle (itself pinned by
exact enumeration, Onsager/Yang, limits): a lattice cut into P row slabs,
with each slab's halo rows copied from its neighbours' edge rows before every
half-sweep, must reproduce ``oracle.run`` bit for bit, and the slabs' parts
of the observables must add up to ``oracle.measure``.  The exchange here is
written independently of the package's decomposition driver.
"""
import numpy as np
import pytest

import oracle

BETA = {0: 0.44068679350977147, 1: 1 / 1.69355839821214427017}


def _cut(L, P):
    step = L // P
    return [(k * step, step if k < P - 1 else L - k * step) for k in range(P)]


def _slabs_from(s, parts):
    L = s.shape[0]
    out = []
    for y0, rows in parts:
        b = np.zeros((rows + 2, L), dtype=np.int8)
        b[1:rows + 1] = s[y0:y0 + rows]
        out.append(b)
    return out


def _exchange(slabs):
    P = len(slabs)
    for k, b in enumerate(slabs):
        b[0] = slabs[(k - 1) % P][-2]  # last owned row of the slab above
        b[-1] = slabs[(k + 1) % P][1]  # first owned row of the slab below


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("L,P", [(64, 1), (64, 2), (128, 4), (96, 3)])
def test_slabs_reproduce_the_whole_lattice(model, L, P):
    seed, n = 0x5EED0 + 7 * L + P, 6
    delta = 0.3 if model == 1 else 0.0
    s = oracle.init_random(L, model, seed)
    parts = _cut(L, P)
    slabs = _slabs_from(s, parts)
    betas = [BETA[model] * (1 + 0.1 * i) for i in range(n)]
    for t in range(n):
        for c in (0, 1):
            _exchange(slabs)
            for (y0, _), b in zip(parts, slabs):
                oracle.slab_half_sweep(b, y0, model, seed, t, c, betas[t], delta)
    oracle.run(s, model, seed, 0, betas, delta=delta)
    union = np.concatenate([b[1:-1] for b in slabs])
    assert np.array_equal(union, s)


@pytest.mark.parametrize("model", [0, 1])
def test_slab_observables_add_up(model):
    rng = np.random.default_rng(5)
    L = 96
    vals = [-1, 1] if model == 0 else [-1, 0, 1]
    s = rng.choice(vals, size=(L, L)).astype(np.int8)
    parts = _cut(L, 3)
    slabs = _slabs_from(s, parts)
    _exchange(slabs)
    B = M = Q = 0
    R, C = [], np.zeros(L, dtype=np.int64)
    for b in slabs:
        b_, m_, q_, r_, c_ = oracle.slab_measure(b)
        B, M, Q = B + b_, M + m_, Q + q_
        R.append(r_)
        C += c_
    B0, M0, Q0, R0, C0 = oracle.measure(s)
    assert (B, M, Q) == (B0, M0, Q0)
    assert np.array_equal(np.concatenate(R), R0) and np.array_equal(C, C0)


def test_slab_keys_are_global():
    """A slab swept with the wrong first row (its keys shifted) departs from
    the whole lattice: the pin above sees the keying."""
    L, model, seed = 64, 0, 99
    s = oracle.init_random(L, model, seed)
    parts = _cut(L, 2)
    slabs = _slabs_from(s, parts)
    for c in (0, 1):
        _exchange(slabs)
        oracle.slab_half_sweep(slabs[0], 0, model, seed, 0, c, 0.3)
        oracle.slab_half_sweep(slabs[1], 0, model, seed, 0, c, 0.3)  # should be y0 = 32
    oracle.run(s, model, seed, 0, [0.3])
    assert not np.array_equal(np.concatenate([b[1:-1] for b in slabs]), s)
