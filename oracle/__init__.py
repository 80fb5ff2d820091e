"""The oracle: a plain CPU implementation of the checkerboard Metropolis sweep
of the 2D Ising and Blume-Capel models and of its per-sweep observables.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never calls it, and it never imports the
product package.  Everything it computes is in ``isg_oracle.c``; this module
only marshals numpy arrays into that C code.

Parity status of each function (what pins it is in ``tests/test_oracle_*``):
  philox4x32_10   pinned: black-box agreement with cuRAND's host Philox4_32_10
  threshold       pinned: closed-form error bound, beta = 0 / infinity limits
  init_random     pinned: T = infinity statistics (spin balance, 1/3 split)
  run (sweeps)    pinned: exact enumeration (Ising L=4, Blume-Capel L=3, 4),
                  Kaufman's exact finite-L energy at beta_c, Onsager / Yang
                  off-critical, acceptance frequencies, beta = 0 and
                  beta = infinity limits, global spin-flip symmetry
  measure         pinned: invariants and closed forms on constructed lattices
  xi2             pinned: closed forms on constructed row/column sums
  correlation     pinned: library FFT autocorrelation, S(1) = B, S(0) = Q,
                  constructed lattices (tests/test_oracle_correlation.py)
  window_init/run pinned: equal to init_random/run on the interior of the
                  light cone (tests/test_oracle_windows.py)
  slab_half_sweep pinned: row slabs with halos exchanged every half-sweep
  slab_measure    reproduce run / measure of the whole lattice
                  (tests/test_oracle_slab.py)
"""
import ctypes
import os

import numpy as np

from . import build as _build

ISING = 0
BLUME_CAPEL = 1

_lib = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i8p = ctypes.POINTER(ctypes.c_int8)
        f64p = ctypes.POINTER(ctypes.c_double)
        L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.oracle_philox4x32_10.restype = None
        L.oracle_site_random.argtypes = [ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.c_uint32, ctypes.c_uint32]
        L.oracle_site_random.restype = ctypes.c_uint32
        L.oracle_threshold.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int]
        L.oracle_threshold.restype = ctypes.c_uint64
        L.oracle_bc_proposal.argtypes = [ctypes.c_int, ctypes.c_int]
        L.oracle_bc_proposal.restype = ctypes.c_int
        L.oracle_init_random.argtypes = [i8p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64]
        L.oracle_init_random.restype = ctypes.c_int
        L.oracle_measure.argtypes = [i8p, ctypes.c_int64, i64p, i32p, i32p]
        L.oracle_measure.restype = ctypes.c_int
        L.oracle_run.argtypes = [i8p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                                 ctypes.c_uint64, ctypes.c_int64, f64p, ctypes.c_double,
                                 ctypes.c_int64, i64p, i32p, i32p, ctypes.c_int, ctypes.c_int]
        L.oracle_run.restype = ctypes.c_int64
        L.oracle_xi2.argtypes = [ctypes.c_int64, ctypes.c_int64, i64p, i32p, i32p]
        L.oracle_xi2.restype = ctypes.c_double
        L.oracle_correlation.argtypes = [i8p, ctypes.c_int64, ctypes.c_int64, i64p, i64p, i64p]
        L.oracle_sw_threshold.argtypes = [ctypes.c_double]
        L.oracle_sw_threshold.restype = ctypes.c_uint64
        L.oracle_swendsen_wang.argtypes = [i8p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_double, i64p]
        L.oracle_swendsen_wang.restype = ctypes.c_int64
        L.oracle_correlation.restype = ctypes.c_int
        L.oracle_window_init.argtypes = [i8p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64]
        L.oracle_window_init.restype = ctypes.c_int
        L.oracle_window_run.argtypes = [i8p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                                        ctypes.c_uint64, ctypes.c_int64, f64p, ctypes.c_double]
        L.oracle_window_run.restype = ctypes.c_int
        L.oracle_slab_half_sweep.argtypes = [i8p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                             ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.oracle_slab_half_sweep.restype = ctypes.c_int
        L.oracle_slab_measure.argtypes = [i8p, ctypes.c_int64, ctypes.c_int64, i64p, i32p, i32p]
        L.oracle_slab_measure.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def philox4x32_10(ctr, key):
    """Philox4x32-10 of one 4-word counter and 2-word key -> 4 words."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def site_random(seed: int, j: int, w2: int, w3: int) -> int:
    """Random word of same-colour index j for counter words (w2, w3)."""
    return int(lib().oracle_site_random(seed & (2**64 - 1), j, w2 & 0xFFFFFFFF,
                                        w3 & 0xFFFFFFFF))


def threshold(beta: float, dE: float, bits: int) -> int:
    """rne(2^bits exp(-beta dE)) for dE > 0; 2^bits (always accept) for dE <= 0."""
    return int(lib().oracle_threshold(float(beta), float(dE), int(bits)))


def bc_proposal(s: int, b: int) -> int:
    return int(lib().oracle_bc_proposal(int(s), int(b)))


def init_random(L: int, model: int, seed: int) -> np.ndarray:
    """Hot start: an L x L int8 lattice drawn from the beta = 0 measure."""
    s = np.zeros((L, L), dtype=np.int8)
    rc = lib().oracle_init_random(_ptr(s, ctypes.c_int8), L, model, seed & (2**64 - 1))
    if rc != 0:
        raise ValueError("oracle_init_random rejected its arguments")
    return s


def measure(s: np.ndarray):
    """(B, M, Q, R[L], C[L]) of a lattice; energy per spin = (-B + Delta Q)/L^2."""
    s = np.ascontiguousarray(s, dtype=np.int8)
    L = s.shape[0]
    bmq = np.zeros(3, dtype=np.int64)
    R = np.zeros(L, dtype=np.int32)
    C = np.zeros(L, dtype=np.int32)
    rc = lib().oracle_measure(_ptr(s, ctypes.c_int8), L, _ptr(bmq, ctypes.c_int64),
                              _ptr(R, ctypes.c_int32), _ptr(C, ctypes.c_int32))
    if rc != 0:
        raise ValueError("oracle_measure rejected its arguments")
    return int(bmq[0]), int(bmq[1]), int(bmq[2]), R, C


def run(s: np.ndarray, model: int, seed: int, t0: int, betas, delta: float = 0.0,
        record_every: int = 0, with_rows: bool = True, nthreads: int = 1,
        sequential: bool = False):
    """Advance lattice ``s`` in place by len(betas) sweeps t0, t0+1, ...

    Returns (bmq[nrec,3], R[nrec,L], C[nrec,L]) of the recorded sweeps (R and
    C are None when with_rows is False).
    """
    assert s.dtype == np.int8 and s.flags.c_contiguous and s.shape[0] == s.shape[1]
    L = s.shape[0]
    betas = np.ascontiguousarray(np.asarray(betas, dtype=np.float64).reshape(-1))
    n = betas.size
    nrec_max = n // record_every if record_every > 0 else 0
    bmq = np.zeros((max(nrec_max, 1), 3), dtype=np.int64)
    R = C = None
    Rp = Cp = ctypes.POINTER(ctypes.c_int32)()
    if with_rows and nrec_max > 0:
        R = np.zeros((nrec_max, L), dtype=np.int32)
        C = np.zeros((nrec_max, L), dtype=np.int32)
        Rp, Cp = _ptr(R, ctypes.c_int32), _ptr(C, ctypes.c_int32)
    nrec = lib().oracle_run(_ptr(s, ctypes.c_int8), L, model, seed & (2**64 - 1), t0, n,
                            _ptr(betas, ctypes.c_double), float(delta), record_every,
                            _ptr(bmq, ctypes.c_int64), Rp, Cp, int(nthreads),
                            int(bool(sequential)))
    if nrec < 0:
        raise ValueError("oracle_run rejected its arguments")
    return bmq[:nrec], (R[:nrec] if R is not None else None), (C[:nrec] if C is not None else None)


def xi2(M, R, C) -> float:
    """Ensemble second-moment correlation length from n replicas' M, R, C."""
    M = np.ascontiguousarray(np.asarray(M, dtype=np.int64).reshape(-1))
    R = np.ascontiguousarray(np.asarray(R, dtype=np.int32))
    C = np.ascontiguousarray(np.asarray(C, dtype=np.int32))
    n = M.size
    L = R.size // max(n, 1)
    assert R.size == n * L and C.size == n * L
    return float(lib().oracle_xi2(n, L, _ptr(M, ctypes.c_int64), _ptr(R, ctypes.c_int32),
                                  _ptr(C, ctypes.c_int32)))


def window_init(h: int, w: int, y0: int, x0: int, L: int, model: int, seed: int) -> np.ndarray:
    """Hot start of the h x w window at (y0, x0) of an L x L lattice (global keys)."""
    s = np.zeros((h, w), dtype=np.int8)
    rc = lib().oracle_window_init(_ptr(s, ctypes.c_int8), h, w, y0, x0, L, model,
                                  seed & (2**64 - 1))
    if rc != 0:
        raise ValueError("oracle_window_init rejected its arguments")
    return s


def window_run(s: np.ndarray, y0: int, x0: int, L: int, model: int, seed: int, t0: int, betas,
               delta: float = 0.0):
    """Sweep a window in place with global keys, its outer ring held fixed;
    after n sweeps the sites farther than 2n from the ring are exact."""
    assert s.dtype == np.int8 and s.flags.c_contiguous
    h, w = s.shape
    betas = np.ascontiguousarray(np.asarray(betas, dtype=np.float64).reshape(-1))
    rc = lib().oracle_window_run(_ptr(s, ctypes.c_int8), h, w, y0, x0, L, model,
                                 seed & (2**64 - 1), t0, betas.size,
                                 _ptr(betas, ctypes.c_double), float(delta))
    if rc != 0:
        raise ValueError("oracle_window_run rejected its arguments")


def correlation(s: np.ndarray, r):
    """(sx[k], sy[k]) = sums of s(x,y) s(x+r_k,y) and s(x,y) s(x,y+r_k)."""
    s = np.ascontiguousarray(s, dtype=np.int8)
    L = s.shape[0]
    r = np.ascontiguousarray(np.asarray(r, dtype=np.int64).reshape(-1))
    sx = np.zeros(r.size, dtype=np.int64)
    sy = np.zeros(r.size, dtype=np.int64)
    rc = lib().oracle_correlation(_ptr(s, ctypes.c_int8), L, r.size, _ptr(r, ctypes.c_int64),
                                  _ptr(sx, ctypes.c_int64), _ptr(sy, ctypes.c_int64))
    if rc != 0:
        raise ValueError("oracle_correlation rejected its arguments")
    return sx, sy


def sw_threshold(beta: float) -> int:
    """Bond threshold rne(2^32 (1 - exp(-2 beta))) of the Swendsen-Wang step."""
    return int(lib().oracle_sw_threshold(float(beta)))


def swendsen_wang(s: np.ndarray, seed: int, k: int, beta: float):
    """One Swendsen-Wang iteration of the +-1 sites of ``s`` (in place), the
    k-th on this lattice.  Returns (labels[L, L] int64, number of clusters)."""
    assert s.dtype == np.int8 and s.flags.c_contiguous and s.shape[0] == s.shape[1]
    L = s.shape[0]
    labels = np.empty((L, L), dtype=np.int64)
    n = lib().oracle_swendsen_wang(_ptr(s, ctypes.c_int8), L, seed & (2**64 - 1), int(k),
                                   float(beta), _ptr(labels, ctypes.c_int64))
    if n < 0:
        raise ValueError("oracle_swendsen_wang rejected its arguments")
    return labels, int(n)


def slab_half_sweep(s: np.ndarray, y0: int, model: int, seed: int, t: int, c: int, beta: float,
                    delta: float = 0.0):
    """Half-sweep of colour c of a row slab in place: s is (rows + 2) x L,
    rows 1..rows the owned global rows y0.., rows 0 and rows + 1 the halos."""
    assert s.dtype == np.int8 and s.flags.c_contiguous
    rows, L = s.shape[0] - 2, s.shape[1]
    rc = lib().oracle_slab_half_sweep(_ptr(s, ctypes.c_int8), rows, L, y0, model,
                                      seed & (2**64 - 1), t, c, float(beta), float(delta))
    if rc != 0:
        raise ValueError("oracle_slab_half_sweep rejected its arguments")


def slab_measure(s: np.ndarray):
    """(B, M, Q, R[rows], C[L]) of the owned rows of a slab (see slab_half_sweep)."""
    s = np.ascontiguousarray(s, dtype=np.int8)
    rows, L = s.shape[0] - 2, s.shape[1]
    bmq = np.zeros(3, dtype=np.int64)
    R = np.zeros(rows, dtype=np.int32)
    C = np.zeros(L, dtype=np.int32)
    rc = lib().oracle_slab_measure(_ptr(s, ctypes.c_int8), rows, L, _ptr(bmq, ctypes.c_int64),
                                   _ptr(R, ctypes.c_int32), _ptr(C, ctypes.c_int32))
    if rc != 0:
        raise ValueError("oracle_slab_measure rejected its arguments")
    return int(bmq[0]), int(bmq[1]), int(bmq[2]), R, C
