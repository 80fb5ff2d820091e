"""Argument marshalling for one lattice of libisg (include/isg.h).

Every method is one C call: numpy arrays become host pointers, a torch
stream becomes a ``cudaStream_t`` handle, a torch tensor can lend the device
memory for the spins.  No arithmetic of the method happens here.
"""
import ctypes
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import _abi
from ._abi import check, lib


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


@dataclass
class Obs:
    """One observable record (see isg_obs)."""
    sweep: int
    B: int
    M: int
    Q: int
    R: Optional[np.ndarray]
    C: Optional[np.ndarray]

    def energy(self, L: int, delta: float = 0.0) -> float:
        return (-self.B + delta * self.Q) / (L * L)


class Lattice:
    """An L x L lattice on the current CUDA device (isg_lattice_create)."""

    def __init__(self, L: int, model: int = _abi.ISG_ISING, seed: int = 0, delta: float = 0.0,
                 stream=None, device_buf=None, record_capacity: int = 16):
        self._lib = lib()
        self.L = int(L)
        self.model = int(model)
        self.delta = float(delta) if model == _abi.ISG_BLUME_CAPEL else 0.0
        self._buf = device_buf  # keep a lent torch tensor alive
        d = _abi.isg_lattice_desc()
        d.model = self.model
        d.L = self.L
        d.seed = int(seed) & (2**64 - 1)
        d.delta = float(delta)
        d.stream = _stream_handle(stream)
        if device_buf is not None:
            d.device_buf = int(device_buf.data_ptr())
            d.device_buf_bytes = int(device_buf.numel() * device_buf.element_size())
        d.record_capacity = int(record_capacity)
        self._h = ctypes.c_void_p()
        check(self._lib.isg_lattice_create(ctypes.byref(d), ctypes.byref(self._h)))

    @staticmethod
    def nbytes(model: int, L: int) -> int:
        return int(lib().isg_lattice_bytes(model, L))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.isg_lattice_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state ------------------------------------------------------------
    def init_random(self):
        check(self._lib.isg_lattice_init_random(self._h))

    def init_uniform(self, value: int):
        check(self._lib.isg_lattice_init_uniform(self._h, int(value)))

    def set(self, spins: np.ndarray, t: int = 0):
        s = np.ascontiguousarray(spins, dtype=np.int8)
        assert s.shape == (self.L, self.L)
        check(self._lib.isg_lattice_set(self._h, s.ctypes.data_as(_abi._I8P), int(t)))

    def get(self) -> np.ndarray:
        out = np.empty((self.L, self.L), dtype=np.int8)
        check(self._lib.isg_lattice_get(self._h, out.ctypes.data_as(_abi._I8P)))
        return out

    def get_rect(self, y0: int, x0: int, h: int, w: int) -> np.ndarray:
        out = np.empty((h, w), dtype=np.int8)
        check(self._lib.isg_lattice_get_rect(self._h, y0, x0, h, w,
                                             out.ctypes.data_as(_abi._I8P)))
        return out

    def save(self, path: str):
        """Checkpoint to a file (isg_save)."""
        check(self._lib.isg_save(self._h, str(path).encode()))

    @classmethod
    def load(cls, path: str, stream=None, record_capacity: int = 16) -> "Lattice":
        """Resume from a checkpoint file (isg_load)."""
        self = cls.__new__(cls)
        self._lib = lib()
        self._buf = None
        self._h = ctypes.c_void_p()
        check(self._lib.isg_load(str(path).encode(), _stream_handle(stream), int(record_capacity),
                                 ctypes.byref(self._h)))
        L, model = ctypes.c_int64(), ctypes.c_int32()
        check(self._lib.isg_lattice_info(self._h, None, ctypes.byref(L), ctypes.byref(model), None))
        self.L, self.model = L.value, model.value
        self.delta = 0.0
        return self

    @property
    def sweep_index(self) -> int:
        t = ctypes.c_int64()
        check(self._lib.isg_lattice_info(self._h, ctypes.byref(t), None, None, None))
        return t.value

    # -- dynamics -----------------------------------------------------------
    def sweep(self, n: int, beta=None, betas=None, record_every: int = 0):
        """n sweeps at constant beta, or at betas[i] for sweep i of this call."""
        if betas is not None:
            b = np.ascontiguousarray(np.asarray(betas, dtype=np.float64).reshape(-1))
            assert b.size == n
            check(self._lib.isg_sweep(self._h, n, b.ctypes.data_as(_abi._F64P), 0.0,
                                      record_every))
        else:
            check(self._lib.isg_sweep(self._h, n, None, float(beta), record_every))

    def sweep_schedule(self, n: int, t_start, beta, record_every: int = 0):
        ts = np.ascontiguousarray(np.asarray(t_start, dtype=np.int64))
        bs = np.ascontiguousarray(np.asarray(beta, dtype=np.float64))
        sch = _abi.isg_schedule(ts.size, ts.ctypes.data_as(_abi._I64P),
                                bs.ctypes.data_as(_abi._F64P))
        check(self._lib.isg_sweep_schedule(self._h, n, ctypes.byref(sch), record_every))

    def half_sweep(self, colour: int, beta: float):
        check(self._lib.isg_half_sweep(self._h, int(colour), float(beta)))

    def record(self):
        check(self._lib.isg_record(self._h))

    # -- observables --------------------------------------------------------
    def pending(self) -> int:
        n = ctypes.c_int64()
        check(self._lib.isg_pending_records(self._h, ctypes.byref(n)))
        return n.value

    def read_records(self, max_records: Optional[int] = None, with_sums: bool = True):
        n = self.pending() if max_records is None else int(max_records)
        if n == 0:
            return []
        obs = (_abi.isg_obs * n)()
        R = C = None
        if with_sums:
            R = np.zeros((n, self.L), dtype=np.int32)
            C = np.zeros((n, self.L), dtype=np.int32)
            for i in range(n):
                obs[i].row_sums = R[i].ctypes.data_as(_abi._I32P)
                obs[i].col_sums = C[i].ctypes.data_as(_abi._I32P)
        cnt = ctypes.c_int64()
        check(self._lib.isg_read_records(self._h, obs, n, ctypes.byref(cnt)))
        return [Obs(obs[i].sweep, obs[i].B, obs[i].M, obs[i].Q,
                    R[i] if with_sums else None, C[i] if with_sums else None)
                for i in range(cnt.value)]

    def correlation(self, r):
        """(Sx[k], Sy[k]): axis correlation sums at distances r[k] (isg_correlation)."""
        r = np.ascontiguousarray(np.asarray(r, dtype=np.int64).reshape(-1))
        sx = np.zeros(r.size, dtype=np.int64)
        sy = np.zeros(r.size, dtype=np.int64)
        check(self._lib.isg_correlation(self._h, r.size, r.ctypes.data_as(_abi._I64P),
                                        sx.ctypes.data_as(_abi._I64P), sy.ctypes.data_as(_abi._I64P)))
        return sx, sy

    def swendsen_wang(self, beta: float, n: int = 1):
        """n Swendsen-Wang iterations of the +-1 spins at beta
        (isg_swendsen_wang; Appendix B)."""
        for _ in range(int(n)):
            check(self._lib.isg_swendsen_wang(self._h, float(beta)))

    def sw_labels(self) -> np.ndarray:
        """Cluster labels (smallest site index) of the last Swendsen-Wang
        iteration, (L, L) int32."""
        out = np.empty((self.L, self.L), dtype=np.int32)
        check(self._lib.isg_sw_labels(self._h, out.ctypes.data_as(_abi._I32P)))
        return out

    @property
    def sw_iterations(self) -> int:
        c = ctypes.c_int64()
        check(self._lib.isg_sw_iterations(self._h, ctypes.byref(c)))
        return c.value

    def emcs(self, n: int, beta: float, sweeps: int = 10, record_every: int = 0):
        """n elementary Monte Carlo steps of Appendix B: `sweeps` Metropolis
        sweeps then one Swendsen-Wang iteration; with record_every = k > 0
        the observables are recorded after every k-th step."""
        for i in range(1, int(n) + 1):
            if sweeps:
                self.sweep(sweeps, beta=beta)
            self.swendsen_wang(beta)
            if record_every and i % record_every == 0:
                self.record()

    def measure(self) -> Obs:
        R = np.zeros(self.L, dtype=np.int32)
        C = np.zeros(self.L, dtype=np.int32)
        o = _abi.isg_obs()
        o.row_sums = R.ctypes.data_as(_abi._I32P)
        o.col_sums = C.ctypes.data_as(_abi._I32P)
        check(self._lib.isg_measure(self._h, ctypes.byref(o)))
        return Obs(o.sweep, o.B, o.M, o.Q, R, C)


def xi2(M, R, C) -> float:
    """Ensemble xi_2 (isg_xi2) from n replicas' M[n], R[n, L], C[n, L]."""
    M = np.ascontiguousarray(np.asarray(M, dtype=np.int64).reshape(-1))
    R = np.ascontiguousarray(np.asarray(R, dtype=np.int32))
    C = np.ascontiguousarray(np.asarray(C, dtype=np.int32))
    n = M.size
    L = R.size // max(n, 1)
    return float(lib().isg_xi2(n, L, M.ctypes.data_as(_abi._I64P), R.ctypes.data_as(_abi._I32P),
                               C.ctypes.data_as(_abi._I32P)))


def measure_planes_noalloc(model: int, L: int, planes, stream=None, sweep: int = 0) -> Obs:
    """isg_measure_planes_noalloc: observables of spin planes held in caller
    device memory (``planes``: a torch tensor or a raw device address), with
    no device allocation inside the call."""
    ptr = planes if isinstance(planes, int) else int(planes.data_ptr())
    R = np.zeros(L, dtype=np.int32)
    C = np.zeros(L, dtype=np.int32)
    o = _abi.isg_obs()
    o.row_sums = R.ctypes.data_as(_abi._I32P)
    o.col_sums = C.ctypes.data_as(_abi._I32P)
    check(lib().isg_measure_planes_noalloc(int(model), int(L), ptr, _stream_handle(stream),
                                           int(sweep), ctypes.byref(o)))
    return Obs(o.sweep, o.B, o.M, o.Q, R, C)


def xi_integral(r, c, r_cut: float) -> float:
    """xi = I2/I1 of a sampled C(r) up to r_cut (isg_xi_integral)."""
    r = np.ascontiguousarray(np.asarray(r, dtype=np.float64))
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64))
    return float(lib().isg_xi_integral(r.size, r.ctypes.data_as(_abi._F64P),
                                       c.ctypes.data_as(_abi._F64P), float(r_cut)))


def inject_fault(what: int, after: int):
    """isg_debug_inject: the after-th device allocation (what =
    ISG_INJECT_ALLOC) or sweep launch (ISG_INJECT_LAUNCH) from now on fails,
    or the after-th streamed record pass runs out its bounded waits
    (ISG_INJECT_WAIT); once; after = 0 disarms.  For testing error paths
    without a device fault."""
    check(lib().isg_debug_inject(int(what), int(after)))
