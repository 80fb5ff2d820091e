"""Argument marshalling for ensembles of independent replicas (isg_ensemble_*).

Every method is one C call; the sweeps run in libisg's persistent kernel.
"""
import ctypes
from typing import List, Optional

import numpy as np

from . import _abi
from ._abi import check, lib
from .lattice import Obs, _stream_handle


class Ensemble:
    """n replicas with sides L[r], models model[r] (default Ising), seeds seed[r]."""

    def __init__(self, L, seeds, models=None, delta: float = 0.0, stream=None,
                 record_capacity: int = 16):
        self._lib = lib()
        self.L = np.ascontiguousarray(np.asarray(L, dtype=np.int64))
        self.n = int(self.L.size)
        self.seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
        assert self.seeds.size == self.n
        self.models = (np.zeros(self.n, dtype=np.int32) if models is None
                       else np.ascontiguousarray(np.asarray(models, dtype=np.int32)))
        self.delta = float(delta)
        d = _abi.isg_ensemble_desc()
        d.n = self.n
        d.L = self.L.ctypes.data_as(_abi._I64P)
        d.model = self.models.ctypes.data_as(_abi._I32P)
        d.seed = self.seeds.ctypes.data_as(_abi._U64P)
        d.delta = self.delta
        d.stream = _stream_handle(stream)
        d.record_capacity = int(record_capacity)
        self._h = ctypes.c_void_p()
        check(self._lib.isg_ensemble_create(ctypes.byref(d), ctypes.byref(self._h)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.isg_ensemble_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_random(self):
        check(self._lib.isg_ensemble_init_random(self._h))

    def sweep(self, n: int, beta=None, betas=None, record_every: int = 0):
        if betas is not None:
            b = np.ascontiguousarray(np.asarray(betas, dtype=np.float64).reshape(-1))
            assert b.size == n
            check(self._lib.isg_ensemble_sweep(self._h, n, b.ctypes.data_as(_abi._F64P), 0.0,
                                               record_every))
        else:
            check(self._lib.isg_ensemble_sweep(self._h, n, None, float(beta), record_every))

    def info(self):
        n, t, p, th = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        check(self._lib.isg_ensemble_info(self._h, ctypes.byref(n), ctypes.byref(t),
                                          ctypes.byref(p), ctypes.byref(th)))
        return {"n": n.value, "sweep": t.value, "pending": p.value, "threads": th.value}

    _TUNING = ("threads_per_cta", "half_teams", "sweeps_per_launch", "multi_words", "multi_band")

    def autotune(self, sweeps: int = 50, with_candidates: bool = False):
        """isg_ensemble_autotune: the chosen launch shape as a dict (and, with
        with_candidates, every candidate tried with its time)."""
        best = _abi.isg_ensemble_tuning()
        tried = (_abi.isg_ensemble_tuning * 64)()
        n = ctypes.c_int64()
        check(self._lib.isg_ensemble_autotune(self._h, int(sweeps), ctypes.byref(best), tried, 64,
                                              ctypes.byref(n)))
        out = {k: getattr(best, k) for k in self._TUNING}
        out["ms"] = best.ms
        if with_candidates:
            cands = [{**{k: getattr(tried[i], k) for k in self._TUNING}, "ms": tried[i].ms,
                      "part": tried[i].part} for i in range(min(n.value, 64))]
            return out, cands
        return out

    def tuning(self) -> dict:
        t = _abi.isg_ensemble_tuning()
        check(self._lib.isg_ensemble_get_tuning(self._h, ctypes.byref(t)))
        return {k: getattr(t, k) for k in self._TUNING}

    def set_tuning(self, **kw):
        t = _abi.isg_ensemble_tuning()
        cur = self.tuning()
        cur.update(kw)
        for k in self._TUNING:
            setattr(t, k, int(cur[k]))
        check(self._lib.isg_ensemble_set_tuning(self._h, ctypes.byref(t)))

    def read_records(self, rows: Optional[int] = None, with_sums: bool = True) -> List[List[Obs]]:
        """Up to `rows` oldest record rows; row i is a list over replicas."""
        k = self.info()["pending"] if rows is None else int(rows)
        if k == 0:
            return []
        obs = (_abi.isg_obs * (k * self.n))()
        keep = []
        if with_sums:
            for i in range(k):
                for r in range(self.n):
                    R = np.zeros(int(self.L[r]), dtype=np.int32)
                    C = np.zeros(int(self.L[r]), dtype=np.int32)
                    keep.append((R, C))
                    obs[i * self.n + r].row_sums = R.ctypes.data_as(_abi._I32P)
                    obs[i * self.n + r].col_sums = C.ctypes.data_as(_abi._I32P)
        cnt = ctypes.c_int64()
        check(self._lib.isg_ensemble_read_records(self._h, k, obs, ctypes.byref(cnt)))
        out = []
        for i in range(cnt.value):
            row = []
            for r in range(self.n):
                o = obs[i * self.n + r]
                R, C = keep[i * self.n + r] if with_sums else (None, None)
                row.append(Obs(o.sweep, o.B, o.M, o.Q, R, C))
            out.append(row)
        return out

    def read_scalars(self, rows: Optional[int] = None):
        """Up to `rows` oldest record rows without the row and column sums, as
        arrays: (sweep[k], B[k, n], M[k, n], Q[k, n]) (int64)."""
        k = self.info()["pending"] if rows is None else int(rows)
        empty = np.zeros((0, self.n), dtype=np.int64)
        if k == 0:
            return np.zeros(0, dtype=np.int64), empty, empty.copy(), empty.copy()
        obs = (_abi.isg_obs * (k * self.n))()
        cnt = ctypes.c_int64()
        check(self._lib.isg_ensemble_read_records(self._h, k, obs, ctypes.byref(cnt)))
        # isg_obs: four int64 (sweep, B, M, Q) then two pointers, 48 bytes
        raw = np.frombuffer(obs, dtype=np.int64).reshape(k, self.n, ctypes.sizeof(_abi.isg_obs) // 8)
        raw = raw[: cnt.value]
        return raw[:, 0, 0].copy(), raw[:, :, 1].copy(), raw[:, :, 2].copy(), raw[:, :, 3].copy()

    def get(self, r: int) -> np.ndarray:
        L = int(self.L[r])
        out = np.empty((L, L), dtype=np.int8)
        check(self._lib.isg_ensemble_get(self._h, int(r), out.ctypes.data_as(_abi._I8P)))
        return out
