"""Argument marshalling for the request server (isg_server_*)."""
import ctypes
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from . import _abi
from ._abi import check, lib
from .lattice import Obs, _stream_handle


@dataclass
class Result:
    state: int
    sweeps_done: int
    B: int
    M: int
    Q: int
    t_arrival: float
    t_admit: float
    t_done: float
    records: int
    error: int = 0


class Server:
    def __init__(self, hbm_budget: int, max_active: int = 64, chunk_sweeps: int = 100,
                 stream=None):
        self._lib = lib()
        d = _abi.isg_server_desc(int(hbm_budget), int(max_active), int(chunk_sweeps),
                                 _stream_handle(stream))
        self._h = ctypes.c_void_p()
        check(self._lib.isg_server_create(ctypes.byref(d), ctypes.byref(self._h)))
        self.L = {}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.isg_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def clock(self) -> float:
        return float(self._lib.isg_server_clock(self._h))

    def submit(self, model: int, L: int, seed: int, n_sweeps: int, t_start, beta,
               delta: float = 0.0, record_every: int = 0, keep: bool = False,
               arrival_time: float = -1.0, deadline: float = 0.0) -> int:
        ts = np.ascontiguousarray(np.asarray(t_start, dtype=np.int64))
        bs = np.ascontiguousarray(np.asarray(beta, dtype=np.float64))
        q = _abi.isg_request(int(model), int(L), int(seed) & (2**64 - 1), float(delta),
                             int(n_sweeps), ts.size, ts.ctypes.data_as(_abi._I64P),
                             bs.ctypes.data_as(_abi._F64P), int(record_every), int(bool(keep)),
                             float(arrival_time), float(deadline))
        rid = ctypes.c_uint64()
        check(self._lib.isg_server_submit(self._h, ctypes.byref(q), ctypes.byref(rid)))
        self.L[rid.value] = int(L)
        return rid.value

    def step(self):
        a, q = ctypes.c_int32(), ctypes.c_int32()
        check(self._lib.isg_server_step(self._h, ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def drain(self):
        check(self._lib.isg_server_drain(self._h))

    def poll(self, rid: int) -> Result:
        r = _abi.isg_result()
        check(self._lib.isg_server_poll(self._h, rid, ctypes.byref(r)))
        return Result(r.state, r.sweeps_done, r.B, r.M, r.Q, r.t_arrival, r.t_admit, r.t_done,
                      r.records, r.error)

    def cancel(self, rid: int):
        check(self._lib.isg_server_cancel(self._h, rid))

    def read_records(self, rid: int) -> List[Obs]:
        n = self.poll(rid).records
        if n == 0:
            return []
        L = self.L[rid]
        obs = (_abi.isg_obs * n)()
        R = np.zeros((n, L), dtype=np.int32)
        C = np.zeros((n, L), dtype=np.int32)
        for i in range(n):
            obs[i].row_sums = R[i].ctypes.data_as(_abi._I32P)
            obs[i].col_sums = C[i].ctypes.data_as(_abi._I32P)
        cnt = ctypes.c_int64()
        check(self._lib.isg_server_read_records(self._h, rid, obs, n, ctypes.byref(cnt)))
        return [Obs(obs[i].sweep, obs[i].B, obs[i].M, obs[i].Q, R[i], C[i])
                for i in range(cnt.value)]

    def get_lattice(self, rid: int) -> np.ndarray:
        L = self.L[rid]
        out = np.empty((L, L), dtype=np.int8)
        check(self._lib.isg_server_get_lattice(self._h, rid, out.ctypes.data_as(_abi._I8P)))
        return out

    def release(self, rid: int):
        check(self._lib.isg_server_release(self._h, rid))

    def stats(self):
        f = ctypes.c_double()
        used, budget = ctypes.c_size_t(), ctypes.c_size_t()
        check(self._lib.isg_server_stats(self._h, ctypes.byref(f), ctypes.byref(used),
                                         ctypes.byref(budget)))
        return {"flips_done": f.value, "bytes_in_use": used.value, "budget": budget.value}
