"""Domain decomposition of one lattice into row slabs -- how the paper runs a
single lattice on many GPUs (Introduction; Table I: L = 2^22 on 64 GPUs).

Host logic only: which rows each slab owns, the halo exchange before every
half-sweep, and the merge of the slabs' observables.  Every step of the
sweep runs in libisg (``isg_slab_*``, include/isg.h); ``Slab`` below only
marshals arguments into it.

One sweep t, on every slab (the order isg.h states):
    colour-1 edge rows -> neighbours' halos; half-sweep colour 0 at beta(t);
    colour-0 edge rows -> neighbours' halos; half-sweep colour 1 at beta(t).
A slab's first owned row becomes the ``below`` halo of the slab above it,
its last owned row the ``above`` halo of the slab below it (periodic).  The
records of the whole lattice are the sums of the slabs' B, M, Q and column
sums and the concatenation of their row sums (before a record the colour-1
halos, one half-sweep old after a sweep, are exchanged once more).

``Decomposition`` drives any engines with the slab interface (``edges``,
``set_halos``, ``half_sweep``, ``measure``, ``y0``, ``rows``) through an
exchange: ``LocalExchange`` when all slabs live in this process (several on
one GPU, or one per GPU of this process), ``DistExchange`` when each process
of a ``torch.distributed`` group holds one slab (gloo: through host memory;
NCCL: device to device).
"""
import ctypes
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import _abi
from ._abi import check, lib
from .lattice import Obs, _stream_handle


def partition(L: int, P: int, quantum: int = 16) -> List[Tuple[int, int]]:
    """(y0, rows) of P row slabs covering an L-row lattice, each a multiple
    of `quantum` rows, as equal as that allows (the first slabs get the
    extra quanta)."""
    if L % quantum != 0 or P < 1 or P * quantum > L:
        raise ValueError(f"cannot cut L = {L} into {P} slabs of multiples of {quantum} rows")
    q = L // quantum
    out, y0 = [], 0
    for k in range(P):
        rows = (q // P + (1 if k < q % P else 0)) * quantum
        out.append((y0, rows))
        y0 += rows
    return out


class Slab:
    """One row slab on the current CUDA device (isg_slab_create).  Edge and
    halo rows are torch uint8 tensors of ``edge_bytes`` bytes, on the device
    (``host_edges=False``) or in pinned host memory (``host_edges=True``, for
    an exchange through the host)."""

    def __init__(self, model: int, L: int, y0: int, rows: int, seed: int = 0, delta: float = 0.0,
                 stream=None, host_edges: bool = False):
        import torch

        self._lib = lib()
        self.model, self.L, self.y0, self.rows = int(model), int(L), int(y0), int(rows)
        d = _abi.isg_slab_desc()
        d.model, d.L, d.y0, d.rows = self.model, self.L, self.y0, self.rows
        d.seed = int(seed) & (2**64 - 1)
        d.delta = float(delta)
        d.stream = _stream_handle(stream)
        self._h = ctypes.c_void_p()
        check(self._lib.isg_slab_create(ctypes.byref(d), ctypes.byref(self._h)))
        self.edge_bytes = int(self._lib.isg_slab_edge_bytes(self.model, self.L))
        dev = "cpu" if host_edges else "cuda"
        kw = {"pin_memory": True} if host_edges else {}
        self._edge = [[torch.empty(self.edge_bytes, dtype=torch.uint8, device=dev, **kw)
                       for _ in range(2)] for _ in range(2)]

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.isg_slab_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_random(self):
        check(self._lib.isg_slab_init_random(self._h))

    def set(self, s: np.ndarray, t: int = 0):
        s = np.ascontiguousarray(s, dtype=np.int8)
        assert s.shape == (self.rows, self.L)
        check(self._lib.isg_slab_set(self._h, s.ctypes.data_as(_abi._I8P), int(t)))

    def get(self) -> np.ndarray:
        out = np.empty((self.rows, self.L), dtype=np.int8)
        check(self._lib.isg_slab_get(self._h, out.ctypes.data_as(_abi._I8P)))
        return out

    def edges(self, colour: int):
        """(first, last) owned rows of colour `colour` (tensors reused per colour)."""
        first, last = self._edge[colour]
        check(self._lib.isg_slab_edges(self._h, int(colour), first.data_ptr(), last.data_ptr()))
        return first, last

    def set_halos(self, colour: int, above, below):
        check(self._lib.isg_slab_set_halos(self._h, int(colour), int(above.data_ptr()),
                                           int(below.data_ptr())))

    def half_sweep(self, colour: int, beta: float):
        check(self._lib.isg_slab_half_sweep(self._h, int(colour), float(beta)))

    def measure(self):
        """(sweep, B, M, Q, row sums [rows], partial column sums [L])."""
        R = np.zeros(self.rows, dtype=np.int32)
        C = np.zeros(self.L, dtype=np.int32)
        o = _abi.isg_obs()
        o.row_sums = R.ctypes.data_as(_abi._I32P)
        o.col_sums = C.ctypes.data_as(_abi._I32P)
        check(self._lib.isg_slab_measure(self._h, ctypes.byref(o)))
        return int(o.sweep), int(o.B), int(o.M), int(o.Q), R, C

    @property
    def sweep_count(self) -> int:
        t = ctypes.c_int64()
        check(self._lib.isg_slab_info(self._h, ctypes.byref(t), None, None, None, None))
        return int(t.value)


def _merge(parts: Sequence[Tuple[int, int, int, int, np.ndarray, np.ndarray]]) -> Obs:
    """Whole-lattice record from the slabs' parts, in slab order."""
    sweeps = {p[0] for p in parts}
    if len(sweeps) != 1:
        raise RuntimeError(f"slabs at different sweeps: {sorted(sweeps)}")
    C = np.zeros_like(parts[0][5], dtype=np.int64)
    for p in parts:
        C += p[5]
    return Obs(parts[0][0], sum(p[1] for p in parts), sum(p[2] for p in parts),
               sum(p[3] for p in parts), np.concatenate([p[4] for p in parts]).astype(np.int32),
               C.astype(np.int32))


class LocalExchange:
    """All P slabs in this process: halos are the neighbours' edge rows."""

    def __init__(self, world: int):
        self.world = world

    def exchange(self, edges: Dict[int, tuple]) -> Dict[int, tuple]:
        P = self.world
        return {r: (edges[(r - 1) % P][1], edges[(r + 1) % P][0]) for r in edges}

    def merge(self, parts: Dict[int, tuple]) -> Obs:
        return _merge([parts[r] for r in sorted(parts)])


class DistExchange:
    """One slab per process of a torch.distributed group; rank r owns slab r.
    Edge rows go point to point to the two neighbour ranks (no collective);
    records are merged by all-reduce (B, M, Q, column sums) and all-gather
    (row sums).  ``device``: where the collective's tensors live ("cpu" for
    gloo, "cuda" for NCCL)."""

    def __init__(self, rank: int, world: int, rows: Sequence[int], group=None, device="cpu"):
        self.rank, self.world, self.rows = rank, world, list(rows)
        self.group, self.device = group, device

    def exchange(self, edges: Dict[int, tuple]) -> Dict[int, tuple]:
        import torch
        import torch.distributed as dist

        (r, (first, last)), = edges.items()
        P = self.world
        if P == 1:
            return {r: (last, first)}
        first_t = torch.as_tensor(first)
        last_t = torch.as_tensor(last)
        above, below = torch.empty_like(first_t), torch.empty_like(first_t)
        up, down = (r - 1) % P, (r + 1) % P
        # tag 0: a first row travelling up; tag 1: a last row travelling down
        reqs = [dist.isend(first_t, up, group=self.group, tag=0),
                dist.isend(last_t, down, group=self.group, tag=1),
                dist.irecv(above, up, group=self.group, tag=1),
                dist.irecv(below, down, group=self.group, tag=0)]
        for q in reqs:
            q.wait()
        if isinstance(first, np.ndarray):
            return {r: (above.numpy(), below.numpy())}
        return {r: (above, below)}

    def merge(self, parts: Dict[int, tuple]) -> Obs:
        import torch
        import torch.distributed as dist

        (r, (sweep, B, M, Q, R, C)), = parts.items()
        dev = self.device
        head = torch.tensor([B, M, Q, sweep], dtype=torch.int64, device=dev)
        head_max = head[3:].clone()
        dist.all_reduce(head, group=self.group)
        dist.all_reduce(head_max, op=dist.ReduceOp.MAX, group=self.group)
        cols = torch.as_tensor(np.asarray(C, dtype=np.int64)).to(dev)
        dist.all_reduce(cols, group=self.group)
        width = max(self.rows)
        mine = torch.zeros(width, dtype=torch.int32, device=dev)
        mine[:len(R)] = torch.as_tensor(np.asarray(R, dtype=np.int32)).to(dev)
        gathered = [torch.empty_like(mine) for _ in range(self.world)]
        dist.all_gather(gathered, mine, group=self.group)
        if int(head_max[0]) * self.world != int(head[3]):
            raise RuntimeError("slabs at different sweeps")
        rows = np.concatenate([g[:n].cpu().numpy() for g, n in zip(gathered, self.rows)])
        return Obs(sweep, int(head[0]), int(head[1]), int(head[2]), rows.astype(np.int32),
                   cols.cpu().numpy().astype(np.int32))


class Decomposition:
    """Sweeps one lattice held as row slabs.  ``slabs``: {rank: engine} for
    the slabs of this process; ``exchange``: LocalExchange or DistExchange."""

    def __init__(self, slabs: Dict[int, object], exchange):
        self.slabs = dict(slabs)
        self.xc = exchange

    def _halos(self, colour: int):
        edges = {r: s.edges(colour) for r, s in self.slabs.items()}
        for r, (above, below) in self.xc.exchange(edges).items():
            self.slabs[r].set_halos(colour, above, below)

    def sweep(self, n: int, beta: Optional[float] = None, betas=None,
              record_every: int = 0) -> List[Obs]:
        """n sweeps at beta or betas[i]; the merged record after every
        record_every-th sweep (every process gets it)."""
        recs = []
        for i in range(n):
            b = float(betas[i] if betas is not None else beta)
            self._halos(1)
            for s in self.slabs.values():
                s.half_sweep(0, b)
            self._halos(0)
            for s in self.slabs.values():
                s.half_sweep(1, b)
            if record_every and (i + 1) % record_every == 0:
                recs.append(self.record())
        return recs

    def record(self) -> Obs:
        """Observables of the whole lattice.  After a sweep the colour-0
        halos are current but the colour-1 halos are one half-sweep old;
        they are refreshed first, so that an engine may read either."""
        self._halos(1)
        return self.xc.merge({r: s.measure() for r, s in self.slabs.items()})

    def get(self) -> Dict[int, np.ndarray]:
        """Owned rows of this process's slabs."""
        return {r: s.get() for r, s in self.slabs.items()}
