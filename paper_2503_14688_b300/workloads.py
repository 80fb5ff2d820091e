"""Seeded synthetic workloads: sizes, seeds, temperatures and schedules of the
paper's protocols, shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method itself (no random numbers of
the dynamics, no thresholds, no observables): only the parameters a run is
started with.  The paper's workloads are lattices generated by the method, so
there is no external dataset to stand in for.

Sources (arXiv 2503.14688): Table I (T_c of both models, t_max), Table II
(pre-cooling T1, t_switch, T2), Models section (T_c^Ising = 2/log(1+sqrt 2)).
"""
import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

ISING = 0
BLUME_CAPEL = 1

BASE_SEED = 0x2503146880000000
T_C_ISING = 2.26918531421302196814          # Table I
BETA_C_ISING = math.log(1 + math.sqrt(2)) / 2
T_C_BLUME_CAPEL = 1.69355839821214427017    # Table I (Delta = 0)
T_PARITY_BLUME_CAPEL = 1.6938               # the Blume-Capel parity workload's bath


@dataclass
class Workload:
    name: str
    model: int
    L: int
    sweeps: int
    seed: int
    beta: Optional[float] = None
    delta: float = 0.0
    hot_start: bool = True
    record_every: int = 1
    betas: Optional[List[float]] = field(default=None)

    def beta_of(self, i: int) -> float:
        return self.betas[i] if self.betas is not None else self.beta


def ising_quench_small() -> Workload:
    """Ising L=256, hot start, quench to beta_c, 100 sweeps, records every sweep."""
    return Workload("ising_L256_quench", ISING, 256, 100, BASE_SEED + 1, beta=BETA_C_ISING)


def blume_capel_parity() -> Workload:
    """Blume-Capel Delta=0, T=1.6938, L=1024, uniform {-1,0,1} start, 1000 sweeps."""
    return Workload("blume_capel_L1024_T1.6938", BLUME_CAPEL, 1024, 1000, BASE_SEED + 2,
                    beta=1.0 / T_PARITY_BLUME_CAPEL)


def ising_large() -> Workload:
    """Ising L=2^20 (2^40 spins, 128 GiB of bit-planes), hot-start quench to T_c."""
    return Workload("ising_L1048576_quench", ISING, 1 << 20, 1000, BASE_SEED + 4,
                    beta=BETA_C_ISING, record_every=10)


def blume_capel_large() -> Workload:
    """Blume-Capel Delta=0 L=2^19 (2^38 spins, 64 GiB), quench to T_c^BC."""
    return Workload("blume_capel_L524288_quench", BLUME_CAPEL, 1 << 19, 1000, BASE_SEED + 4,
                    beta=1.0 / T_C_BLUME_CAPEL, record_every=10)


def ensemble_sizes(n: int = 4096, seed: int = BASE_SEED + 3,
                   sizes=(64, 128, 256, 512, 1024)) -> np.ndarray:
    """Uneven mix of lattice sides for the replica ensemble (uniform over sizes)."""
    rng = np.random.default_rng(seed)
    return np.asarray(sizes, dtype=np.int64)[rng.integers(0, len(sizes), size=n)]


def precooling_schedule(model: int, t_switch: int, T1: Optional[float] = None,
                        T2: Optional[float] = None):
    """Two-temperature bath (Table II): T1 for t < t_switch, then T2.

    Returns (t_start, beta) for a piecewise-constant schedule.
    """
    if model == ISING:
        T1 = 1.66 if T1 is None else T1
        T2 = 2.27414861561203 if T2 is None else T2
    else:
        T1 = 1.24 if T1 is None else T1
        T2 = 1.69661396797728 if T2 is None else T2
    return [0, int(t_switch)], [1.0 / T1, 1.0 / T2]


def stepped_bath(T_c: float, n_sweeps: int, steps: int = 10, hi: float = 1.5, lo: float = 1.01):
    """T(t) in `steps` equal pieces, linear in T from hi*T_c down to lo*T_c."""
    edges = [int(round(k * n_sweeps / steps)) for k in range(steps)]
    temps = [T_c * (hi + (lo - hi) * k / (steps - 1)) for k in range(steps)]
    return edges, [1.0 / T for T in temps]


def served_requests(n: int, seed: int = BASE_SEED + 5, kmin: int = 8, kmax: int = 14,
                    sweeps_lo: int = 1000, sweeps_hi: int = 10000):
    """The served-stream workload: n requests, each Ising or Blume-Capel with
    probability 1/2, L = 2^k with k uniform in [kmin, kmax], a sweep count
    log-uniform in [sweeps_lo, sweeps_hi], seed BASE+5+i, and a bath stepping
    in 10 equal pieces, linear in T, from 1.5 T_c down to 1.01 T_c."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        model = int(rng.integers(0, 2))
        L = 1 << int(rng.integers(kmin, kmax + 1))
        sweeps = int(round(math.exp(rng.uniform(math.log(sweeps_lo), math.log(sweeps_hi)))))
        Tc = T_C_ISING if model == ISING else T_C_BLUME_CAPEL
        t_start, beta = stepped_bath(Tc, sweeps, steps=10)
        out.append({"model": model, "L": L, "sweeps": sweeps, "seed": seed + i,
                    "t_start": t_start, "beta": beta})
    return out


def poisson_arrivals(n: int, rate_per_s: float, seed: int = BASE_SEED + 55) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
