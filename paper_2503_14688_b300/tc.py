"""Critical temperature of the Blume-Capel model at scaled size (Appendix B).

Equilibrium configurations come from the elementary Monte Carlo step of
Appendix B (10 Metropolis sweeps + one Swendsen-Wang iteration of the +-1
spins) at one inverse temperature beta0 near the critical point.  Histogram
reweighting extends the averages to neighbouring beta (for Delta = 0 the
weight of a configuration changes by exp((beta - beta0) B), B the bond sum).
For each L the inverse temperatures beta_{L,U} and beta_{L,xi} where

    U4 = <M^4> / <M^2>^2 = 1.1679229   and   xi_2 / L = 0.9050488292

(the universal values of Appendix B) are located; they tend to beta_c
(Eq. (11)), and the paper finds them compatible with a constant from
L >= 64 on.

Every lattice operation runs in the library's kernels; this module does the
host FP64 reweighting, root finding and jackknife.

Readings (the paper leaves them open): the records are the observables after
each EMCS (every `every` steps); the jackknife blocks are the independent
lattices; chi(k_min) averages the two axis directions as in isg_xi2; the
constant fit over L >= L_min is a weighted mean of beta_{L,U} and
beta_{L,xi} together.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Sequence

import numpy as np

from . import workloads as wl

U4_STAR = 1.1679229
XI_STAR = 0.9050488292


@dataclass
class Samples:
    L: int
    beta0: float
    B: np.ndarray    # (lattices, measurements) bond sums
    M: np.ndarray    # magnetisation
    Sk: np.ndarray   # |M(k_min)|^2 averaged over the two axes


def _sk(R: np.ndarray, C: np.ndarray) -> float:
    L = R.size
    ph = np.exp(2j * np.pi * np.arange(L) / L)
    return 0.5 * (abs(np.dot(C, ph)) ** 2 + abs(np.dot(R, ph)) ** 2)


def sample(L: int, beta0: float, n_lattices: int, therm: int, meas: int, every: int = 1,
           sweeps: int = 10, seed: int = wl.BASE_SEED + 9900, delta: float = 0.0) -> Samples:
    """Equilibrium samples of the Blume-Capel model: n_lattices hot starts,
    `therm` EMCS to equilibrate, then `meas` EMCS recording every `every`."""
    from .lattice import Lattice

    n_rec = meas // every
    B = np.empty((n_lattices, n_rec))
    M = np.empty((n_lattices, n_rec))
    Sk = np.empty((n_lattices, n_rec))
    for i in range(n_lattices):
        lat = Lattice(L, wl.BLUME_CAPEL, seed=seed + i, delta=delta, record_capacity=n_rec + 1)
        try:
            lat.init_random()
            lat.emcs(therm, beta0, sweeps=sweeps)
            lat.emcs(meas, beta0, sweeps=sweeps, record_every=every)
            recs = lat.read_records()
        finally:
            lat.close()
        for j, o in enumerate(recs[:n_rec]):
            B[i, j], M[i, j] = o.B, o.M
            Sk[i, j] = _sk(o.R.astype(np.float64), o.C.astype(np.float64))
    return Samples(L, beta0, B, M, Sk)


def observables(s: Samples, beta: float, keep=None):
    """(U4, xi_2/L) at beta by reweighting the samples of beta0 (Delta = 0:
    weight exp((beta - beta0) B)); `keep` selects lattices (jackknife)."""
    B = s.B if keep is None else s.B[keep]
    M = s.M if keep is None else s.M[keep]
    Sk = s.Sk if keep is None else s.Sk[keep]
    a = (beta - s.beta0) * B.reshape(-1)
    w = np.exp(a - a.max())
    w /= w.sum()
    m = M.reshape(-1)
    m2, m4 = float(w @ m ** 2), float(w @ m ** 4)
    sk = float(w @ Sk.reshape(-1))
    u4 = m4 / (m2 * m2)
    ratio = m2 / sk - 1.0
    xi = math.sqrt(ratio) / (2.0 * math.sin(math.pi / s.L)) if ratio > 0 else math.nan
    return u4, xi / s.L


def default_span(L: int) -> float:
    """Reweighting range around beta0: the energy histogram's width shrinks
    as 1/L in beta (L^2 sites, fluctuations ~ L), so 1.5/L keeps the
    reweighted averages dominated by many samples."""
    return 1.5 / L


def crossing(s: Samples, which: str, span=None, keep=None, target=None) -> float:
    """The beta in [beta0 - span, beta0 + span] where U4 (which = "u4") or
    xi_2/L (which = "xi") takes `target` (default: its universal value), by
    Brent's method on the reweighted curve."""
    from scipy.optimize import brentq

    k = 0 if which == "u4" else 1
    if target is None:
        target = U4_STAR if which == "u4" else XI_STAR
    span = default_span(s.L) if span is None else span

    def f(b):
        return observables(s, b, keep)[k] - target

    lo, hi = s.beta0 - span, s.beta0 + span
    if f(lo) * f(hi) > 0:
        raise ValueError(f"{which} does not cross its universal value within +-{span}")
    return float(brentq(f, lo, hi, xtol=1e-12))


def crossing_with_error(s: Samples, which: str, span=None):
    """The crossing and its jackknife error over the lattices."""
    n = s.B.shape[0]
    full = crossing(s, which, span)
    jk = []
    for i in range(n):
        keep = np.ones(n, bool)
        keep[i] = False
        jk.append(crossing(s, which, span, keep))
    jk = np.asarray(jk)
    return full, math.sqrt((n - 1) * np.mean((jk - jk.mean()) ** 2))


def constant_fit(values: Sequence[float], errors: Sequence[float]):
    """Weighted mean, its error and chi^2/dof (the paper fits the crossings
    for L >= 64 to a constant)."""
    v = np.asarray(values, dtype=np.float64)
    e = np.asarray(errors, dtype=np.float64)
    w = 1.0 / e ** 2
    mean = float((w * v).sum() / w.sum())
    err = float(1.0 / math.sqrt(w.sum()))
    chi2 = float((w * (v - mean) ** 2).sum())
    return mean, err, chi2 / max(v.size - 1, 1)
