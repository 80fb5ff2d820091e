"""Direct quench to T_c at scaled size: the dynamic exponent z from xi(t)
and from E(t) ("Results", Eqs. (5)-(6)).

A hot-start lattice is put in a bath at T_c and left to relax; its
coherence length xi(t) = I2/I1 (Appendix C) grows as t^(1/z) and the Ising
energy excess E(t) - E_eq, E_eq = -sqrt 2, decays as t^(-1/z) (Eq. (4)).
The paper fits

    log t = z log xi + b + b' xi^(-omega)                              (Eq. (5))
    E(t) - E_eq = b t^(-1/z) + b' t^(-2/z) + b'' t^(-(omega+1)/z)      (Eq. (6))

with omega = 1.75, and finds z = 2.1676(1) for both models.

All lattice work runs in the library's kernels (hot start, sweeps, the axis
correlation sums, the on-device record of B); this module picks the check
times and does the host FP64 fits.

Readings (the paper leaves them open):
  * the errors of xi come from the jackknife over independent lattices; in
    Eq. (5) they enter as errors of log t through d(log t) = z d(log xi),
    with z from the previous iteration of the fit (two iterations);
  * E(t) is the energy per spin, -B / L^2, averaged over the same lattices;
    its error is their standard error.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import precooling as pc
from . import workloads as wl

OMEGA = 1.75      # leading correction-to-scaling exponent (Results)
Z_PAPER = 2.1676  # Eq. (7)


@dataclass
class QuenchData:
    t: np.ndarray        # sweeps
    xi: np.ndarray       # I2/I1 (NaN where Appendix C's distances are unresolved)
    xi_err: np.ndarray
    e: np.ndarray        # energy per spin, mean over lattices
    e_err: np.ndarray


def run(model: int, L: int, t_checks: Sequence[int], n_lattices: int = 4,
        seed: int = wl.BASE_SEED + 9500, delta: float = 0.0, r_max: Optional[int] = None,
        beta: Optional[float] = None) -> QuenchData:
    """Hot-start lattices quenched to T_c (the paper's, Table I; or `beta`),
    measured at the sweep counts t_checks: xi = I2/I1 by Appendix C with the
    lattices as jackknife samples, and the energy per spin."""
    from .lattice import Lattice

    if beta is None:
        beta = wl.BETA_C_ISING if model == wl.ISING else 1.0 / wl.T_C_BLUME_CAPEL
    r_max = L // 2 if r_max is None else int(r_max)
    lats = [Lattice(L, model, seed=seed + i, delta=delta) for i in range(n_lattices)]
    out = {k: [] for k in ("t", "xi", "xi_err", "e", "e_err")}
    try:
        for lat in lats:
            lat.init_random()
        done = 0
        for t in t_checks:
            t = int(t)
            es, S = [], []
            for lat in lats:
                lat.sweep(t - done, beta=beta)
                o = lat.measure()
                es.append((-o.B + delta * o.Q) / (float(L) * L))
                S.append(pc.axis_correlation(lat, r_max))
            done = t
            try:
                xi, err, _ = pc.coherence_length(np.stack(S))
            except ValueError:
                xi, err = math.nan, math.nan
            es = np.asarray(es)
            out["t"].append(t)
            out["xi"].append(xi)
            out["xi_err"].append(err)
            out["e"].append(es.mean())
            out["e_err"].append(es.std(ddof=1) / math.sqrt(es.size))
    finally:
        for lat in lats:
            lat.close()
    return QuenchData(*(np.asarray(out[k], dtype=np.float64) for k in ("t", "xi", "xi_err", "e",
                                                                        "e_err")))


@dataclass
class ZFit:
    z: float
    z_err: float
    coef: np.ndarray     # the linear coefficients (Eq. (5): b, b'; Eq. (6): b, b', b'')
    chi2: float
    dof: int


def fit_z_from_xi(t, xi, xi_err, t_min: float = 0.0, omega: float = OMEGA,
                  corrections: bool = True, iterations: int = 3) -> ZFit:
    """Weighted least squares of Eq. (5), log t = z log xi + b + b' xi^-omega
    (b' dropped with corrections=False), over t >= t_min.  The model is
    linear in (z, b, b'); the errors of log t are z * xi_err / xi with z from
    the previous iteration (starting at the paper's value)."""
    t = np.asarray(t, dtype=np.float64)
    xi = np.asarray(xi, dtype=np.float64)
    er = np.asarray(xi_err, dtype=np.float64)
    sel = np.isfinite(xi) & np.isfinite(er) & (er > 0) & (t >= t_min)
    t, xi, er = t[sel], xi[sel], er[sel]
    cols = [np.log(xi), np.ones_like(xi)] + ([xi ** -omega] if corrections else [])
    X = np.column_stack(cols)
    y = np.log(t)
    if y.size <= X.shape[1]:
        raise ValueError("not enough points for the fit")
    z = Z_PAPER
    for _ in range(iterations):
        s = z * er / xi
        coef, *_ = np.linalg.lstsq(X / s[:, None], y / s, rcond=None)
        z = float(coef[0])
    s = z * er / xi
    r = (y - X @ coef) / s
    cov = np.linalg.inv((X / s[:, None]).T @ (X / s[:, None]))
    return ZFit(z=z, z_err=float(math.sqrt(cov[0, 0])), coef=coef[1:].copy(), chi2=float(r @ r),
                dof=int(y.size - X.shape[1]))


def _energy_design(t, z, omega):
    return np.column_stack([t ** (-1.0 / z), t ** (-2.0 / z), t ** (-(omega + 1.0) / z)])


def fit_z_from_energy(t, e, e_err, e_eq: float = -math.sqrt(2.0), t_min: float = 0.0,
                      omega: float = OMEGA, z_bounds=(1.5, 3.5)) -> ZFit:
    """Weighted least squares of Eq. (6), E(t) - E_eq = b t^(-1/z) +
    b' t^(-2/z) + b'' t^(-(omega+1)/z), over t >= t_min: linear in the
    amplitudes for fixed z, z by a bounded scalar search of chi^2; its error
    from the curvature of the profiled chi^2 (delta chi^2 = 1)."""
    from scipy.optimize import minimize_scalar

    t = np.asarray(t, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    s = np.asarray(e_err, dtype=np.float64)
    sel = np.isfinite(e) & (s > 0) & (t >= t_min)
    t, e, s = t[sel], e[sel], s[sel]
    y = e - e_eq
    if y.size <= 4:
        raise ValueError("not enough points for the fit")

    def chi2(z):
        X = _energy_design(t, z, omega) / s[:, None]
        coef, *_ = np.linalg.lstsq(X, y / s, rcond=None)
        r = y / s - X @ coef
        return float(r @ r), coef

    grid = np.linspace(z_bounds[0], z_bounds[1], 201)
    k = int(np.argmin([chi2(g)[0] for g in grid]))
    lo, hi = grid[max(k - 1, 0)], grid[min(k + 1, grid.size - 1)]
    opt = minimize_scalar(lambda g: chi2(g)[0], bounds=(lo, hi), method="bounded",
                          options={"xatol": 1e-10})
    z = float(opt.x)
    c0, coef = chi2(z)
    h = 1e-3
    curv = (chi2(z + h)[0] - 2 * c0 + chi2(z - h)[0]) / (h * h)
    z_err = math.sqrt(2.0 / curv) if curv > 0 else math.inf
    return ZFit(z=z, z_err=z_err, coef=coef, chi2=c0, dof=int(y.size - 4))
