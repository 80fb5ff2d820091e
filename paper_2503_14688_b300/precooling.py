"""Pre-cooling protocol at scaled size ("Thermal protocols", Eq. (8), Table II).

The paper's second thermal protocol starts from a hot-start lattice.  The
lattice relaxes in a bath at T1 ~ 0.73 T_c until its coherence length
xi(t, T1) reaches a fraction f of xi_eq(T2), the equilibrium coherence length
at the final temperature T2 (just above T_c).  At that moment the bath jumps
to T2.  The late approach of the energy to equilibrium follows

    E(t; f) = E_eq + b(f) exp(-t / tau)                               (Eq. (8))

with tau independent of f.  The paper fits all f jointly and finds the
amplitude b(f) change sign at f = 0.59(5), where the approach is
exponentially faster, for both models at xi_eq(T2) ~ 400.

Every lattice operation here runs in the library's kernels: hot starts,
sweeps, on-device records of B and Q, and the axis correlation sums behind
C(r).  This module chooses sweep counts and does the host FP64 analysis: the
coherence length xi = I2/I1 of Appendix C, the joint fit of Eq. (8), and the
zero of b(f).

Readings (the paper fixes neither):
  * t counts sweeps from the hot start (the origin of the protocol).
    Measuring t from the switch instead rescales b(f) by exp(t_switch/tau) > 0,
    so the sign of b(f) and its zero do not change.
  * The energy is the energy per spin e = (-B + Delta Q) / L^2.  Eq. (3)'s
    nearest-neighbour sum has the opposite sign for Ising; the fit and b's
    zero are insensitive to the overall sign.
  * C(r) is sampled at every integer r up to r_max, so the integrals of
    Eq. (12) use the trapezoid rule on the integer grid.  The paper's cubic
    spline is only needed for sparse r.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import workloads as wl

T1_OVER_TC = 0.73   # "Thermal protocols": T1 ~ 0.73 T_c


# ---------------------------------------------------------------------------
# Equilibrium energy of the infinite Ising lattice (E_eq of Eq. (8))
# ---------------------------------------------------------------------------
def onsager_energy(beta: float) -> float:
    """Energy per spin of the infinite square-lattice Ising model, J = 1
    (Onsager 1944): u = -coth(2b) [1 + (2/pi)(2 tanh^2(2b) - 1) K(k)],
    k = 2 sinh(2b) / cosh^2(2b), K the complete elliptic integral of the
    first kind.  At beta_c (k = 1) the product tends to zero and u = -sqrt 2
    (the Results' E_eq(T_c))."""
    from scipy.special import ellipk

    b2 = 2.0 * beta
    k = 2.0 * math.sinh(b2) / math.cosh(b2) ** 2
    a = 2.0 * math.tanh(b2) ** 2 - 1.0
    if abs(1.0 - k) < 1e-15:
        return -math.sqrt(2.0)
    return -(1.0 / math.tanh(b2)) * (1.0 + (2.0 / math.pi) * a * float(ellipk(k * k)))


# ---------------------------------------------------------------------------
# Coherence length xi = I2 / I1 (Appendix C, Eq. (12), Eq. (13))
# ---------------------------------------------------------------------------
def axis_correlation(lat, r_max: int) -> np.ndarray:
    """C(r), r = 0..r_max, of one lattice: the mean of C((r,0)) and C((0,r))
    (Eq. (2) along the axes), from the exact sums of isg_correlation."""
    r = np.arange(r_max + 1)
    sx, sy = lat.correlation(r)
    L = float(lat.L)
    return (sx.astype(np.float64) + sy.astype(np.float64)) / (2.0 * L * L)


def _trapezoid(y: np.ndarray, x: np.ndarray) -> float:
    return float(np.sum(0.5 * (y[1:] + y[:-1]) * (x[1:] - x[:-1])))


def _f_tail(r, A, xi_F, beta_F):
    # Eq. (13): F(r) = A exp[-(r / xi_F)^beta] / sqrt(r)
    return A * np.exp(-np.power(r / xi_F, beta_F)) / np.sqrt(r)


@dataclass
class XiResult:
    xi: float
    r_cut: int
    r_star: int
    r_min: int
    r_max: int
    tail_fit: bool
    I1: float
    I2: float


def xi_cutoffs(C: np.ndarray, C_err: np.ndarray):
    """Steps (i)-(ii) of Appendix C on a mean curve C(r), r = 0..len-1:
      (i)  r_cut: the first r with C(r + 1) < 3 err(r + 1);
      (ii) r*: the maximum of r^2 C(r) below r_cut; r_min, r_max: the first
           r > r* where r^2 C drops below 0.9 and below 1/3 of that maximum.
    Returns (r_cut, r_star, r_min, r_max).  Raises ValueError where the paper
    would ask for more statistics (r* < r_min < r_max < r_cut not met)."""
    C = np.asarray(C, dtype=np.float64)
    C_err = np.asarray(C_err, dtype=np.float64)
    r = np.arange(C.size, dtype=np.float64)
    below = np.nonzero(C[1:] < 3.0 * C_err[1:])[0]
    if below.size == 0:
        raise ValueError("C(r) stays above three errors up to the last distance")
    r_cut = int(below[0])  # C(r_cut + 1) < 3 err
    w = r[: r_cut + 1] ** 2 * C[: r_cut + 1]
    r_star = int(np.argmax(w))
    peak = w[r_star]
    after = np.arange(r_star + 1, r_cut + 1)
    mins = after[w[after] < 0.9 * peak]
    maxs = after[w[after] < peak / 3.0]
    if mins.size == 0 or maxs.size == 0:
        raise ValueError("r_min or r_max not found below r_cut")
    r_min, r_max = int(mins[0]), int(maxs[0])
    if not (r_star < r_min < r_max < r_cut):
        raise ValueError("Appendix C condition r* < r_min < r_max < r_cut not met")
    return r_cut, r_star, r_min, r_max


def xi_integrate(C: np.ndarray, C_err: np.ndarray, cuts) -> XiResult:
    """Step (iii) of Appendix C with the distances `cuts` of xi_cutoffs:
    r_max - r_min <= 8: I1, I2 (Eq. (12)) by the trapezoid rule up to r_cut;
    otherwise fit Eq. (13) to C on [r_min, r_max] (weights 1/err^2),
    integrate the data up to r_max and F(r) from r_max to 20 xi_F."""
    r_cut, r_star, r_min, r_max = cuts
    C = np.asarray(C, dtype=np.float64)
    C_err = np.asarray(C_err, dtype=np.float64)
    r = np.arange(C.size, dtype=np.float64)
    if r_max - r_min <= 8:
        rr, cc = r[: r_cut + 1], C[: r_cut + 1]
        I1, I2 = _trapezoid(rr * cc, rr), _trapezoid(rr * rr * cc, rr)
        return XiResult(I2 / I1, r_cut, r_star, r_min, r_max, False, I1, I2)
    from scipy.integrate import quad
    from scipy.optimize import curve_fit

    rf = r[r_min: r_max + 1]
    cf = C[r_min: r_max + 1]
    sf = np.maximum(C_err[r_min: r_max + 1], 1e-300)
    # start: a pure exponential through the two ends of the window
    lo, hi = max(cf[0] * math.sqrt(rf[0]), 1e-300), max(cf[-1] * math.sqrt(rf[-1]), 1e-300)
    xi0 = (rf[-1] - rf[0]) / max(math.log(lo / hi), 1e-3)
    p0 = (lo * math.exp(rf[0] / xi0), xi0, 1.0)
    (A, xi_F, beta_F), _ = curve_fit(_f_tail, rf, cf, p0=p0, sigma=sf, absolute_sigma=True,
                                     bounds=([0.0, 1e-3, 0.05], [np.inf, 1e7, 10.0]),
                                     maxfev=20000)
    rr, cc = r[: r_max + 1], C[: r_max + 1]
    I1, I2 = _trapezoid(rr * cc, rr), _trapezoid(rr * rr * cc, rr)
    top = 20.0 * xi_F
    if top > r_max:
        I1 += quad(lambda x: x * _f_tail(x, A, xi_F, beta_F), r_max, top, limit=400)[0]
        I2 += quad(lambda x: x * x * _f_tail(x, A, xi_F, beta_F), r_max, top, limit=400)[0]
    return XiResult(I2 / I1, r_cut, r_star, r_min, r_max, True, I1, I2)


def xi_from_curve(C: np.ndarray, C_err: np.ndarray) -> XiResult:
    """xi = I2/I1 of one mean correlation curve with its errors (Appendix C)."""
    return xi_integrate(C, C_err, xi_cutoffs(C, C_err))


def coherence_length(samples: np.ndarray):
    """xi = I2/I1 and its jackknife error from n independent samples of C(r)
    (rows: lattices or independent runs; Appendix C: jackknife on the
    measured correlation functions).  Returns (xi, xi_err, XiResult of the
    mean curve)."""
    S = np.asarray(samples, dtype=np.float64)
    n = S.shape[0]
    if n < 2:
        raise ValueError("need at least two independent samples for the errors")
    mean = S.mean(axis=0)
    err = S.std(axis=0, ddof=1) / math.sqrt(n)
    cuts = xi_cutoffs(mean, err)
    full = xi_integrate(mean, err, cuts)
    # jackknife with the distances of the full sample held fixed
    jk = []
    for k in range(n):
        keep = np.ones(n, dtype=bool)
        keep[k] = False
        Sk = S[keep]
        jk.append(xi_integrate(Sk.mean(axis=0), Sk.std(axis=0, ddof=1) / math.sqrt(n - 1), cuts).xi)
    jk = np.asarray(jk)
    xi_err = math.sqrt((n - 1) * np.mean((jk - jk.mean()) ** 2))
    return full.xi, xi_err, full


# ---------------------------------------------------------------------------
# Coherence length on the GPU: growth at T1, equilibrium at T2
# ---------------------------------------------------------------------------
def _lattices(model: int, L: int, n: int, seed: int, delta: float):
    from .lattice import Lattice

    lats = [Lattice(L, model, seed=seed + i, delta=delta, record_capacity=1) for i in range(n)]
    for lat in lats:
        lat.init_random()
    return lats


def xi_growth(model: int, L: int, T: float, t_checks: Sequence[int], n_lattices: int = 8,
              seed: int = wl.BASE_SEED + 7000, delta: float = 0.0, r_max: Optional[int] = None,
              stop_at: float = math.inf):
    """xi(t) = I2/I1 of hot-start lattices in a bath at T, at the sweep counts
    t_checks (increasing).  Independent lattices (seeds seed + i) are the
    samples of the jackknife.  Returns (t, xi, xi_err) arrays; NaN where the
    Appendix C distances are not resolved (xi of order one lattice spacing).
    Stops after the first check with xi >= stop_at."""
    r_max = L // 2 if r_max is None else int(r_max)
    lats = _lattices(model, L, n_lattices, seed, delta)
    out_t, out_xi, out_err = [], [], []
    try:
        done = 0
        for t in t_checks:
            t = int(t)
            for lat in lats:
                lat.sweep(t - done, beta=1.0 / T)
            done = t
            S = np.stack([axis_correlation(lat, r_max) for lat in lats])
            try:
                xi, err, _ = coherence_length(S)
            except ValueError:  # Appendix C distances not resolved (xi ~ 1)
                xi, err = math.nan, math.nan
            out_t.append(t)
            out_xi.append(xi)
            out_err.append(err)
            if xi >= stop_at:
                break
    finally:
        for lat in lats:
            lat.close()
    return np.asarray(out_t), np.asarray(out_xi), np.asarray(out_err)


def equilibrium_xi(model: int, L: int, T: float, t_therm: int, n_meas: int, gap: int,
                   n_lattices: int = 8, seed: int = wl.BASE_SEED + 8000, delta: float = 0.0,
                   r_max: Optional[int] = None):
    """xi_eq(T) = I2/I1 in equilibrium: hot-start lattices thermalised for
    t_therm sweeps at T, then C(r) averaged over n_meas measurements `gap`
    sweeps apart; each lattice's time average is one jackknife sample.
    Returns (xi, xi_err, XiResult)."""
    r_max = L // 2 if r_max is None else int(r_max)
    lats = _lattices(model, L, n_lattices, seed, delta)
    try:
        for lat in lats:
            lat.sweep(t_therm, beta=1.0 / T)
        acc = np.zeros((n_lattices, r_max + 1))
        for _ in range(n_meas):
            for i, lat in enumerate(lats):
                lat.sweep(gap, beta=1.0 / T)
                acc[i] += axis_correlation(lat, r_max)
    finally:
        for lat in lats:
            lat.close()
    return coherence_length(acc / n_meas)


def switch_time(t: np.ndarray, xi: np.ndarray, target: float) -> int:
    """The first sweep count at which xi(t) reaches `target`, by linear
    interpolation of log xi against log t between the checked times
    (xi grows as a power of t in the ordered phase); rounded up."""
    t = np.asarray(t, dtype=np.float64)
    xi = np.asarray(xi, dtype=np.float64)
    ok = np.isfinite(xi)
    t, xi = t[ok], xi[ok]
    if xi.size == 0:
        raise ValueError("no resolved xi")
    if target <= xi[0]:
        return int(t[0])
    k = int(np.argmax(xi >= target))
    if xi[k] < target:
        raise ValueError("xi never reaches the target within the checked times")
    lt0, lt1 = math.log(t[k - 1]), math.log(t[k])
    lx0, lx1 = math.log(xi[k - 1]), math.log(xi[k])
    lt = lt0 + (math.log(target) - lx0) * (lt1 - lt0) / (lx1 - lx0)
    return int(math.ceil(math.exp(lt) - 1e-9))


# ---------------------------------------------------------------------------
# The protocol on a replica ensemble: E(t; f)
# ---------------------------------------------------------------------------
def energy_relaxation(model: int, L: int, T1: float, T2: float, t_switch: int, t_total: int,
                      record_every: int, n_replicas: int, seed: int, delta: float = 0.0,
                      chunk: int = 4096, raw: bool = False):
    """Run the two-temperature protocol on n_replicas hot-start replicas of
    side L in one persistent ensemble: t_switch sweeps at T1, then T2 up to
    t_total sweeps, recording B and Q every `record_every` sweeps of the T2
    stage (record sweeps t_switch + k record_every).  Replica r has seed
    seed + r.  Returns (t, E_mean, E_err) with E the energy per spin averaged
    over replicas and its standard error; with raw=True also the recorded
    B and Q as (records x replicas) int64 arrays."""
    from .ensemble import Ensemble

    if not (0 <= t_switch < t_total) or record_every <= 0:
        raise ValueError("need 0 <= t_switch < t_total and record_every > 0")
    per_call = max(record_every, (chunk // record_every) * record_every)
    ens = Ensemble([L] * n_replicas, [seed + r for r in range(n_replicas)],
                   models=[model] * n_replicas, delta=delta,
                   record_capacity=per_call // record_every + 1)
    ts, means, errs, Bs, Qs = [], [], [], [], []
    try:
        ens.init_random()
        if t_switch:
            ens.sweep(t_switch, beta=1.0 / T1)
        done = t_switch
        while done < t_total:
            n = min(per_call, t_total - done)
            n -= n % record_every
            if n == 0:
                ens.sweep(t_total - done, beta=1.0 / T2)
                break
            ens.sweep(n, beta=1.0 / T2, record_every=record_every)
            sw, B, _, Q = ens.read_scalars()
            if raw:
                Bs.append(B)
                Qs.append(Q)
            e = (-B.astype(np.float64) + delta * Q.astype(np.float64)) / (float(L) * float(L))
            ts.extend(sw.tolist())
            means.extend(e.mean(axis=1).tolist())
            errs.extend((e.std(axis=1, ddof=1) / math.sqrt(n_replicas)).tolist())
            done += n
    finally:
        ens.close()
    if raw:
        return (np.asarray(ts), np.asarray(means), np.asarray(errs),
                np.concatenate(Bs), np.concatenate(Qs))
    return np.asarray(ts), np.asarray(means), np.asarray(errs)


# ---------------------------------------------------------------------------
# Joint fit of Eq. (8) and the zero of b(f)
# ---------------------------------------------------------------------------
@dataclass
class ApproachFit:
    tau: float
    tau_err: float
    b: np.ndarray          # one amplitude per protocol (per f)
    b_err: np.ndarray
    E_eq: float
    E_eq_err: float
    chi2: float
    dof: int


def _design(ts, tau, free_eq):
    """Rows: every retained time of every protocol; columns: exp(-t/tau)
    in protocol i's own column, then 1 for E_eq when it is free."""
    n_f = len(ts)
    blocks = []
    for i, t in enumerate(ts):
        X = np.zeros((t.size, n_f + (1 if free_eq else 0)))
        X[:, i] = np.exp(-t / tau)
        if free_eq:
            X[:, n_f] = 1.0
        blocks.append(X)
    return np.vstack(blocks)


def fit_approach(ts: Sequence[np.ndarray], Es: Sequence[np.ndarray], errs: Sequence[np.ndarray],
                 E_eq: Optional[float] = None, t_min: float = 0.0, t_max: float = math.inf,
                 tau_bounds=(1.0, 1e7)) -> ApproachFit:
    """Joint weighted least-squares fit of Eq. (8) to several protocols:
    E_i(t) = E_eq + b_i exp(-t / tau) for t_min <= t <= t_max, one tau for
    all.
    E_eq is fixed when given (Ising: Onsager) and an f-independent free
    parameter otherwise (Blume-Capel).  For fixed tau the model is linear in
    the b_i (and E_eq), solved exactly; tau minimises chi^2 (bounded scalar
    search on log tau).  Errors: the inverse of the chi^2 curvature matrix
    (J^T W J) at the minimum, tau included."""
    from scipy.optimize import minimize_scalar

    sel = [(np.asarray(t, dtype=np.float64) >= t_min) & (np.asarray(t, dtype=np.float64) <= t_max)
           for t in ts]
    T = [np.asarray(t, dtype=np.float64)[s] for t, s in zip(ts, sel)]
    Y = np.concatenate([np.asarray(e, dtype=np.float64)[s] for e, s in zip(Es, sel)])
    S = np.concatenate([np.asarray(e, dtype=np.float64)[s] for e, s in zip(errs, sel)])
    if np.any(S <= 0):
        raise ValueError("errors must be positive")
    free_eq = E_eq is None
    y = Y if free_eq else Y - E_eq
    w = 1.0 / S

    def solve(log_tau):
        X = _design(T, math.exp(log_tau), free_eq)
        p, *_ = np.linalg.lstsq(X * w[:, None], y * w, rcond=None)
        res = (y - X @ p) * w
        return float(res @ res), p

    lo, hi = math.log(tau_bounds[0]), math.log(tau_bounds[1])
    grid = np.linspace(lo, hi, 121)
    chis = [solve(g)[0] for g in grid]
    k = int(np.argmin(chis))
    a, b = grid[max(k - 1, 0)], grid[min(k + 1, grid.size - 1)]
    opt = minimize_scalar(lambda g: solve(g)[0], bounds=(a, b), method="bounded",
                          options={"xatol": 1e-10})
    log_tau = float(opt.x)
    chi2, p = solve(log_tau)
    tau = math.exp(log_tau)
    n_f = len(T)
    # curvature: d model / d(b_i, [E_eq], tau)
    X = _design(T, tau, free_eq)
    tt = np.concatenate(T)
    dtau = np.zeros_like(tt)
    off = 0
    for i, t in enumerate(T):
        dtau[off: off + t.size] = p[i] * np.exp(-t / tau) * t / tau ** 2
        off += t.size
    J = np.column_stack([X, dtau]) * w[:, None]
    cov = np.linalg.pinv(J.T @ J)
    err = np.sqrt(np.maximum(np.diag(cov), 0.0))
    dof = int(y.size - (n_f + (1 if free_eq else 0) + 1))
    return ApproachFit(tau=tau, tau_err=float(err[-1]), b=p[:n_f].copy(), b_err=err[:n_f].copy(),
                       E_eq=float(p[n_f]) if free_eq else float(E_eq),
                       E_eq_err=float(err[n_f]) if free_eq else 0.0, chi2=chi2, dof=dof)


def choose_window(ts, Es, errs, E_eq: Optional[float], t_mins: Sequence[float], span: float,
                  max_chi2_per_dof: float = 1.5):
    """The late-time window of Eq. (8): the earliest t_min of `t_mins` whose
    joint fit on [t_min, t_min + span] has chi^2/dof <= max_chi2_per_dof
    (faster modes still present give a poor single-exponential fit).
    Returns (t_min, t_max, ApproachFit); the last candidate if none passes."""
    fit = None
    for t_min in t_mins:
        fit = fit_approach(ts, Es, errs, E_eq=E_eq, t_min=t_min, t_max=t_min + span)
        if fit.dof > 0 and fit.chi2 / fit.dof <= max_chi2_per_dof:
            return float(t_min), float(t_min + span), fit
    return float(t_mins[-1]), float(t_mins[-1] + span), fit


def zero_crossing(f: Sequence[float], b: Sequence[float], b_err: Sequence[float]):
    """The f at which b(f) = 0, by linear interpolation between the two
    adjacent f (in increasing order) where b changes sign; the error is
    propagated from the two amplitudes' errors (taken independent).
    Returns (f_star, f_star_err); raises ValueError without a sign change."""
    f = np.asarray(f, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = np.asarray(b_err, dtype=np.float64)
    order = np.argsort(f)
    f, b, s = f[order], b[order], s[order]
    for k in range(f.size - 1):
        if b[k] == 0.0:
            return float(f[k]), float(s[k] * (f[k + 1] - f[k]) / abs(b[k + 1] - b[k]))
        if b[k] * b[k + 1] < 0.0:
            f0, f1, b0, b1 = f[k], f[k + 1], b[k], b[k + 1]
            fs = f0 + (f1 - f0) * b0 / (b0 - b1)
            # d f*/d b0 = (f1 - f0) (-b1) / (b0 - b1)^2, d f*/d b1 = (f1 - f0) b0 / (b0 - b1)^2
            d = (f1 - f0) / (b0 - b1) ** 2
            err = math.sqrt((d * b1 * s[k]) ** 2 + (d * b0 * s[k + 1]) ** 2)
            return float(fs), float(err)
    raise ValueError("b(f) does not change sign")


# ---------------------------------------------------------------------------
# The whole scan
# ---------------------------------------------------------------------------
def scan(model: int, fs: Sequence[float], T2_over_Tc: float = 1.04, L: int = 512,
         n_replicas: int = 4096, L_xi: int = 1024, n_xi: int = 16, t_after: int = 1000,
         record_every: int = 10, t_mins: Sequence[float] = (100, 150, 200, 250, 300, 400, 500),
         span: float = 600.0, seed: int = wl.BASE_SEED + 9000, delta: float = 0.0) -> dict:
    """The pre-cooling experiment at scaled size for one model:
      1. xi_eq(T2) from n_xi lattices of side L_xi in equilibrium at T2;
      2. xi(t) at T1 = 0.73 T_c from hot starts (n_xi lattices of side L_xi),
         and the switch time t_f at which xi(t_f) = f xi_eq(T2), per f;
      3. per f, the protocol on n_replicas replicas of side L: t_f sweeps at
         T1, then t_after sweeps at T2, energy recorded every record_every;
      4. the joint fit of Eq. (8) on the earliest window [t_min, t_min + span]
         (t_min from t_mins) with chi^2/dof <= 1.5 (E_eq: Onsager for Ising,
         free for Blume-Capel), and the zero f* of b(f).
    T_c is the paper's (Table I).  Returns a dict of every intermediate
    result plus the ensemble throughput of step 3 (flips/ns, host time)."""
    import time

    Tc = wl.T_C_ISING if model == wl.ISING else wl.T_C_BLUME_CAPEL
    T1, T2 = T1_OVER_TC * Tc, T2_over_Tc * Tc
    fs = [float(f) for f in fs]
    xi_eq, xi_eq_err, xr = equilibrium_xi(model, L_xi, T2, t_therm=4000, n_meas=100, gap=100,
                                          n_lattices=n_xi, seed=seed + 100, delta=delta)
    checks = sorted(set(int(round(2 ** (k / 4))) for k in range(4, 49)))
    t_g, xi_g, err_g = xi_growth(model, L_xi, T1, checks, n_lattices=n_xi, seed=seed + 200,
                                 delta=delta, stop_at=max(fs) * xi_eq)
    t_sw = [0 if f == 0.0 else switch_time(t_g, xi_g, f * xi_eq) for f in fs]
    runs, flips, secs = [], 0.0, 0.0
    for i, (f, ts) in enumerate(zip(fs, t_sw)):
        t0 = time.perf_counter()
        t, E, Ee = energy_relaxation(model, L, T1, T2, ts, ts + t_after, record_every, n_replicas,
                                     seed + 1000 + 100000 * i, delta=delta)
        secs += time.perf_counter() - t0
        flips += float(n_replicas) * L * L * (ts + t_after)
        runs.append((t, E, Ee))
    E_eq = onsager_energy(1.0 / T2) if model == wl.ISING else None
    t_min, t_max, fit = choose_window([r[0] for r in runs], [r[1] for r in runs],
                                      [r[2] for r in runs], E_eq, t_mins, span)
    nz = [k for k, f in enumerate(fs) if f > 0.0]
    f_star, f_star_err = zero_crossing([fs[k] for k in nz], fit.b[nz], fit.b_err[nz])
    return {
        "model": "ising" if model == wl.ISING else "blume_capel", "T1": T1, "T2": T2,
        "L": L, "n_replicas": n_replicas, "xi_eq": xi_eq, "xi_eq_err": xi_eq_err,
        "xi_eq_cuts": [xr.r_cut, xr.r_star, xr.r_min, xr.r_max, xr.tail_fit],
        "growth": {"t": t_g.tolist(), "xi": xi_g.tolist(), "xi_err": err_g.tolist()},
        "f": fs, "t_switch": t_sw,
        "fit": {"t_min": t_min, "t_max": t_max, "tau": fit.tau, "tau_err": fit.tau_err,
                "b": fit.b.tolist(), "b_err": fit.b_err.tolist(), "E_eq": fit.E_eq,
                "E_eq_err": fit.E_eq_err, "chi2_per_dof": fit.chi2 / max(fit.dof, 1)},
        "f_star": f_star, "f_star_err": f_star_err,
        "runs": {"t": [r[0].tolist() for r in runs], "E": [r[1].tolist() for r in runs],
                 "E_err": [r[2].tolist() for r in runs]},
        "ensemble_flips_per_ns": flips / secs / 1e9, "ensemble_seconds": secs,
    }


def main(argv=None):
    """python -m paper_2503_14688_b300.precooling [--model ising|blume_capel]
    [--f 0,0.3,...] [--replicas N] [--L L] [--json out.json]: run `scan` and
    print f*, tau and b(f)."""
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--model", default="ising", choices=["ising", "blume_capel"])
    ap.add_argument("--f", default="0,0.3,0.4,0.5,0.6,0.7,0.8")
    ap.add_argument("--T2-over-Tc", type=float, default=1.04)
    ap.add_argument("--L", type=int, default=512)
    ap.add_argument("--replicas", type=int, default=4096)
    ap.add_argument("--t-after", type=int, default=1000)
    ap.add_argument("--span", type=float, default=600.0)
    ap.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    model = wl.ISING if a.model == "ising" else wl.BLUME_CAPEL
    res = scan(model, [float(x) for x in a.f.split(",")], T2_over_Tc=a.T2_over_Tc, L=a.L,
               n_replicas=a.replicas, t_after=a.t_after, span=a.span)
    print(f"{res['model']}: xi_eq(T2) = {res['xi_eq']:.2f}({res['xi_eq_err']:.2f}), "
          f"tau = {res['fit']['tau']:.1f}({res['fit']['tau_err']:.1f}), "
          f"f* = {res['f_star']:.3f}({res['f_star_err']:.3f}), "
          f"chi2/dof = {res['fit']['chi2_per_dof']:.2f} on t in "
          f"[{res['fit']['t_min']:.0f}, {res['fit']['t_max']:.0f}], "
          f"ensemble {res['ensemble_flips_per_ns']:.0f} flips/ns")
    for f, ts, b, e in zip(res["f"], res["t_switch"], res["fit"]["b"], res["fit"]["b_err"]):
        print(f"  f = {f:.2f}  t_switch = {ts:5d}  b = {b:+.3e} +- {e:.1e}")
    if a.json:
        with open(a.json, "w") as fh:
            json.dump(res, fh)


if __name__ == "__main__":
    main()
