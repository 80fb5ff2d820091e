"""Host analysis of the pre-cooling protocol (paper_2503_14688_b300.precooling),
pinned against closed forms and independent computations:

  * E_eq: Onsager's energy against a numerical derivative-free route, the
    average over the Brillouin zone of d/dbeta of the free-energy integrand
    (Onsager 1944), and -sqrt 2 at beta_c (Results);
  * xi = I2/I1 (Appendix C): the distances of steps (i)-(ii) by brute force;
    the tail-fit branch on an exact Eq. (13) curve against the closed form
    I2/I1 = xi_F Gamma(5/(2b)) / Gamma(3/(2b));
  * the joint fit of Eq. (8): exact recovery on noise-free data, coverage on
    noisy data, the window rule on a two-exponential curve;
  * the zero of b(f) and the switch time on exact inputs.
"""
import math

import numpy as np
import pytest

from paper_2503_14688_b300 import precooling as pc


def _u_zone_average(beta, n=1200):
    # -(d/dbeta) of ln Z/N = ln 2 + (1/8pi^2) int int ln[cosh^2 2b - sinh 2b (cos p + cos q)]
    th = (np.arange(n) + 0.5) * 2.0 * np.pi / n
    c = np.cos(th)[:, None] + np.cos(th)[None, :]
    ch, sh = math.cosh(2 * beta), math.sinh(2 * beta)
    return -0.5 * float(((4 * ch * sh - 2 * ch * c) / (ch * ch - sh * c)).mean())


@pytest.mark.parametrize("beta", [0.1, 0.25, 0.35, 0.5, 0.7])
def test_onsager_energy_matches_free_energy_derivative(beta):
    assert pc.onsager_energy(beta) == pytest.approx(_u_zone_average(beta), abs=1e-9)


def test_onsager_energy_limits():
    bc = math.log(1 + math.sqrt(2)) / 2
    assert pc.onsager_energy(bc) == -math.sqrt(2)
    # continuous through beta_c, -2 tanh(beta) at high temperature, -2 at T -> 0
    assert pc.onsager_energy(bc * (1 + 1e-9)) == pytest.approx(-math.sqrt(2), abs=1e-6)
    assert pc.onsager_energy(1e-3) == pytest.approx(-2 * math.tanh(1e-3), rel=1e-5)
    assert pc.onsager_energy(3.0) == pytest.approx(-2.0, abs=1e-9)


def _brute_cuts(C, err):
    n = len(C)
    r_cut = next(r for r in range(n - 1) if C[r + 1] < 3 * err[r + 1])
    w = [r * r * C[r] for r in range(r_cut + 1)]
    r_star = max(range(r_cut + 1), key=lambda r: w[r])
    r_min = next(r for r in range(r_star + 1, r_cut + 1) if w[r] < 0.9 * w[r_star])
    r_max = next(r for r in range(r_star + 1, r_cut + 1) if w[r] < w[r_star] / 3)
    return r_cut, r_star, r_min, r_max


def test_appendix_c_distances_brute_force():
    rng = np.random.default_rng(5)
    r = np.arange(400, dtype=float)
    for xi in (3.0, 7.5, 20.0):
        C = np.exp(-r / xi) * (1 + 0.01 * rng.standard_normal(r.size))
        err = np.full(r.size, 1e-6) + 0.002 * np.exp(-r / (3 * xi))
        assert pc.xi_cutoffs(C, err) == _brute_cuts(C, err)


def test_appendix_c_rejects_unresolved_curves():
    r = np.arange(50, dtype=float)
    with pytest.raises(ValueError):
        pc.xi_cutoffs(np.exp(-r / 0.3), np.full(r.size, 1e-3))   # xi well below one spacing
    with pytest.raises(ValueError):
        pc.xi_cutoffs(np.ones(50), np.full(50, 1e-3))             # never below 3 errors


@pytest.mark.parametrize("xi_F,beta_F", [(40.0, 1.0), (25.0, 1.3), (60.0, 0.8)])
def test_tail_fit_branch_against_closed_form(xi_F, beta_F):
    """Eq. (13) sampled exactly: I_n = A xi_F^(n+1/2) Gamma((n+1/2)/b) / b,
    so I2/I1 = xi_F Gamma(5/(2b)) / Gamma(3/(2b)).  The data part of the
    integral starts at r = 0 where F is singular (C(0) = 1 here), a bias of
    order 1/xi_F^(3/2) in I1."""
    r = np.arange(int(30 * xi_F), dtype=float)
    C = np.ones_like(r)
    C[1:] = 0.7 * np.exp(-np.power(r[1:] / xi_F, beta_F)) / np.sqrt(r[1:])
    err = 1e-8 + 1e-7 * C
    res = pc.xi_from_curve(C, err)
    assert res.tail_fit and res.r_max - res.r_min > 8
    want = xi_F * math.gamma(2.5 / beta_F) / math.gamma(1.5 / beta_F)
    assert res.xi == pytest.approx(want, rel=0.01)


def test_trapezoid_branch_short_range():
    # xi_exp = 1.2: r* = 2, r_min/r_max within 8 of each other -> plain integration
    r = np.arange(60, dtype=float)
    C = np.exp(-r / 1.2)
    err = np.full(r.size, 1e-9)
    res = pc.xi_from_curve(C, err)
    assert not res.tail_fit
    # integer-grid trapezoid of r^n e^{-r/x} in closed form (geometric sums)
    q = math.exp(-1 / 1.2)
    k = np.arange(0, res.r_cut + 1, dtype=float)
    w = np.ones_like(k)
    w[0] = w[-1] = 0.5
    I1 = float(np.sum(w * k * q ** k))
    I2 = float(np.sum(w * k * k * q ** k))
    assert res.xi == pytest.approx(I2 / I1, rel=1e-12)


def test_coherence_length_jackknife_error_scales():
    rng = np.random.default_rng(11)
    r = np.arange(300, dtype=float)
    base = np.exp(-r / 15.0) / np.sqrt(np.maximum(r, 1.0))
    def samples(n, noise):
        return base[None, :] + noise * rng.standard_normal((n, r.size))
    xi_a, e_a, _ = pc.coherence_length(samples(16, 2e-4))
    xi_b, e_b, _ = pc.coherence_length(samples(64, 2e-4))
    assert abs(xi_a - xi_b) < 4 * math.hypot(e_a, e_b)
    assert 0.3 < e_b / e_a < 0.8   # ~ 1/2 for four times the samples


def _synthetic(taus_amps, b, t, E_eq):
    return [E_eq + bi * sum(a * np.exp(-t / tau) for tau, a in taus_amps) for bi in b]


def test_fit_exact_recovery_fixed_and_free_E_eq():
    t = np.arange(50.0, 2000.0, 10.0)
    b = [3e-3, 1e-3, -2e-4, -4e-3]
    for E_eq in (-1.25, None):
        Es = _synthetic([(120.0, 1.0)], b, t, -1.25)
        fit = pc.fit_approach([t] * 4, Es, [np.full(t.size, 1e-7)] * 4, E_eq=E_eq)
        assert fit.tau == pytest.approx(120.0, rel=1e-8)
        assert np.allclose(fit.b, b, rtol=1e-7, atol=1e-12)
        assert fit.E_eq == pytest.approx(-1.25, abs=1e-10)
        assert fit.chi2 < 1e-6


def test_fit_noisy_coverage():
    rng = np.random.default_rng(3)
    t = np.arange(100.0, 800.0, 10.0)
    b = [4e-3, 1e-3, -1e-3]
    pulls = []
    for _ in range(40):
        Es = [e + 5e-5 * rng.standard_normal(t.size) for e in _synthetic([(80.0, 1.0)], b, t, -0.98)]
        fit = pc.fit_approach([t] * 3, Es, [np.full(t.size, 5e-5)] * 3, E_eq=None)
        pulls.append((fit.tau - 80.0) / fit.tau_err)
        assert abs(fit.chi2 / fit.dof - 1) < 0.5
    pulls = np.asarray(pulls)
    assert abs(pulls.mean()) < 0.6 and 0.6 < pulls.std() < 1.5


def test_window_rule_skips_fast_mode():
    t = np.arange(10.0, 3000.0, 10.0)
    b = [2e-3, -2e-3]
    Es = _synthetic([(200.0, 1.0), (25.0, 60.0)], b, t, -1.0)
    err = [np.full(t.size, 1e-6)] * 2
    t_min, t_max, fit = pc.choose_window([t] * 2, Es, err, -1.0, (50, 100, 200, 300, 400, 600), 800)
    # the fast mode's residual, 2e-3 * 60 exp(-t/25), is 4e-5 (40 errors) at
    # t = 200 and 7e-7 at t = 300
    assert (t_min, t_max) == (300.0, 1100.0)
    assert fit.tau == pytest.approx(200.0, rel=1e-3)


def test_zero_crossing_interpolation_and_error():
    f = [0.3, 0.4, 0.5, 0.6, 0.7]
    b = [5.0, 3.0, 1.0, -2.0, -6.0]
    e = [0.1, 0.1, 0.2, 0.3, 0.4]
    fs, err = pc.zero_crossing(f, b, e)
    assert fs == pytest.approx(0.5 + 0.1 * 1.0 / 3.0, rel=1e-12)
    # error by finite differences of the two bracketing amplitudes
    h = 1e-6
    d0 = (pc.zero_crossing(f, [5, 3, 1 + h, -2, -6], e)[0] - fs) / h
    d1 = (pc.zero_crossing(f, [5, 3, 1, -2 + h, -6], e)[0] - fs) / h
    assert err == pytest.approx(math.hypot(d0 * 0.2, d1 * 0.3), rel=1e-4)
    assert pc.zero_crossing(f[::-1], b[::-1], e[::-1])[0] == pytest.approx(fs, rel=1e-12)
    with pytest.raises(ValueError):
        pc.zero_crossing(f, [1, 2, 3, 4, 5], e)


def test_switch_time_power_law():
    t = 2.0 ** np.arange(2, 12)
    xi = 1.7 * np.sqrt(t)
    for target in (5.0, 12.3, 40.0):
        want = math.ceil((target / 1.7) ** 2 - 1e-9)
        assert pc.switch_time(t, xi, target) == want
    assert pc.switch_time(t, xi, 1.0) == 4
    xi_nan = xi.copy()
    xi_nan[:2] = np.nan
    assert pc.switch_time(t, xi_nan, 12.3) == math.ceil((12.3 / 1.7) ** 2 - 1e-9)
    with pytest.raises(ValueError):
        pc.switch_time(t, xi, 1e4)
