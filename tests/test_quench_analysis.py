"""Host fits of the direct quench (paper_2503_14688_b300.quench), pinned on
synthetic data with known parameters:

  * Eq. (5), log t = z log xi + b + b' xi^-omega: exact recovery, with and
    without the correction term; error coverage on noisy xi;
  * Eq. (6), E - E_eq = b t^(-1/z) + b' t^(-2/z) + b'' t^(-(omega+1)/z):
    exact recovery; error coverage on noisy E;
  * the t_min window and the refusal of too few points.
"""
import math

import numpy as np
import pytest

from paper_2503_14688_b300 import quench as q


def _times_from_xi(xi, z, b, bp, omega=q.OMEGA):
    return np.exp(z * np.log(xi) + b + bp * xi ** -omega)


def test_xi_fit_exact_recovery():
    xi = np.geomspace(3.0, 150.0, 16)
    for z, b, bp in ((2.1676, 0.4, -0.8), (2.0, -0.3, 0.5)):
        t = _times_from_xi(xi, z, b, bp)
        f = q.fit_z_from_xi(t, xi, 1e-3 * xi)
        assert f.z == pytest.approx(z, abs=1e-10)
        assert np.allclose(f.coef, [b, bp], atol=1e-9)
        assert f.chi2 < 1e-12 and f.dof == xi.size - 3
    # without the correction the pure power law is recovered exactly
    t = _times_from_xi(xi, 2.1676, 0.4, 0.0)
    f = q.fit_z_from_xi(t, xi, 1e-3 * xi, corrections=False)
    assert f.z == pytest.approx(2.1676, abs=1e-10) and f.dof == xi.size - 2


def test_xi_fit_window_and_errors():
    xi = np.geomspace(3.0, 150.0, 16)
    t = _times_from_xi(xi, 2.17, 0.4, -0.8)
    xi_bad = xi.copy()
    xi_bad[:4] = np.nan                      # unresolved early points are skipped
    f = q.fit_z_from_xi(t, xi_bad, 1e-3 * xi)
    assert f.z == pytest.approx(2.17, abs=1e-10) and f.dof == 12 - 3
    f = q.fit_z_from_xi(t, xi, 1e-3 * xi, t_min=t[10])
    assert f.dof == 6 - 3
    with pytest.raises(ValueError):
        q.fit_z_from_xi(t[:3], xi[:3], 1e-3 * xi[:3])


def test_xi_fit_noise_coverage():
    rng = np.random.default_rng(7)
    t = 2.0 ** np.arange(3, 14)
    z, b, bp = 2.1676, 0.4, -0.8
    # xi solving log t = z log xi + b + b' xi^-omega, by fixed-point iteration
    xi = np.exp((np.log(t) - b) / z)
    for _ in range(200):
        xi = np.exp((np.log(t) - b - bp * xi ** -q.OMEGA) / z)
    pulls = []
    for _ in range(60):
        rel = 0.003
        xn = xi * (1 + rel * rng.standard_normal(xi.size))
        f = q.fit_z_from_xi(t, xn, rel * xi)
        pulls.append((f.z - z) / f.z_err)
    pulls = np.asarray(pulls)
    assert abs(pulls.mean()) < 0.5 and 0.6 < pulls.std() < 1.5


def _energy(t, z, b, bp, bpp, omega=q.OMEGA, e_eq=-math.sqrt(2.0)):
    return e_eq + b * t ** (-1 / z) + bp * t ** (-2 / z) + bpp * t ** (-(omega + 1) / z)


def test_energy_fit_exact_recovery():
    t = 2.0 ** np.arange(2, 15)
    e = _energy(t, 2.1676, 0.3, 0.1, -0.05)
    g = q.fit_z_from_energy(t, e, np.full(t.size, 1e-9))
    assert g.z == pytest.approx(2.1676, abs=1e-6)
    assert np.allclose(g.coef, [0.3, 0.1, -0.05], atol=1e-6)
    with pytest.raises(ValueError):
        q.fit_z_from_energy(t[:4], e[:4], np.full(4, 1e-9))


def test_energy_fit_noise_coverage():
    rng = np.random.default_rng(9)
    t = 2.0 ** np.arange(2, 14)
    e0 = _energy(t, 2.1676, 0.3, 0.1, -0.05)
    pulls = []
    for _ in range(60):
        s = 2e-6 + 1e-4 * t ** -0.5
        g = q.fit_z_from_energy(t, e0 + s * rng.standard_normal(t.size), s)
        pulls.append((g.z - 2.1676) / g.z_err)
    pulls = np.asarray(pulls)
    assert abs(pulls.mean()) < 0.5 and 0.6 < pulls.std() < 1.6
