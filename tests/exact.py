"""Exact equilibrium results used to pin the oracle's dynamics.

Independent of the oracle: these are the Boltzmann averages of Eq. (1)
computed by brute-force enumeration (small L) and by Kaufman's exact
partition function of the Ising model on an L x L torus (any L), plus the
infinite-lattice closed forms of Onsager (energy) and Yang (spontaneous
magnetisation).
"""
import itertools
import math

import mpmath
import numpy as np
from scipy.special import ellipk


def _spins_from_codes(codes, nsite, q):
    """Rows of site values for integer state codes (base q digits)."""
    codes = np.asarray(codes, dtype=np.int64)
    out = np.empty((codes.size, nsite), dtype=np.int64)
    c = codes.copy()
    for i in range(nsite):
        out[:, i] = c % q
        c //= q
    return out


def _bond_sum(sp, L):
    """sum over sites of s_x (s_{x+e1} + s_{x+e2}), periodic, for rows of spins."""
    g = sp.reshape(-1, L, L)
    return (g * (np.roll(g, -1, axis=2) + np.roll(g, -1, axis=1))).sum(axis=(1, 2))


def enumerate_ising(L, beta):
    """Exact <e>, <|m|>, <m^2>, <m^4> (per spin) by summing 2^(L^2) states."""
    n = L * L
    codes = np.arange(2 ** n, dtype=np.int64)
    sp = 2 * _spins_from_codes(codes, n, 2) - 1
    B = _bond_sum(sp, L)
    M = sp.sum(axis=1)
    w = np.exp(beta * (B - B.max()))
    Z = w.sum()
    avg = lambda f: float((w * f).sum() / Z)
    return {"e": avg(-B / n), "absm": avg(np.abs(M) / n), "m2": avg((M / n) ** 2),
            "m4": avg((M / n) ** 4)}


def enumerate_blume_capel(L, beta, delta):
    """Exact <e>, <|m|>, <m^2>, <q> (per spin) for the Blume-Capel model.

    Sums the 3^(L^2) states row by row: a state is L row states, each one of
    3^L; the bond sum splits into bonds inside rows and bonds between
    consecutive rows (periodic), so the sum is a loop over the first row and
    a broadcast over the others.
    """
    nr = 3 ** L
    rows = _spins_from_codes(np.arange(nr), L, 3) - 1           # (nr, L)
    r_m = rows.sum(axis=1)
    r_q = (rows * rows).sum(axis=1)
    r_b = (rows * np.roll(rows, -1, axis=1)).sum(axis=1)          # inside a row
    inter = rows @ rows.T                                         # (nr, nr) between rows
    n = L * L
    Z = e1 = am = m2 = qq = 0.0
    emax = beta * 2 * n + abs(beta * delta) * n                   # bound for scaling
    for r0 in range(nr):
        # accumulate over r1..r_{L-1} with arrays indexed by the last row
        # state: partial sums of B, M, Q carried as explicit arrays.
        B = r_b[r0] + np.zeros(1)
        M = r_m[r0] + np.zeros(1, dtype=np.int64)
        Q = r_q[r0] + np.zeros(1, dtype=np.int64)
        last = np.array([r0])
        for _ in range(1, L):
            B = (B[:, None] + inter[last][:, :] + r_b[None, :]).reshape(-1)
            M = (M[:, None] + r_m[None, :]).reshape(-1)
            Q = (Q[:, None] + r_q[None, :]).reshape(-1)
            last = np.tile(np.arange(nr), last.size)
        B = B + inter[last, r0]                                    # wrap bond
        logw = beta * B - beta * delta * Q - emax
        w = np.exp(logw)
        E = -B + delta * Q
        Z += w.sum()
        e1 += (w * E).sum() / n
        am += (w * np.abs(M)).sum() / n
        m2 += (w * (M / n) ** 2).sum()
        qq += (w * Q).sum() / n
    return {"e": e1 / Z, "absm": am / Z, "m2": m2 / Z, "q": qq / Z}


def kaufman_log_z(L, K, prec=60):
    """ln Z of the L x L periodic Ising model at coupling K (Kaufman 1949).

    Z = 1/2 (2 sinh 2K)^(L^2/2) [P1 + P2 + P3 + P4] with
      P1 = prod_r 2 cosh(L g_{2r+1}/2), P2 = prod_r 2 sinh(L g_{2r+1}/2),
      P3 = prod_r 2 cosh(L g_{2r}/2),   P4 = prod_r 2 sinh(L g_{2r}/2),
    r = 0..L-1, cosh g_l = cosh 2K cosh 2K* - sinh 2K sinh 2K* cos(pi l / L),
    tanh K* = e^{-2K}, and g_0 = 2 (K - K*) carrying its sign.
    """
    with mpmath.workdps(prec):
        K = mpmath.mpf(K)
        Ks = -mpmath.log(mpmath.tanh(K)) / 2
        c2, s2 = mpmath.cosh(2 * K), mpmath.sinh(2 * K)
        c2s, s2s = mpmath.cosh(2 * Ks), mpmath.sinh(2 * Ks)

        def gamma(l):
            if l % (2 * L) == 0:
                return 2 * (K - Ks)
            return mpmath.acosh(c2 * c2s - s2 * s2s * mpmath.cos(mpmath.pi * l / L))

        P = [mpmath.mpf(1)] * 4
        for r in range(L):
            go, ge = gamma(2 * r + 1), gamma(2 * r)
            P[0] *= 2 * mpmath.cosh(L * go / 2)
            P[1] *= 2 * mpmath.sinh(L * go / 2)
            P[2] *= 2 * mpmath.cosh(L * ge / 2)
            P[3] *= 2 * mpmath.sinh(L * ge / 2)
        Z = mpmath.mpf(0.5) * (2 * s2) ** (mpmath.mpf(L * L) / 2) * (P[0] + P[1] + P[2] + P[3])
        return mpmath.log(Z)


def kaufman_energy(L, K, prec=60):
    """Exact <e> per spin, -d ln Z / dK / L^2, by a high-precision central difference."""
    with mpmath.workdps(prec):
        h = mpmath.mpf(10) ** (-(prec // 3))
        d = (kaufman_log_z(L, mpmath.mpf(K) + h, prec) - kaufman_log_z(L, mpmath.mpf(K) - h, prec)) / (2 * h)
        return float(-d / (L * L))


def onsager_energy(beta):
    """Infinite-lattice energy per spin, u = -coth 2b [1 + (2/pi)(2 tanh^2 2b - 1) K(k)]."""
    k = 2 * math.sinh(2 * beta) / math.cosh(2 * beta) ** 2
    return -1 / math.tanh(2 * beta) * (1 + 2 / math.pi * (2 * math.tanh(2 * beta) ** 2 - 1) * ellipk(k * k))


def yang_magnetisation(beta):
    """Spontaneous magnetisation (1 - sinh^-4 2b)^(1/8) for b > b_c, else 0."""
    s = math.sinh(2 * beta)
    return (1 - s ** -4) ** 0.125 if s > 1 else 0.0
