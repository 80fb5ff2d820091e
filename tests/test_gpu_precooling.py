"""The pre-cooling protocol on the GPU ("Thermal protocols", Eq. (8)).

Parity: the protocol's replica ensemble (t_switch sweeps at T1, then T2,
records during the T2 stage) reproduces the oracle's B and Q bit for bit for
every replica and record, for both models, and the vectorised record read
equals the per-object read.

Physics at scaled size (xi_eq(T2) ~ 20 instead of the paper's ~400): the
amplitude b(f) of the late exponential approach is positive for a short
pre-cooling (energy approaching equilibrium from above), negative for a long
one, and its zero f* lies near the paper's universal 0.59(5).  The scan
takes about 30 s per model.
"""
import math

import numpy as np
import pytest

from paper_2503_14688_b300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def isg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2503_14688_b300 import build

    build.build()
    import paper_2503_14688_b300 as P

    return P


@pytest.mark.parametrize("model,delta", [(wl.ISING, 0.0), (wl.BLUME_CAPEL, 0.3)])
def test_protocol_records_match_oracle(isg, orc, model, delta):
    from paper_2503_14688_b300 import precooling as pc
    Tc = wl.T_C_ISING if model == wl.ISING else wl.T_C_BLUME_CAPEL
    T1, T2 = pc.T1_OVER_TC * Tc, 1.04 * Tc
    L, n, seed, t_sw, t_tot, k = 64, 3, wl.BASE_SEED + 4321, 20, 60, 10
    t, E, Ee, B, Q = pc.energy_relaxation(model, L, T1, T2, t_sw, t_tot, k, n, seed, delta=delta,
                                          raw=True)
    assert t.tolist() == [30, 40, 50, 60]
    betas = [1.0 / T1] * t_sw + [1.0 / T2] * (t_tot - t_sw)
    for r in range(n):
        s = orc.init_random(L, model, seed + r)
        bmq, _, _ = orc.run(s, model, seed + r, 0, betas, delta=delta, record_every=k,
                            with_rows=False)
        assert np.array_equal(B[:, r], bmq[2:, 0]), r
        assert np.array_equal(Q[:, r], bmq[2:, 2]), r
    e = (-B.astype(np.float64) + delta * Q) / (L * L)
    assert np.array_equal(E, e.mean(axis=1))


def test_read_scalars_equals_read_records(isg):
    ens = isg.Ensemble([64, 128, 64], [1, 2, 3], models=[0, 1, 0], delta=0.2, record_capacity=4)
    ens.init_random()
    ens.sweep(6, beta=0.4, record_every=3)
    rows = ens.read_records(with_sums=False)
    ens.sweep(6, beta=0.4, record_every=3)
    sw, B, M, Q = ens.read_scalars()
    ens.close()
    ens = isg.Ensemble([64, 128, 64], [1, 2, 3], models=[0, 1, 0], delta=0.2, record_capacity=4)
    ens.init_random()
    ens.sweep(6, beta=0.4, record_every=3)
    sw0, B0, M0, Q0 = ens.read_scalars()
    ens.close()
    assert sw.tolist() == [9, 12] and sw0.tolist() == [3, 6]
    for i, row in enumerate(rows):
        assert [o.B for o in row] == B0[i].tolist()
        assert [o.M for o in row] == M0[i].tolist()
        assert [o.Q for o in row] == Q0[i].tolist()


@pytest.mark.parametrize("model", [wl.ISING, wl.BLUME_CAPEL])
def test_precooling_amplitude_changes_sign_near_paper_value(isg, model):
    from paper_2503_14688_b300 import precooling as pc
    fs = [0.0, 0.3, 0.45, 0.6, 0.75]
    res = pc.scan(model, fs, n_replicas=4096, n_xi=16, t_after=1000)
    b, e = np.asarray(res["fit"]["b"]), np.asarray(res["fit"]["b_err"])
    assert 15.0 < res["xi_eq"] < 30.0, res["xi_eq"]
    assert res["fit"]["chi2_per_dof"] < 1.5
    # short pre-cooling approaches from above, long from below (Fig. 4)
    assert b[1] > 3 * e[1] and b[-1] < -3 * e[-1], (b, e)
    # the zero: paper 0.59(5) at xi_eq ~ 400; here xi_eq ~ 20
    assert 0.45 < res["f_star"] < 0.70, (res["f_star"], res["f_star_err"])
    # switch times grow with f; the ensemble ran on the GPU at speed
    assert all(a < b2 for a, b2 in zip(res["t_switch"][1:], res["t_switch"][2:]))
    assert res["ensemble_flips_per_ns"] > 100.0
    assert math.isfinite(res["fit"]["tau"]) and res["fit"]["tau"] > 10
