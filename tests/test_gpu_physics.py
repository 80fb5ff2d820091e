"""Physics of the GPU path, independent of the oracle: equilibrium ensembles at
criticality must reproduce the universal values quoted in Appendix B for the
2D Ising universality class on the square lattice,
    U4* = <M^4>/<M^2>^2 = 1.1679229(47),   (xi_2/L)* = 0.9050488292(4),
for the Ising model at beta_c = ln(1 + sqrt 2)/2 and for the Blume-Capel
model at Delta = 0 at the paper's T_c = 1.69355839821214427017 (Table I).
This checks the equilibrium of the dynamics, the observables and the xi_2
formula together (and, loosely, the paper's Blume-Capel T_c estimate).

Tolerance: 4 jackknife standard errors (blocks of replicas) plus an allowance
for corrections to scaling at L = 64 (the paper finds crossings compatible
with their L -> infinity value from L >= 64 on, Appendix B).
"""
import math

import numpy as np
import pytest

from paper_2503_14688_b300 import workloads as wl

pytestmark = pytest.mark.gpu

U4_STAR = 1.1679229
XI_STAR = 0.9050488292


@pytest.fixture(scope="module")
def isg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2503_14688_b300 import build

    build.build()
    import paper_2503_14688_b300 as P

    return P


def _equilibrium(isg, model, L, beta, n=4096, therm=20000, meas=40000, every=500):
    seeds = [wl.BASE_SEED + 900 + 1000 * model + r for r in range(n)]
    ens = isg.Ensemble([L] * n, seeds, models=[model] * n, record_capacity=meas // every + 1)
    ens.init_random()
    ens.sweep(therm, beta=beta)
    ens.sweep(meas, beta=beta, record_every=every)
    rows = ens.read_records()
    ens.close()
    M = np.array([[o.M for o in row] for row in rows], dtype=np.int64)       # (k, n)
    R = np.array([[o.R for o in row] for row in rows], dtype=np.int32)       # (k, n, L)
    C = np.array([[o.C for o in row] for row in rows], dtype=np.int32)
    return M, R, C


def _u4(M):
    m = M.astype(np.float64)
    return (m ** 4).mean() / (m ** 2).mean() ** 2


def _xi_over_L(isg, M, R, C, L):
    return isg.xi2(M.reshape(-1), R.reshape(-1, L), C.reshape(-1, L)) / L


def _jackknife(f, n, blocks=16):
    bs = n // blocks
    vals = []
    for b in range(blocks):
        keep = np.ones(n, bool)
        keep[b * bs:(b + 1) * bs] = False
        vals.append(f(keep))
    vals = np.array(vals)
    return math.sqrt((blocks - 1) * ((vals - vals.mean()) ** 2).mean())


@pytest.mark.parametrize("model,beta", [(wl.ISING, wl.BETA_C_ISING),
                                        (wl.BLUME_CAPEL, 1.0 / wl.T_C_BLUME_CAPEL)])
def test_critical_u4_and_xi2_over_L(isg, model, beta):
    L = 64
    M, R, C = _equilibrium(isg, model, L, beta)
    n = M.shape[1]
    u4 = _u4(M)
    du4 = _jackknife(lambda k: _u4(M[:, k]), n)
    xi = _xi_over_L(isg, M, R, C, L)
    dxi = _jackknife(lambda k: _xi_over_L(isg, M[:, k], R[:, k], C[:, k], L), n)
    assert abs(u4 - U4_STAR) < 4 * du4 + 0.003, (u4, du4)
    assert abs(xi - XI_STAR) < 4 * dxi + 0.006, (xi, dxi)
    # sanity: the errors are small enough for the check to mean something
    assert du4 < 0.002 and dxi < 0.004
