"""The critical temperature of the Blume-Capel model at Delta = 0 from
equilibrium EMCS runs and histogram reweighting (Appendix B), at scaled
statistics: 16 lattices x 3000 EMCS (10 Metropolis sweeps + one
Swendsen-Wang iteration each) per size at the paper's beta_c, for L = 128
and 256.  The crossings beta_{L,U} and beta_{L,xi} of U4 and xi_2/L with
their universal values must lie within four jackknife errors plus 1e-4 of
the paper's beta_c = 1/1.69355839821214427017 (Table I); the paper finds
them constant from L = 64 on.  About 40 s on a B300.
"""
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


@pytest.mark.parametrize("L", [128, 256])
def test_blume_capel_critical_temperature(isg, L):
    from paper_2503_14688_b300 import tc

    beta_c = 1.0 / wl.T_C_BLUME_CAPEL
    s = tc.sample(L, beta_c, n_lattices=16, therm=200, meas=3000, seed=wl.BASE_SEED + 9900 + L)
    for which in ("u4", "xi"):
        b, e = tc.crossing_with_error(s, which)
        assert abs(b - beta_c) < 4 * e + 1e-4, (which, b, e)
        assert e < 1e-4
