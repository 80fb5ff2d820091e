"""Pins for the oracle's window mode (used for light-cone parity on lattices
too large for the full oracle): a window evolved with global keys and a fixed
outer ring must equal the full-lattice oracle on every site farther than 2n
from the ring after n sweeps -- the dependency of a site on its neighbours
moves one site per half-sweep -- and must differ near the ring."""
import numpy as np
import pytest


@pytest.mark.parametrize("model,delta", [(0, 0.0), (1, 0.0), (1, 0.4)])
def test_window_matches_full_lattice_inside_light_cone(orc, model, delta):
    L, seed, n = 128, 0x2503146880000021, 6
    full = orc.init_random(L, model, seed)
    betas = np.linspace(0.3, 0.6, n)
    for (y0, x0, h, w) in [(10, 20, 40, 50), (100, 110, 48, 44)]:  # second one wraps
        win = orc.window_init(h, w, y0, x0, L, model, seed)
        ref = np.roll(np.roll(full, -y0, 0), -x0, 1)[:h, :w]
        assert np.array_equal(win, ref)
    orc.run(full, model, seed, 0, betas, delta=delta)
    for (y0, x0, h, w) in [(10, 20, 40, 50), (100, 110, 48, 44)]:
        win = orc.window_init(h, w, y0, x0, L, model, seed)
        orc.window_run(win, y0, x0, L, model, seed, 0, betas, delta=delta)
        ref = np.roll(np.roll(full, -y0, 0), -x0, 1)[:h, :w]
        m = 2 * n + 1
        assert np.array_equal(win[m:h - m, m:w - m], ref[m:h - m, m:w - m])
        assert not np.array_equal(win, ref)  # the fixed ring does spoil the edge
