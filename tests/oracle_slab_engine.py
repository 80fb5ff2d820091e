"""A row slab backed by the oracle (test helper): the slab interface the
package's decomposition driver expects (edges, set_halos, half_sweep,
measure), computed by ``oracle.slab_half_sweep`` / ``oracle.slab_measure``
on one byte per site.  The edge and halo rows it exchanges are whole int8
rows (both colours), so the driver's exchange is tested on the CPU."""
import numpy as np

import oracle


class OracleSlab:
    def __init__(self, model, L, y0, rows, seed, delta=0.0):
        self.model, self.L, self.y0, self.rows = model, L, y0, rows
        self.seed, self.delta, self.t = seed, delta, 0
        self.buf = np.zeros((rows + 2, L), dtype=np.int8)
        self.buf[1:rows + 1] = oracle.window_init(rows, L, y0, 0, L, model, seed)

    def edges(self, colour):
        return self.buf[1].copy(), self.buf[self.rows].copy()

    def set_halos(self, colour, above, below):
        self.buf[0] = np.asarray(above)
        self.buf[self.rows + 1] = np.asarray(below)

    def half_sweep(self, colour, beta):
        oracle.slab_half_sweep(self.buf, self.y0, self.model, self.seed, self.t, colour, beta,
                               self.delta)
        if colour == 1:
            self.t += 1

    def measure(self):
        B, M, Q, R, C = oracle.slab_measure(self.buf)
        return self.t, B, M, Q, R, C

    def get(self):
        return self.buf[1:self.rows + 1].copy()
