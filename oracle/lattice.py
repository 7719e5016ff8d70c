"""Four-dimensional periodic lattice with fermion boundary phases.

The paper (Sec. 2, Eq. 1) splits sites into even and odd by checkerboard
parity; it does not print the indexing.  Reading taken: extents
(Lx, Ly, Lz, Lt), all even; site index i = x + Lx*(y + Ly*(z + Lz*t));
parity (x + y + z + t) mod 2, even = 0.  A hop that crosses the boundary in
direction mu multiplies the spinor it carries by bc[mu] (+1 periodic,
-1 antiperiodic; the default is periodic in x, y, z and antiperiodic in t).
"""

from __future__ import annotations

import numpy as np


class Lattice:
    def __init__(self, dims):
        self.dims = tuple(int(d) for d in dims)
        if len(self.dims) != 4 or any(d < 2 or d % 2 for d in self.dims):
            raise ValueError(f"extents must be four even numbers >= 2, got {dims}")
        Lx, Ly, Lz, Lt = self.dims
        self.V = Lx * Ly * Lz * Lt
        i = np.arange(self.V)
        self.coords = np.stack([i % Lx, (i // Lx) % Ly, (i // (Lx * Ly)) % Lz, i // (Lx * Ly * Lz)])
        self.parity = self.coords.sum(axis=0) % 2
        self.even = np.nonzero(self.parity == 0)[0]
        self.odd = np.nonzero(self.parity == 1)[0]

    def index(self, c) -> np.ndarray:
        Lx, Ly, Lz, _ = self.dims
        return c[0] + Lx * (c[1] + Ly * (c[2] + Lz * c[3]))

    def neighbor(self, sites, mu: int, step: int):
        """Sites x + step*mu-hat (step = +1 or -1) and whether the hop wraps."""
        c = self.coords[:, sites].copy()
        L = self.dims[mu]
        wraps = (c[mu] == L - 1) if step > 0 else (c[mu] == 0)
        c[mu] = (c[mu] + step) % L
        return self.index(c), wraps

    def sites_of(self, parity: int) -> np.ndarray:
        return self.even if parity == 0 else self.odd

    def embed(self, v_half, parity: int) -> np.ndarray:
        """Full-lattice spinor that equals v_half on one parity and 0 elsewhere."""
        full = np.zeros((self.V,) + v_half.shape[1:], dtype=np.complex128)
        full[self.sites_of(parity)] = v_half
        return full
