"""Lattice geometry for the oracle (test infrastructure only).

Sec. 2.2: staggered fermions carry N_c = 3 colour components per site; the
chirality is eps(x) = (-1)^(x+y+z+t); the Kahler-Dirac split groups sites into
aligned 2^d hypercubes.  Sec. 2.1 / Table 1: coarse levels aggregate blocks of
sites.  The paper writes none of the index conventions; the ones used here are:

* lexical site index x + Lx*(y + Ly*(z + Lz*t)), periodic boundaries;
* staggered phases eta_0 = 1, eta_1 = (-1)^x, eta_2 = (-1)^(x+y),
  eta_3 = (-1)^(x+y+z);
* hypercube of x = floor(x_mu / 2) per axis (lexical over the half lattice),
  position inside it b = (x&1) + 2(y&1) + 4(z&1) + 8(t&1);
* aggregate of x = floor(x_mu / a_mu) (lexical over the coarse lattice),
  position inside it lexical over the a_mu extents.
"""
from __future__ import annotations

import itertools

import numpy as np


class Lattice:
    def __init__(self, dims):
        self.dims = tuple(int(d) for d in dims)
        if len(self.dims) != 4 or any(d <= 0 for d in self.dims):
            raise ValueError(f"bad lattice extents {dims}")
        self.V = int(np.prod(self.dims))
        self.stride = (1, self.dims[0], self.dims[0] * self.dims[1],
                       self.dims[0] * self.dims[1] * self.dims[2])
        idx = np.arange(self.V, dtype=np.int64)
        c = np.empty((self.V, 4), dtype=np.int64)
        rem = idx
        for mu in range(4):
            c[:, mu] = rem % self.dims[mu]
            rem //= self.dims[mu]
        self.coords = c
        self._nbr = {}

    def index(self, coords) -> np.ndarray:
        coords = np.asarray(coords, dtype=np.int64)
        return (coords % np.asarray(self.dims)) @ np.asarray(self.stride, dtype=np.int64)

    def neighbor(self, mu: int, k: int) -> np.ndarray:
        """Index of x + k*mu_hat for every x (periodic)."""
        key = (mu, k)
        if key not in self._nbr:
            c = self.coords.copy()
            c[:, mu] += k
            self._nbr[key] = self.index(c)
        return self._nbr[key]

    def eta(self, mu: int) -> np.ndarray:
        """Staggered phase eta_mu(x) as +-1.0."""
        s = self.coords[:, :mu].sum(axis=1)
        return np.where(s % 2 == 0, 1.0, -1.0)

    def eps(self) -> np.ndarray:
        """Chirality eps(x) = (-1)^(x+y+z+t) (Sec. 2.2)."""
        return np.where(self.coords.sum(axis=1) % 2 == 0, 1.0, -1.0)

    def parity(self) -> np.ndarray:
        """0 on even sites (eps=+1), 1 on odd sites."""
        return (self.coords.sum(axis=1) % 2).astype(np.int64)

    # --- Kahler-Dirac hypercubes -------------------------------------------
    def kd_block(self):
        """(hypercube index, position inside the hypercube) per site."""
        if any(d % 2 for d in self.dims):
            raise ValueError("hypercube blocking needs even extents")
        half = [d // 2 for d in self.dims]
        hs = (1, half[0], half[0] * half[1], half[0] * half[1] * half[2])
        blk = (self.coords // 2) @ np.asarray(hs, dtype=np.int64)
        pos = ((self.coords & 1) * np.asarray([1, 2, 4, 8])).sum(axis=1)
        return blk, pos

    def n_kd_blocks(self) -> int:
        return self.V // 16

    def kd_sites(self) -> np.ndarray:
        """(V/16, 16) table: site index of position b in hypercube n."""
        blk, pos = self.kd_block()
        out = np.empty((self.V // 16, 16), dtype=np.int64)
        out[blk, pos] = np.arange(self.V)
        return out

    # --- aggregates ------------------------------------------------------------
    def coarse_dims(self, agg) -> tuple:
        agg = tuple(int(a) for a in agg)
        if any(d % a for d, a in zip(self.dims, agg)):
            raise ValueError(f"aggregate {agg} does not tile {self.dims}")
        return tuple(d // a for d, a in zip(self.dims, agg))

    def aggregate(self, agg):
        """(aggregate index, position inside the aggregate) per site."""
        agg = np.asarray(agg, dtype=np.int64)
        cd = self.coarse_dims(agg)
        cs = np.asarray((1, cd[0], cd[0] * cd[1], cd[0] * cd[1] * cd[2]), dtype=np.int64)
        a_s = np.asarray((1, agg[0], agg[0] * agg[1], agg[0] * agg[1] * agg[2]), dtype=np.int64)
        return (self.coords // agg) @ cs, (self.coords % agg) @ a_s

    def in_aggregate_coord(self, agg, mu: int) -> np.ndarray:
        """x_mu mod a_mu for every site."""
        return self.coords[:, mu] % int(agg[mu])


def enumerate_sites(dims):
    """Brute-force (t, z, y, x) nested loops: lexical index -> coordinates."""
    out = []
    for t, z, y, x in itertools.product(*(range(d) for d in reversed(dims))):
        out.append((x, y, z, t))
    return np.asarray(out, dtype=np.int64)
