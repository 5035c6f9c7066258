"""Block-preconditioned and Schur (even/odd) forms of a coarse operator (oracle).

Test infrastructure.  Sec. 2.3 coarsens the block-preconditioned version of
each coarse operator, analogous to even-odd preconditioning of Wilson-clover,
and Table 1 solves levels 2 and 3 with the "Schur-preconditioned" operator.
For the 9-point coarse stencil A_hat = X + Y (X the per-site self block, Y the
hops to the eight neighbouring sites):

* block-preconditioned: A' = X^{-1} A_hat = 1 + K with K = X^{-1} Y;
* with even extents the coarse lattice is bipartite (every hop changes the
  parity of the site), so A' = [[1, K_eo], [K_oe, 1]] and
  A_hat x = b  <=>  S x_e = c_e - K_eo c_o,  x_o = c_o - K_oe x_e,
  with c = X^{-1} b and the Schur complement S = 1 - K_eo K_oe on the even
  sites.

Fields are (V, N) arrays on the coarse lattice; even-site fields are (V_e, N)
in the order of the even sites.
"""
from __future__ import annotations

import numpy as np

from .coarse import CoarseStencil


class SchurCoarse:
    def __init__(self, S: CoarseStencil):
        lat = S.lat
        assert all(l % 2 == 0 for l in lat.dims), "even/odd needs even coarse extents"
        self.S = S
        self.lat = lat
        self.xinv = np.linalg.inv(S.X)                 # (V, N, N)
        par = lat.parity()
        self.even = np.flatnonzero(par == 0)
        self.odd = np.flatnonzero(par == 1)

    # -- pieces ----------------------------------------------------------------
    def hops(self, v):
        """Y v = A_hat v - X v."""
        return self.S.apply(v) - np.einsum("xij,xj->xi", self.S.X, v)

    def K(self, v):
        return np.einsum("xij,xj->xi", self.xinv, self.hops(v))

    def block_apply(self, v):
        """A' v = X^{-1} A_hat v."""
        return v + self.K(v)

    def _embed(self, ve, sites):
        out = np.zeros((self.lat.V, self.S.n), dtype=np.complex128)
        out[sites] = ve
        return out

    # -- Schur complement --------------------------------------------------------
    def schur_apply(self, ve):
        """S v_e = v_e - K_eo K_oe v_e."""
        to = self.K(self._embed(ve, self.even))[self.odd]
        return ve - self.K(self._embed(to, self.odd))[self.even]

    def schur_rhs(self, b):
        """c_e - K_eo c_o with c = X^{-1} b."""
        c = np.einsum("xij,xj->xi", self.xinv, b)
        return c[self.even] - self.K(self._embed(c[self.odd], self.odd))[self.even], c

    def reconstruct(self, xe, c):
        """Full solution from the even part: x_o = c_o - K_oe x_e."""
        x = self._embed(xe, self.even)
        x[self.odd] = c[self.odd] - self.K(self._embed(xe, self.even))[self.odd]
        return x

    def solve(self, b, solver):
        """A_hat x = b through the Schur system; `solver(apply, rhs)` returns x_e."""
        rhs, c = self.schur_rhs(b)
        return self.reconstruct(solver(self.schur_apply, rhs), c)
