"""Staggered operator, its Kahler-Dirac split and the KD-preconditioned operator.

Test infrastructure (oracle).  Definitions followed:

* M = m + D (Sec. 2.2 writes D_stag = (B + m) + C, Eq. 1).  The paper prints
  no formula for D.  The reading used here is the standard staggered form with
  a factor 1/2 on the hops, which is the normalisation whose free-field
  eigenvalues are +-i*sqrt(sum_mu sin^2 p_mu):

      (D psi)(x) = 1/2 sum_mu eta_mu(x) [ V_mu(x) psi(x+mu) - V_mu(x-mu)^dag psi(x-mu) ]
                 + c_N/2 sum_mu eta_mu(x) [ W_mu(x) psi(x+3mu) - W_mu(x-3mu)^dag psi(x-3mu) ]

  with fat links V and, for the HISQ-shaped operator (Sec. 2.2, 3.1), Naik
  links W at distance three.
* B = the distance-one hops that stay inside an aligned 2^4 hypercube; C = all
  other hops, including every Naik hop (Eq. 1, Sec. 2.2).
* (B + m)^{-1} is block local: one dense 48x48 matrix per hypercube
  (16 sites x 3 colours), ordered (position b, colour a) -> 3*b + a (Sec. 3.1).
* A = (B + m)^{-1} M (Eq. 2 with the mass, Sec. 3.1).
* Boundary conditions: periodic, or antiperiodic in time (``bc_t = -1``):
  psi(x + L_t t) = -psi(x), so a hop whose neighbour wraps around the time
  extent carries a factor -1.  (Thermal / propagator work on staggered
  fermions uses the antiperiodic time boundary; the paper does not state its
  boundary conditions.)
"""
from __future__ import annotations

import numpy as np

from .lattice import Lattice


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


class Staggered:
    """M = m + D on one lattice, optionally with Naik links."""

    def __init__(self, lat: Lattice, fat, naik=None, c_naik: float = 0.0, mass: float = 0.0, bc_t: int = 1):
        self.lat = lat
        self.fat = np.asarray(fat, dtype=np.complex128)
        self.naik = None if naik is None else np.asarray(naik, dtype=np.complex128)
        self.c_naik = float(c_naik)
        self.mass = float(mass)
        assert bc_t in (1, -1)
        self.bc_t = int(bc_t)
        assert self.fat.shape == (4, lat.V, 3, 3)
        self._eta = [lat.eta(mu) for mu in range(4)]

    def boundary_phase(self, mu, k):
        """Per site: the factor of psi(x + k mu) relative to the periodic
        value, -1 where an antiperiodic time hop wraps around, else +1."""
        if mu != 3 or self.bc_t == 1:
            return np.ones(self.lat.V)
        t = self.lat.coords[:, 3] + k
        wraps = (t >= self.lat.dims[3]) | (t < 0)
        return np.where(wraps, -1.0, 1.0)

    # -- individual hops -------------------------------------------------------
    def _hops(self):
        """(mu, k, sign, links, coefficient) for every hop family of D."""
        fams = []
        for mu in range(4):
            fams.append((mu, 1, +1, self.fat, 0.5))
            fams.append((mu, 1, -1, self.fat, 0.5))
        if self.naik is not None:
            for mu in range(4):
                fams.append((mu, 3, +1, self.naik, 0.5 * self.c_naik))
                fams.append((mu, 3, -1, self.naik, 0.5 * self.c_naik))
        return fams

    def hop(self, psi, mu, k, sign, links, coef):
        """One hop family applied to psi, including eta_mu(x) and the coefficient.

        sign=+1: +coef*eta_mu(x) * L_mu(x) psi(x + k mu)
        sign=-1: -coef*eta_mu(x) * L_mu(x - k mu)^dag psi(x - k mu)
        """
        lat = self.lat
        if sign > 0:
            n = lat.neighbor(mu, k)
            t = np.einsum("xab,xb->xa", links[mu], psi[n])
        else:
            n = lat.neighbor(mu, -k)
            t = -np.einsum("xab,xb->xa", _dag(links[mu][n]), psi[n])
        return coef * (self._eta[mu] * self.boundary_phase(mu, sign * k))[:, None] * t

    def D(self, psi):
        out = np.zeros_like(psi, dtype=np.complex128)
        for fam in self._hops():
            out += self.hop(psi, *fam)
        return out

    def M(self, psi):
        return self.mass * psi + self.D(psi)

    def Mdag(self, psi):
        # D is anti-Hermitian (pinned by tests), so M^dag = m - D.
        return self.mass * psi - self.D(psi)

    # -- Kahler-Dirac split (Eq. 1) -------------------------------------------
    def _in_block(self, mu, sign):
        """Mask of sites whose distance-one hop in (mu, sign) stays in the hypercube."""
        xm = self.lat.coords[:, mu]
        return (xm % 2 == 0) if sign > 0 else (xm % 2 == 1)

    def B(self, psi):
        out = np.zeros_like(psi, dtype=np.complex128)
        for mu in range(4):
            for sign in (+1, -1):
                t = self.hop(psi, mu, 1, sign, self.fat, 0.5)
                out += np.where(self._in_block(mu, sign)[:, None], t, 0.0)
        return out

    def C(self, psi):
        return self.D(psi) - self.B(psi)

    # -- hops split by aggregate crossing (for the Galerkin stencil) ------------
    def M_parts(self, psi, agg):
        """All nine aggregate-crossing parts of M psi from one pass over the
        hops (see ``M_part``); their sum is M psi."""
        keys = ["self"] + [(mu, s) for mu in range(4) for s in (+1, -1)]
        out = {k: np.zeros_like(psi, dtype=np.complex128) for k in keys}
        out["self"] += self.mass * psi
        for (mu, k, sign, links, coef) in self._hops():
            r = self.lat.in_aggregate_coord(agg, mu)
            a = int(agg[mu])
            cross = ((r + k >= a) if sign > 0 else (r - k < 0))[:, None]
            t = self.hop(psi, mu, k, sign, links, coef)
            out["self"] += np.where(cross, 0.0, t)
            out[(mu, sign)] += np.where(cross, t, 0.0)
        return out

    def M_part(self, psi, agg, part):
        """The part of M psi that, at output site x, reads psi from:

        part == "self":       x's own aggregate (and the mass term);
        part == (mu, +1):     the next aggregate along +mu;
        part == (mu, -1):     the previous aggregate along -mu.

        A hop of k sites from x crosses forward when (x_mu mod a_mu) + k >= a_mu
        and backward when (x_mu mod a_mu) - k < 0; the split is geometric, so
        it stays well defined when the coarse lattice has extent 1 or 2.
        """
        out = np.zeros_like(psi, dtype=np.complex128)
        if part == "self":
            out += self.mass * psi
        for (mu, k, sign, links, coef) in self._hops():
            r = self.lat.in_aggregate_coord(agg, mu)
            a = int(agg[mu])
            cross = (r + k >= a) if sign > 0 else (r - k < 0)
            if part == "self":
                keep = ~cross
            else:
                pmu, psign = part
                if pmu != mu or psign != sign:
                    continue
                keep = cross
            out += np.where(keep[:, None], self.hop(psi, mu, k, sign, links, coef), 0.0)
        return out


class KahlerDirac:
    """The block inverse (B+m)^{-1} and A = (B+m)^{-1} M (Eq. 2)."""

    def __init__(self, op: Staggered):
        self.op = op
        self.lat = op.lat
        self.sites = self.lat.kd_sites()            # (nblk, 16)
        self.blocks = self.build_blocks()           # (nblk, 48, 48): B + m
        self.inv = np.linalg.inv(self.blocks)       # (B + m)^{-1}

    def build_blocks(self):
        """Dense B + m per hypercube, column by column from the operator.

        Column (b, a) of every block at once: put a 1 at colour a of position
        b in every hypercube, apply B + m, read each block back.  B is block
        local, so the hypercubes do not mix.
        """
        nblk = self.sites.shape[0]
        mats = np.zeros((nblk, 48, 48), dtype=np.complex128)
        for b in range(16):
            for a in range(3):
                e = np.zeros((self.lat.V, 3), dtype=np.complex128)
                e[self.sites[:, b], a] = 1.0
                col = self.op.B(e) + self.op.mass * e
                mats[:, :, 3 * b + a] = col[self.sites].reshape(nblk, 48)
        return mats

    def gather(self, psi):
        return psi[self.sites].reshape(-1, 48)

    def scatter(self, blk):
        out = np.empty((self.lat.V, 3), dtype=np.complex128)
        out[self.sites] = blk.reshape(-1, 16, 3)
        return out

    def apply_inv(self, psi):
        return self.scatter(np.einsum("nij,nj->ni", self.inv, self.gather(psi)))

    def apply_inv_dag(self, psi):
        return self.scatter(np.einsum("nji,nj->ni", np.conj(self.inv), self.gather(psi)))

    def A(self, psi):
        return self.apply_inv(self.op.M(psi))

    def Adag(self, psi):
        return self.op.Mdag(self.apply_inv_dag(psi))

    def A_parts(self, psi, agg):
        return {k: self.apply_inv(v) for k, v in self.op.M_parts(psi, agg).items()}

    def A_part(self, psi, agg, part):
        """(B+m)^{-1} applied to one aggregate-crossing part of M (hypercubes
        nest inside aggregates, so the block inverse never changes the part)."""
        return self.apply_inv(self.op.M_part(psi, agg, part))


def gauge_transform_links(lat: Lattice, links, g, k: int = 1):
    """L_mu(x) -> g(x) L_mu(x) g(x + k mu)^dag for a link of length k."""
    out = np.empty_like(links)
    for mu in range(4):
        n = lat.neighbor(mu, k)
        out[mu] = g @ links[mu] @ _dag(g[n])
    return out
