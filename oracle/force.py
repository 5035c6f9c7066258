"""Fermion action and its derivative (oracle, test infrastructure).

S = phi^dag (M^dag M)^{-1} phi.  The paper names gauge generation (HMC) as a
future use of the solver (Sec. 4); the action's derivative is worked out here
from the operator of Sec. 2.2:

* X = (M^dag M)^{-1} phi, computed as Z = M^{-1} (eps phi), Y = eps Z, which
  equals M^{-dag} phi because eps M eps = M^dag, then X = M^{-1} Y;
  S = phi^dag X = ||Y||^2.
* dS = -2 Re[ Y^dag dM X ] with Y = M X.
* The link U_mu(x) enters the forward hop at x and the backward hop at x+mu
  with the same phase, so with G = dS/dRe U + i dS/dIm U (PyTorch's
  convention for the gradient of a real function of a complex tensor):

      G_mu(x) = -c eta_mu(x) [ Y(x) X(x+k mu)^dag - X(x) Y(x+k mu)^dag ]

  for a hop of length k with coefficient c/2 (c = 1 for fat links, c = c_N
  for Naik links, k = 3).
* dS/dm = -2 m ||X||^2, because Re(X^dag D X) = 0 for anti-Hermitian D.
"""
from __future__ import annotations

import numpy as np

from .dirac import Staggered


def action_vectors(op: Staggered, solve, phi):
    """(S, X, Y) with ``solve(b)`` returning M^{-1} b."""
    eps = op.lat.eps()[:, None]
    z = solve(eps * phi)
    y = eps * z
    x = solve(y)
    s = float(np.vdot(phi, x).real)
    return s, x, y


def link_gradient(op: Staggered, x, y, naik: bool = False):
    """G_mu(x) for the fat (or, with naik=True, the Naik) links, shape (4, V, 3, 3)."""
    k, c = (3, op.c_naik) if naik else (1, 1.0)
    g = np.empty((4, op.lat.V, 3, 3), dtype=np.complex128)
    for mu in range(4):
        n = op.lat.neighbor(mu, k)
        # the hop through U_mu(x) carries the boundary factor of x + k mu
        eta = (op.lat.eta(mu) * op.boundary_phase(mu, k))[:, None, None]
        outer = np.einsum("xa,xb->xab", y, np.conj(x[n])) - np.einsum("xa,xb->xab", x, np.conj(y[n]))
        g[mu] = -c * eta * outer
    return g


def mass_gradient(op: Staggered, x) -> float:
    return float(-2.0 * op.mass * np.vdot(x, x).real)
