"""The K-cycle multigrid preconditioner inside flexible GCR (oracle).

Test infrastructure.  Sec. 2.1 lists the preconditioner's five steps
(pre-smooth, restrict, iterate on the coarse system to a fixed tolerance,
prolongate and correct, post-smooth); Sec. 2.3 and Table 1 fix the levels:

* level 0: the full staggered operator M, outer flexible GCR to
  ||b - M x|| / ||b|| <= 1e-10 (Sec. 3.2), no pre-smoother, CA-GCR(8)
  post-smoother;
* level 1: the KD-preconditioned operator A = (B+m)^{-1} M on the same
  lattice ("pseudo-fine"), GCR to 0.25 or 8 iterations, CA-GCR(8)
  post-smoother.  The right-hand side handed down from level 0 is
  (B+m)^{-1} r, because M e = r and A e = (B+m)^{-1} r have the same
  solution;
* level 2, 3, ...: the Galerkin operators, GCR to 0.25 or 8 iterations with
  CA-GCR(8) post-smoothing, and on the coarsest level an exact dense solve
  (when it has at most ``dense_max`` unknowns) or GCR to 0.25 / 8
  iterations.

Table 1 offers two level-1 operators: the KD-preconditioned HISQ operator
above, or the "truncated" one, which drops the distance-three Naik hops from
the pseudo-fine operator (Sec. 3.1): A' = (B+m)^{-1} (m + D_fat).  The outer
level keeps the full M, so the truncation only changes the preconditioner
(the outer GCR is flexible); B holds distance-one hops only, so (B+m)^{-1} is
the same block inverse.  ``truncate_naik`` selects it.

Sec. 2.3 generates the near-null vectors of each coarse level with its
coarse operator A_hat and then coarsens the block-preconditioned operator
X^{-1} A_hat (X the self blocks), the coarse analogue of the KD
preconditioning of level 1.  ``block_coarse`` selects this: the level's GCR,
smoother and Galerkin product use X^{-1} A_hat, the right-hand side handed
down is X^{-1} R r, and the near-null CGNE runs on A_hat.

Table 1 solves the coarsest level with an SVD-deflated Chebyshev-basis
CA-GCR(16).  ``coarsest_deflate`` = k > 0 selects it (when the coarsest level
is not solved densely): the start V diag(1/sigma) U^dag b from the k lowest
singular triplets, then CA-GCR(s) steps with a Chebyshev basis on the real
interval [sigma_k, sigma_max] (the k-th singular value, the first one not
deflated, up to the largest one, which bounds the real part of every
eigenvalue), to the level's 0.25 / 8-step rule.  The interval only conditions
the basis: the correction is the minimum-residual one over K_s(A, r) for any
interval.  ``coarsest_basis = "shifted"`` builds the same Krylov space from
the power basis ((A - c)/h)^k r of the disk around the interval's centre,
which stays well conditioned when the spectrum fills a disk rather than
lying near the real interval (the synthetic coarse operators here).

Table 1 runs that coarsest solver on the "Schur-preconditioned" operator:
``coarsest_schur`` (with ``coarsest_deflate``) solves the coarsest system
through its even/odd Schur complement S = 1 - K_eo K_oe (oracle/schur.py):
the right-hand side c_e - K_eo c_o, the deflated Chebyshev-basis CA-GCR on S
with the singular triplets of S, then x_o = c_o - K_oe x_e.

``schur_coarse`` (with ``block_coarse``) puts the intermediate coarse levels
(level 2 of Table 1: "MG-preconditioned GCR" on the "Schur-preconditioned"
operator) in the same form: the level's GCR and post-smoother run on S with
right-hand side c_e - K_eo c_o, and the K-cycle below preconditions S as
follows.  For an even iterate x_e completed by x_o = c_o - K_oe x_e, the full
residual of A x = c is (r_e, 0) with r_e = c_e - K_eo c_o - S x_e the Schur
residual; so the K-cycle applied to the embedded residual (r_e, 0) corrects
the full system, and its even part corrects x_e.  Its coarse operator is the
Galerkin product of the full block-preconditioned operator (Sec. 2.3).

Readings taken where the paper is silent: no pre-smoothing anywhere (Table 1
lists none), "0.25 or 8 iterations" stops at whichever comes first, the
coarse levels use the un-preconditioned Galerkin operator unless
``block_coarse`` / ``schur_coarse`` / ``coarsest_schur`` select Table 1's
block-preconditioned and Schur forms above, and the outer GCR restarts every
16 directions with the residual recomputed at each restart.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

from .coarse import FineLevelOp, Transfer, block_preconditioned, galerkin, near_null_vectors
from .dirac import KahlerDirac, Staggered
from .lattice import Lattice
from .schur import SchurCoarse
from .solvers import ca_gcr, ca_gcr_basis, gcr, lowest_singular_triplets, norm


@dataclass
class MGParams:
    agg: list = field(default_factory=lambda: [(4, 4, 4, 4)])
    nvec: list = field(default_factory=lambda: [24])
    setup_tol: float = 1e-6
    setup_maxiter: int = 2000
    inner_tol: float = 0.25
    inner_maxiter: int = 8
    smoother_s: int = 8
    dense_max: int = 4096
    nkrylov: int = 16
    truncate_naik: bool = False
    block_coarse: bool = False
    coarsest_deflate: int = 0     # > 0: SVD-deflated Chebyshev-basis CA-GCR on the coarsest level
    coarsest_cheb_s: int = 8     # Table 1: 16; a real-interval basis that long is numerically singular here
    coarsest_basis: str = "chebyshev"   # or "shifted": the power basis of the disk around the interval's centre
    coarsest_schur: bool = False  # with coarsest_deflate: deflated CA-GCR on the even/odd Schur complement
    schur_coarse: bool = False    # intermediate coarse levels: GCR and smoother on the Schur complement
    coarse_inner_tol: float = 0.0     # levels >= 2: their own inner tolerance (0: inner_tol)
    coarse_inner_maxiter: int = 0     # levels >= 2: their own iteration cap (0: inner_maxiter)

    def tol_of(self, l: int) -> float:
        """Inner GCR tolerance of level l >= 1."""
        return self.coarse_inner_tol if (l >= 2 and self.coarse_inner_tol > 0) else self.inner_tol

    def maxiter_of(self, l: int) -> int:
        """Inner GCR iteration cap of level l >= 1."""
        return self.coarse_inner_maxiter if (l >= 2 and self.coarse_inner_maxiter > 0) else self.inner_maxiter


class MultigridSolver:
    def __init__(self, op: Staggered, params: MGParams, phi0):
        """op: M at level 0; phi0[l]: (nvec[l], V_l, n_l) random starts."""
        self.op = op
        self.p = params
        op1 = op
        if params.truncate_naik and op.naik is not None:
            op1 = Staggered(op.lat, op.fat, None, 0.0, op.mass, bc_t=op.bc_t)
        self.kd = KahlerDirac(op1)                # (B+m)^{-1}: distance-one hops only
        self.levels = [FineLevelOp(self.kd)]      # level 1 operator A (or A')
        self.raw = [self.levels[0]]              # operator the near-null CGNE uses, per level
        self.xinv = [None]                       # X^{-1} of each block-preconditioned level
        self.transfers = []
        self.setup_iters = []
        for l, (agg, nv) in enumerate(zip(params.agg, params.nvec)):
            lop = self.levels[-1]
            vecs, its = near_null_vectors(self.raw[-1], np.asarray(phi0[l]), params.setup_tol,
                                          params.setup_maxiter)
            self.setup_iters.append(its)
            T = Transfer(lop.lat, lop.n, lop.chirality(), agg, vecs)
            self.transfers.append(T)
            S = galerkin(lop, T)
            self.raw.append(S)
            if params.block_coarse:
                self.levels.append(block_preconditioned(S))
                self.xinv.append(np.linalg.inv(S.X))
            else:
                self.levels.append(S)
                self.xinv.append(None)
        coarsest = self.levels[-1]
        self.dense_lu = None
        self.defl = None
        self.schur = None
        if coarsest.lat.V * coarsest.n <= params.dense_max:
            self.dense_lu = scipy.linalg.lu_factor(coarsest.dense())
        elif params.coarsest_deflate > 0:
            self.schur = SchurCoarse(coarsest) if params.coarsest_schur else None
            Ad = coarsest.dense() if self.schur is None else self.schur_dense()
            U, sig, V = lowest_singular_triplets(Ad, params.coarsest_deflate)
            self.defl = (U, sig, V, float(sig[-1]), float(np.linalg.norm(Ad, 2)))

    def schur_dense(self):
        """The Schur complement S on the even sites as a dense matrix, column by
        column from unit vectors."""
        sc = self.schur
        ne, N = len(sc.even), sc.S.n
        D = np.empty((ne * N, ne * N), dtype=np.complex128)
        for j in range(ne * N):
            e = np.zeros(ne * N, dtype=np.complex128)
            e[j] = 1.0
            D[:, j] = sc.schur_apply(e.reshape(ne, N)).ravel()
        return D

    # --- the K-cycle -------------------------------------------------------------
    def coarse_solve(self, l, rc):
        """Approximate solve on level l >= 2 (index into self.levels is l-1)."""
        lop = self.levels[l - 1]
        if self.xinv[l - 1] is not None:          # X^{-1} A_hat e = X^{-1} rc
            rc = np.einsum("xij,xj->xi", self.xinv[l - 1], rc)
        if l - 1 == len(self.levels) - 1:
            if self.dense_lu is not None:
                x = scipy.linalg.lu_solve(self.dense_lu, rc.ravel())
                return x.reshape(rc.shape)
            if self.defl is not None:
                if self.schur is not None:
                    return self.schur.solve(rc, lambda apply, rhs: self.deflated_coarsest_op(apply, rhs))
                return self.deflated_coarsest(lop, rc)
            x, _, _ = gcr(lop.apply, rc, tol=self.p.tol_of(l), maxiter=self.p.maxiter_of(l),
                          nkrylov=self.p.maxiter_of(l), true_residual=False)
            return x
        if self.p.schur_coarse:
            sc = SchurCoarse(lop)
            rhs, c = sc.schur_rhs(rc)
            xe, _, _ = gcr(sc.schur_apply, rhs, precond=lambda r: self.kcycle_schur(l, sc, r),
                           tol=self.p.tol_of(l), maxiter=self.p.maxiter_of(l),
                           nkrylov=self.p.maxiter_of(l), true_residual=False)
            return sc.reconstruct(xe, c)
        x, _, _ = gcr(lop.apply, rc, precond=lambda r: self.kcycle(l, r),
                      tol=self.p.tol_of(l), maxiter=self.p.maxiter_of(l),
                      nkrylov=self.p.maxiter_of(l), true_residual=False)
        return x

    def deflated_coarsest(self, lop, rc):
        """SVD-deflated start, then Chebyshev-basis CA-GCR(s) steps until the
        residual is 0.25 of ||rc|| or after inner_maxiter steps."""
        return self.deflated_coarsest_op(lop.apply, rc)

    def deflated_coarsest_op(self, apply, rc):
        U, sig, V, lmin, lmax = self.defl
        x = (V @ ((U.conj().T @ rc.ravel()) / sig)).reshape(rc.shape)
        r = rc - apply(x)
        lc = len(self.levels)              # the coarsest level's number (levels[0] is level 1)
        target = self.p.tol_of(lc) * norm(rc)
        for _ in range(self.p.maxiter_of(lc)):
            if norm(r) <= target:
                break
            x = x + ca_gcr_basis(apply, r, self.p.coarsest_cheb_s, lmin, lmax, self.p.coarsest_basis)
            r = rc - apply(x)
        return x

    def kcycle(self, l, r):
        """K_l(r) for l >= 1: restrict, coarse solve, prolong, post-smooth."""
        lop = self.levels[l - 1]
        T = self.transfers[l - 1]
        e = T.prolong(self.coarse_solve(l + 1, T.restrict(r)))
        e = e + ca_gcr(lop.apply, r - lop.apply(e), self.p.smoother_s)
        return e

    def kcycle_schur(self, l, sc, re):
        """K-cycle for the Schur system of level l: the full-system K-cycle on
        the embedded residual (r_e, 0) (restrict, coarse solve, prolong), its
        even part, then CA-GCR(s) post-smoothing on S."""
        T = self.transfers[l - 1]
        full = sc._embed(re, sc.even)
        e = T.prolong(self.coarse_solve(l + 1, T.restrict(full)))[sc.even]
        e = e + ca_gcr(sc.schur_apply, re - sc.schur_apply(e), self.p.smoother_s)
        return e

    def precondition(self, r):
        """K_0(r): level-1 GCR on A e = (B+m)^{-1} r, then CA-GCR(8) on M."""
        r1 = self.kd.apply_inv(r)
        e, _, _ = gcr(self.levels[0].apply, r1, precond=lambda v: self.kcycle(1, v),
                      tol=self.p.inner_tol, maxiter=self.p.inner_maxiter,
                      nkrylov=self.p.inner_maxiter, true_residual=False)
        e = e + ca_gcr(self.op.M, r - self.op.M(e), self.p.smoother_s)
        return e

    def solve(self, b, tol=1e-10, maxiter=500):
        """Outer flexible GCR on M; returns (x, iterations, true residual)."""
        return gcr(self.op.M, b, precond=self.precondition, tol=tol, maxiter=maxiter,
                   nkrylov=self.p.nkrylov, true_residual=True)


def build(dims, fat, naik, c_naik, mass, params: MGParams, phi0):
    lat = Lattice(dims)
    return MultigridSolver(Staggered(lat, fat, naik, c_naik, mass), params, phi0)
