"""Near-null vectors, transfer operators and the Galerkin coarse operator.

Test infrastructure (oracle).  Sec. 2.1 and 2.3:

* near-null vectors: inverse iteration on the homogeneous system
  A phi = 0 from a random phi_0, here CGNE to a relative residual of 1e-6 or
  2000 iterations, whichever comes first (Table 1);
* chiral doubling: every vector v gives the two projections (1 +- Gamma) v / 2,
  Gamma = eps(x) on the fine lattice and +1 / -1 on the first / second half
  of a coarse site's components (Sec. 2.1, 2.2);
* block orthonormalisation of the doubled set inside each aggregate and
  chirality: modified Gram-Schmidt in vector order, done twice;
* R is built from the orthonormal vectors, P = R^dag, and the coarse operator
  A_hat = R A P is constructed explicitly (Sec. 2.1).  Because the block
  inverse is local to hypercubes nested in aggregates of extent >= 4 and the
  longest hop is three sites, A_hat couples an aggregate only to itself and
  its eight nearest aggregates: it is a 9-point stencil with a self block X
  and hop blocks Y_{+mu}, Y_{-mu}, each N x N with N = 2 * n_vec.

Coarse vectors have shape (V_c, N); component s*n_vec + k holds chirality s
(0: Gamma = +1) of vector k.
"""
from __future__ import annotations

import numpy as np

from .lattice import Lattice
from .solvers import cgne


class FineLevelOp:
    """Adapter: the KD-preconditioned operator A as a level operator."""

    def __init__(self, kd):
        self.kd = kd
        self.lat = kd.lat
        self.n = 3

    def apply(self, v):
        return self.kd.A(v)

    def apply_dag(self, v):
        return self.kd.Adag(v)

    def apply_parts(self, v, agg):
        return self.kd.A_parts(v, agg)

    def chirality(self):
        return np.repeat(self.lat.parity()[:, None], 3, axis=1)


class CoarseStencil:
    """9-point stencil operator (A_hat v)(X) = X v(X) + sum_mu Y_{+mu} v(X+mu) + Y_{-mu} v(X-mu)."""

    def __init__(self, lat: Lattice, X, Yf, Yb):
        self.lat = lat
        self.X = X          # (V, N, N)
        self.Yf = Yf        # (4, V, N, N), reads v(x + mu)
        self.Yb = Yb        # (4, V, N, N), reads v(x - mu)
        self.n = X.shape[-1]

    def apply(self, v):
        lat = self.lat
        out = np.einsum("xij,xj->xi", self.X, v)
        for mu in range(4):
            out += np.einsum("xij,xj->xi", self.Yf[mu], v[lat.neighbor(mu, 1)])
            out += np.einsum("xij,xj->xi", self.Yb[mu], v[lat.neighbor(mu, -1)])
        return out

    def apply_dag(self, v):
        """Adjoint: block (x, x+mu) of A_hat^dag is Y_{-mu}(x+mu)^dag, etc."""
        lat = self.lat
        out = np.einsum("xji,xj->xi", np.conj(self.X), v)
        for mu in range(4):
            fp, fm = lat.neighbor(mu, 1), lat.neighbor(mu, -1)
            out += np.einsum("xji,xj->xi", np.conj(self.Yb[mu][fp]), v[fp])
            out += np.einsum("xji,xj->xi", np.conj(self.Yf[mu][fm]), v[fm])
        return out

    def apply_parts(self, v, agg):
        lat = self.lat
        parts = {"self": np.einsum("xij,xj->xi", self.X, v)}
        for mu in range(4):
            r = lat.in_aggregate_coord(agg, mu)
            a = int(agg[mu])
            tf = np.einsum("xij,xj->xi", self.Yf[mu], v[lat.neighbor(mu, 1)])
            tb = np.einsum("xij,xj->xi", self.Yb[mu], v[lat.neighbor(mu, -1)])
            cf = (r + 1 >= a)[:, None]
            cb = (r - 1 < 0)[:, None]
            parts["self"] = parts["self"] + np.where(cf, 0.0, tf) + np.where(cb, 0.0, tb)
            parts[(mu, +1)] = np.where(cf, tf, 0.0)
            parts[(mu, -1)] = np.where(cb, tb, 0.0)
        return parts

    def chirality(self):
        half = self.n // 2
        return np.broadcast_to((np.arange(self.n) >= half).astype(np.int64),
                               (self.lat.V, self.n)).copy()

    def dense(self):
        """Dense (V*N, V*N) matrix, column by column (small lattices only)."""
        n = self.lat.V * self.n
        out = np.empty((n, n), dtype=np.complex128)
        for j in range(n):
            e = np.zeros(n, dtype=np.complex128)
            e[j] = 1.0
            out[:, j] = self.apply(e.reshape(self.lat.V, self.n)).ravel()
        return out


def block_preconditioned(S: CoarseStencil) -> CoarseStencil:
    """X^{-1} A_hat as a 9-point stencil (Sec. 2.3, the block-preconditioned
    coarse operator): identity self blocks, hops X(x)^{-1} Y_{+-mu}(x)."""
    xinv = np.linalg.inv(S.X)
    eye = np.broadcast_to(np.eye(S.n, dtype=np.complex128), S.X.shape).copy()
    Yf = np.einsum("xij,mxjk->mxik", xinv, S.Yf)
    Yb = np.einsum("xij,mxjk->mxik", xinv, S.Yb)
    return CoarseStencil(S.lat, eye, Yf, Yb)


def near_null_vectors(op, phi0, tol=1e-6, maxiter=2000):
    """CGNE on op.apply(phi) = 0 from each start phi0[k] (Table 1, Sec. 2.1).

    Returns (vectors, iteration counts)."""
    vecs, its = [], []
    zero = np.zeros_like(phi0[0], dtype=np.complex128)
    for k in range(phi0.shape[0]):
        x, it, _ = cgne(op.apply, op.apply_dag, zero, phi0[k], tol, maxiter)
        vecs.append(x)
        its.append(it)
    return np.stack(vecs), its


def block_rows(lat: Lattice, n: int, chi, agg):
    """(V_c, 2, rows) flat indices into a (V, n) field: the components of each
    aggregate with chirality 0 and 1, in (position in aggregate, component) order."""
    aidx, apos = lat.aggregate(agg)
    Vc = int(aidx.max()) + 1
    order = np.lexsort((apos, aidx))                 # sites by (aggregate, position)
    flat = (order[:, None] * n + np.arange(n)[None, :])          # (V, n) flat index
    chis = chi[order]                                             # (V, n)
    per_agg = lat.V // Vc
    flat = flat.reshape(Vc, per_agg * n)
    chis = chis.reshape(Vc, per_agg * n)
    rows0 = [f[c == 0] for f, c in zip(flat, chis)]
    rows1 = [f[c == 1] for f, c in zip(flat, chis)]
    return np.stack([np.stack(rows0), np.stack(rows1)], axis=1)


def block_orthonormalize(vecs, rows):
    """Modified Gram-Schmidt, in vector order, twice, inside every
    (aggregate, chirality) block.  vecs: (n_vec, V, n); returns the same shape
    with each chirality projection orthonormal on each aggregate."""
    nvec = vecs.shape[0]
    flat = vecs.reshape(nvec, -1)
    Q = flat[:, rows].transpose(1, 2, 3, 0).copy()    # (Vc, 2, rows, nvec)
    for _ in range(2):
        for k in range(nvec):
            for j in range(k):
                c = np.einsum("abr,abr->ab", np.conj(Q[..., j]), Q[..., k])
                Q[..., k] -= c[..., None] * Q[..., j]
            nrm = np.sqrt(np.einsum("abr,abr->ab", np.conj(Q[..., k]), Q[..., k]).real)
            Q[..., k] /= nrm[..., None]
    out = np.zeros_like(flat)
    for k in range(nvec):
        out[k, rows] = Q[..., k]
    return out.reshape(vecs.shape)


class Transfer:
    """Restriction R and prolongation P = R^dag between a level and its coarsening."""

    def __init__(self, lat: Lattice, n: int, chi, agg, vecs):
        self.lat = lat
        self.n = n
        self.agg = tuple(int(a) for a in agg)
        self.chi = chi
        self.nvec = vecs.shape[0]
        self.rows = block_rows(lat, n, chi, agg)
        self.P = block_orthonormalize(vecs, self.rows)    # (nvec, V, n)
        self.aidx, _ = lat.aggregate(agg)
        self.coarse_lat = Lattice(lat.coarse_dims(agg))
        self.N = 2 * self.nvec

    def restrict(self, v):
        """r_hat(X, s, k) = sum over (x, d) in X with chirality s of conj(P_k(x,d)) v(x,d)."""
        Vc = self.coarse_lat.V
        out = np.zeros((Vc, 2, self.nvec), dtype=np.complex128)
        prod = np.conj(self.P) * v[None]                 # (nvec, V, n)
        for s in (0, 1):
            contrib = np.where((self.chi == s)[None], prod, 0.0).sum(axis=2)   # (nvec, V)
            for k in range(self.nvec):
                out[:, s, k] = np.bincount(self.aidx, weights=contrib[k].real, minlength=Vc) \
                    + 1j * np.bincount(self.aidx, weights=contrib[k].imag, minlength=Vc)
        return out.reshape(Vc, self.N)

    def prolong(self, vc):
        """e(x, d) = sum_k P_k(x, d) v_hat(X(x), chirality(x, d), k)."""
        vc = vc.reshape(-1, 2, self.nvec)
        coeff = vc[self.aidx[:, None], self.chi, :]      # (V, n, nvec)
        return np.einsum("kxd,xdk->xd", self.P, coeff)


def galerkin(op, T: Transfer):
    """A_hat = R A P as a 9-point stencil, one coarse column j at a time.

    Column j of P on every aggregate at once is P e_j (e_j = 1 at component j
    of every coarse site).  Applying the operator split by aggregate crossing
    and restricting gives column j of X (self part) and of Y_{+-mu} (crossing
    parts): the +mu part seen at aggregate X only reads aggregate X + mu.
    """
    Vc, N = T.coarse_lat.V, T.N
    X = np.zeros((Vc, N, N), dtype=np.complex128)
    Yf = np.zeros((4, Vc, N, N), dtype=np.complex128)
    Yb = np.zeros((4, Vc, N, N), dtype=np.complex128)
    for j in range(N):
        e = np.zeros((Vc, N), dtype=np.complex128)
        e[:, j] = 1.0
        parts = op.apply_parts(T.prolong(e), T.agg)
        X[:, :, j] = T.restrict(parts["self"])
        for mu in range(4):
            Yf[mu][:, :, j] = T.restrict(parts[(mu, +1)])
            Yb[mu][:, :, j] = T.restrict(parts[(mu, -1)])
    return CoarseStencil(T.coarse_lat, X, Yf, Yb)
