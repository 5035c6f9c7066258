"""Pins of the oracle's near-null setup, transfer operators and Galerkin stencil.

Checks against: numpy's QR (block orthonormalisation is the unique thin QR
with a positive diagonal), adjointness R = P^dag, exact chirality of P,
the matrix-free definition A_hat v = R A P v, a dense brute-force product
P^dag A P on tiny lattices, Gamma-Hermiticity of the coarsened M (Sec. 2.1)
and gauge invariance of A_hat.
"""
import numpy as np
import pytest

from oracle.coarse import (CoarseStencil, FineLevelOp, Transfer, block_orthonormalize,
                           block_rows, galerkin, near_null_vectors)
from oracle.dirac import KahlerDirac, Staggered, gauge_transform_links
from oracle.lattice import Lattice
from paper_2212_12559_gb300 import inputs


def make_op(dims, hisq, mass, seed=31):
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, seed)
    if hisq:
        return Staggered(lat, inputs.fat_links(thin, dims), inputs.naik_links(thin, dims),
                         -1 / 24, mass)
    return Staggered(lat, thin, None, 0.0, mass)


class MLevel:
    """M itself as a level operator (for Gamma-Hermiticity of the coarse M)."""

    def __init__(self, op):
        self.op, self.lat, self.n = op, op.lat, 3

    def apply(self, v):
        return self.op.M(v)

    def apply_parts(self, v, agg):
        return self.op.M_parts(v, agg)

    def chirality(self):
        return np.repeat(self.lat.parity()[:, None], 3, axis=1)


def test_block_orthonormalize_is_qr():
    dims = (8, 4, 4, 4)
    lat = Lattice(dims)
    nvec = 5
    vecs = inputs.gaussian_fields(nvec, lat.V, 3, 17)
    chi = np.repeat(lat.parity()[:, None], 3, axis=1)
    rows = block_rows(lat, 3, chi, (4, 4, 4, 4))
    assert rows.shape == (2, 2, 384)
    P = block_orthonormalize(vecs, rows)
    flat_v, flat_p = vecs.reshape(nvec, -1), P.reshape(nvec, -1)
    for X in range(2):
        for s in range(2):
            A = flat_v[:, rows[X, s]].T
            Q, R = np.linalg.qr(A)
            Q = Q * (np.sign(np.diag(R).real))[None, :]
            got = flat_p[:, rows[X, s]].T
            assert np.allclose(got, Q, atol=1e-12)
            assert np.allclose(got.conj().T @ got, np.eye(nvec), atol=1e-12)


@pytest.mark.parametrize("dims,agg", [((8, 4, 4, 4), (4, 4, 4, 4)), ((8, 8, 4, 4), (4, 4, 2, 2))])
def test_transfer_chirality_and_adjoint(dims, agg):
    lat = Lattice(dims)
    nvec = 4
    chi = np.repeat(lat.parity()[:, None], 3, axis=1)
    vecs = inputs.gaussian_fields(nvec, lat.V, 3, 23)
    T = Transfer(lat, 3, chi, agg, vecs)
    Vc = T.coarse_lat.V
    v = inputs.gaussian_field(lat.V, 3, 1)
    w = inputs.gaussian_fields(1, Vc, T.N, 2)[0]
    assert np.isclose(np.vdot(T.restrict(v), w), np.vdot(v, T.prolong(w)), rtol=1e-12)
    # eps P = P Gamma
    gamma = np.where(np.arange(T.N) < nvec, 1.0, -1.0)
    eps = lat.eps()[:, None]
    assert np.allclose(eps * T.prolong(w), T.prolong(w * gamma[None, :]), atol=1e-13)
    # R P = 1 and P R is the projector onto the chirally split vectors
    assert np.allclose(T.restrict(T.prolong(w)), w, atol=1e-12)
    for k in range(nvec):
        for s in (0, 1):
            vk = np.where(chi == s, vecs[k], 0.0)
            assert np.allclose(T.prolong(T.restrict(vk)), vk, atol=1e-11)


@pytest.mark.parametrize("dims,hisq", [((8, 8, 8, 8), False), ((8, 4, 4, 4), True),
                                       ((12, 8, 4, 8), True)])
def test_galerkin_stencil_equals_RAP(dims, hisq):
    """Coarse extents 3, 2 and 1 (folded +-mu neighbours) along different axes."""
    op = make_op(dims, hisq, 0.1)
    kd = KahlerDirac(op)
    lop = FineLevelOp(kd)
    nvec = 3
    vecs = inputs.gaussian_fields(nvec, op.lat.V, 3, 41)
    T = Transfer(op.lat, 3, lop.chirality(), (4, 4, 4, 4), vecs)
    S = galerkin(lop, T)
    v = inputs.gaussian_fields(1, T.coarse_lat.V, T.N, 3)[0]
    assert np.allclose(S.apply(v), T.restrict(kd.A(T.prolong(v))), atol=1e-12)
    u = inputs.gaussian_fields(1, T.coarse_lat.V, T.N, 4)[0]
    assert np.isclose(np.vdot(u, S.apply(v)), np.vdot(S.apply_dag(u), v), rtol=1e-12)
    parts = S.apply_parts(v, (1, 1, 1, 1))
    assert np.allclose(sum(parts.values()), S.apply(v), atol=1e-13)


def test_galerkin_dense_brute_force():
    """Naive operator, 4^4 lattice, 2^4 aggregates: dense P^dag A P."""
    dims = (4, 4, 4, 4)
    op = make_op(dims, False, 0.2)
    kd = KahlerDirac(op)
    lop = FineLevelOp(kd)
    nvec = 2
    T = Transfer(op.lat, 3, lop.chirality(), (2, 2, 2, 2), inputs.gaussian_fields(nvec, op.lat.V, 3, 5))
    S = galerkin(lop, T)
    n = 3 * op.lat.V
    nc = T.coarse_lat.V * T.N
    Pm = np.empty((n, nc), dtype=np.complex128)
    for j in range(nc):
        e = np.zeros(nc, dtype=np.complex128); e[j] = 1
        Pm[:, j] = T.prolong(e.reshape(-1, T.N)).ravel()
    Am = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128); e[j] = 1
        Am[:, j] = kd.A(e.reshape(-1, 3)).ravel()
    assert np.allclose(Pm.conj().T @ Pm, np.eye(nc), atol=1e-12)
    assert np.allclose(S.dense(), Pm.conj().T @ Am @ Pm, atol=1e-12)


def test_coarse_M_gamma_hermitian():
    """Coarsening M with chirally split P gives Gamma M_hat Gamma = M_hat^dag (Sec. 2.1)."""
    op = make_op((8, 4, 4, 4), True, 0.07)
    lev = MLevel(op)
    nvec = 3
    T = Transfer(op.lat, 3, lev.chirality(), (4, 4, 4, 4), inputs.gaussian_fields(nvec, op.lat.V, 3, 9))
    S = galerkin(lev, T)
    Md = S.dense()
    g = np.tile(np.where(np.arange(T.N) < nvec, 1.0, -1.0), T.coarse_lat.V)
    assert np.allclose(g[:, None] * Md * g[None, :], Md.conj().T, atol=1e-12)


def test_galerkin_gauge_invariant():
    dims = (8, 4, 4, 4)
    op = make_op(dims, True, 0.1)
    lat = op.lat
    g = inputs.random_su3_field(dims, 77)
    op_g = Staggered(lat, gauge_transform_links(lat, op.fat, g, 1),
                     gauge_transform_links(lat, op.naik, g, 3), op.c_naik, op.mass)
    vecs = inputs.gaussian_fields(3, lat.V, 3, 8)
    vecs_g = np.einsum("xab,kxb->kxa", g, vecs)
    chi = np.repeat(lat.parity()[:, None], 3, axis=1)
    S = galerkin(FineLevelOp(KahlerDirac(op)), Transfer(lat, 3, chi, (4, 4, 4, 4), vecs))
    Sg = galerkin(FineLevelOp(KahlerDirac(op_g)), Transfer(lat, 3, chi, (4, 4, 4, 4), vecs_g))
    assert np.allclose(S.X, Sg.X, atol=1e-11)
    assert np.allclose(S.Yf, Sg.Yf, atol=1e-11)
    assert np.allclose(S.Yb, Sg.Yb, atol=1e-11)


def test_coarse_of_coarse_stencil():
    """Second coarsening (2^4 aggregates of a coarse stencil) is again R A_hat P."""
    op = make_op((8, 8, 8, 8), False, 0.1)
    lop = FineLevelOp(KahlerDirac(op))
    T1 = Transfer(op.lat, 3, lop.chirality(), (4, 4, 4, 4), inputs.gaussian_fields(3, op.lat.V, 3, 1))
    S1 = galerkin(lop, T1)
    T2 = Transfer(S1.lat, S1.n, S1.chirality(), (2, 2, 2, 2),
                  inputs.gaussian_fields(2, S1.lat.V, S1.n, 2))
    S2 = galerkin(S1, T2)
    v = inputs.gaussian_fields(1, 1, T2.N, 3)[0]
    assert S2.lat.V == 1
    assert np.allclose(S2.apply(v), T2.restrict(S1.apply(T2.prolong(v))), atol=1e-12)


def test_near_null_vectors_are_low_modes():
    """Inverse iteration lowers the Rayleigh quotient ||A v|| / ||v|| of the start."""
    op = make_op((4, 4, 4, 4), False, 0.05)
    kd = KahlerDirac(op)
    lop = FineLevelOp(kd)
    phi0 = inputs.gaussian_fields(2, op.lat.V, 3, 12)
    vecs, its = near_null_vectors(lop, phi0, tol=1e-6, maxiter=300)
    for k in range(2):
        r0 = np.linalg.norm(kd.A(phi0[k])) / np.linalg.norm(phi0[k])
        r1 = np.linalg.norm(kd.A(vecs[k])) / np.linalg.norm(vecs[k])
        assert r1 < 0.5 * r0
