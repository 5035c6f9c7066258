"""Pins of the oracle's coarse-level solver forms of Table 1 (levels 2 and 3):
the block-preconditioned and Schur (even/odd) coarse operators, the
Chebyshev-basis CA-GCR and the SVD-deflated coarsest solve.

* X^{-1} A_hat applied matrix-free equals the dense product; its even-even
  and odd-odd blocks are identities (every coarse hop changes parity).
* The matrix-free Schur operator equals 1 - A'_eo A'_oe built from the dense
  blocks, and the Schur solve with reconstruction reproduces the dense
  solution of A_hat x = b.
* The Chebyshev basis vectors equal T_k((A - c)/h) r evaluated from the
  polynomials' power-series coefficients (numpy.polynomial), not the
  recurrence; Chebyshev-basis CA-GCR(s) spans K_s(A, r): its residual equals
  the minimum over an Arnoldi basis, and for small s the power-basis result.
* The deflated start leaves no residual along the deflated left singular
  vectors (exact identity), is the exact solution when every triplet is
  deflated, and the deflated GCR reaches the dense solution.
"""
import numpy as np
import pytest

from oracle.coarse import FineLevelOp, Transfer, galerkin
from oracle.dirac import KahlerDirac, Staggered
from oracle.lattice import Lattice
from oracle.schur import SchurCoarse
from oracle.solvers import (ca_gcr, ca_gcr_basis, ca_gcr_chebyshev, chebyshev_basis, gcr,
                            lowest_singular_triplets, shifted_power_basis, svd_deflated_gcr)
from paper_2212_12559_gb300 import inputs


@pytest.fixture(scope="module")
def coarse():
    """Galerkin operator of an 8^4 HISQ-shaped KD operator on 4^4 aggregates
    (coarse lattice 2^4, N = 8)."""
    dims = (8, 8, 8, 8)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 41)
    op = Staggered(lat, inputs.fat_links(thin, dims), inputs.naik_links(thin, dims), -1 / 24, 0.1)
    lop = FineLevelOp(KahlerDirac(op))
    T = Transfer(lat, 3, lop.chirality(), (4, 4, 4, 4), inputs.gaussian_fields(4, lat.V, 3, 42))
    S = galerkin(lop, T)
    return S, S.dense()


def test_block_preconditioned_operator(coarse):
    S, Ad = coarse
    sc = SchurCoarse(S)
    V, N = S.lat.V, S.n
    Xd = np.zeros_like(Ad)
    for x in range(V):
        Xd[x * N:(x + 1) * N, x * N:(x + 1) * N] = S.X[x]
    Bd = np.linalg.solve(Xd, Ad)                         # X^{-1} A_hat, dense
    v = inputs.gaussian_field(V, N, 43)
    np.testing.assert_allclose(sc.block_apply(v).ravel(), Bd @ v.ravel(), rtol=0, atol=1e-11 * np.abs(Bd).max())
    ev = np.concatenate([np.arange(x * N, (x + 1) * N) for x in sc.even])
    od = np.concatenate([np.arange(x * N, (x + 1) * N) for x in sc.odd])
    assert np.allclose(Bd[np.ix_(ev, ev)], np.eye(len(ev)), atol=1e-12)
    assert np.allclose(Bd[np.ix_(od, od)], np.eye(len(od)), atol=1e-12)


def test_schur_operator_and_solve(coarse):
    S, Ad = coarse
    sc = SchurCoarse(S)
    V, N = S.lat.V, S.n
    Xd = np.zeros_like(Ad)
    for x in range(V):
        Xd[x * N:(x + 1) * N, x * N:(x + 1) * N] = S.X[x]
    Bd = np.linalg.solve(Xd, Ad)
    ev = np.concatenate([np.arange(x * N, (x + 1) * N) for x in sc.even])
    od = np.concatenate([np.arange(x * N, (x + 1) * N) for x in sc.odd])
    Sd = np.eye(len(ev)) - Bd[np.ix_(ev, od)] @ Bd[np.ix_(od, ev)]
    ve = inputs.gaussian_field(len(sc.even), N, 44)
    np.testing.assert_allclose(sc.schur_apply(ve).ravel(), Sd @ ve.ravel(), rtol=0,
                               atol=1e-11 * np.abs(Sd).max())
    b = inputs.gaussian_field(V, N, 45)
    x = sc.solve(b, lambda apply, rhs: np.linalg.solve(Sd, rhs.ravel()).reshape(rhs.shape))
    xs = np.linalg.solve(Ad, b.ravel())
    assert np.linalg.norm(x.ravel() - xs) <= 1e-10 * np.linalg.norm(xs)
    # the same through GCR on the Schur system (matrix-free)
    x2 = sc.solve(b, lambda apply, rhs: gcr(apply, rhs, tol=1e-12, maxiter=400, nkrylov=64)[0])
    assert np.linalg.norm(x2.ravel() - xs) <= 1e-8 * np.linalg.norm(xs)


def arnoldi_min_residual(Am, r, s):
    Q = np.zeros((r.size, s), dtype=np.complex128)
    Q[:, 0] = r / np.linalg.norm(r)
    for j in range(1, s):
        w = Am @ Q[:, j - 1]
        for i in range(j):
            w -= np.vdot(Q[:, i], w) * Q[:, i]
        Q[:, j] = w / np.linalg.norm(w)
    y, *_ = np.linalg.lstsq(Am @ Q, r, rcond=None)
    return np.linalg.norm(r - Am @ (Q @ y))


@pytest.mark.parametrize("s", [3, 6, 10])
def test_chebyshev_ca_gcr_is_krylov_min_residual(coarse, s):
    S, Ad = coarse
    r = inputs.gaussian_field(S.lat.V, S.n, 46)
    ev = np.linalg.eigvals(Ad)
    lmin, lmax = float(ev.real.min()), float(ev.real.max())
    apply = lambda v: (Ad @ v.ravel()).reshape(v.shape)
    e = ca_gcr_chebyshev(apply, r, s, lmin, lmax).ravel()
    got = np.linalg.norm(r.ravel() - Ad @ e)
    best = arnoldi_min_residual(Ad, r.ravel(), s)
    assert abs(got - best) <= 1e-9 * np.linalg.norm(r)
    if s <= 6:
        e_pow = ca_gcr(apply, r, s).ravel()
        assert np.linalg.norm(e - e_pow) <= 1e-7 * np.linalg.norm(e_pow)


def test_svd_deflation(coarse):
    S, Ad = coarse
    n = Ad.shape[0]
    b = inputs.gaussian_field(S.lat.V, S.n, 47)
    U, sig, V = lowest_singular_triplets(Ad, 16)
    assert np.all(np.diff(sig) >= 0)
    np.testing.assert_allclose(Ad @ V, U * sig, rtol=0, atol=1e-11 * np.abs(Ad).max())
    x0 = (V @ ((U.conj().T @ b.ravel()) / sig))
    r0 = b.ravel() - Ad @ x0
    assert np.linalg.norm(U.conj().T @ r0) <= 1e-11 * np.linalg.norm(b)
    Uall, sall, Vall = lowest_singular_triplets(Ad, n)
    xfull = Vall @ ((Uall.conj().T @ b.ravel()) / sall)
    xs = np.linalg.solve(Ad, b.ravel())
    assert np.linalg.norm(xfull - xs) <= 1e-10 * np.linalg.norm(xs)
    apply = lambda v: (Ad @ v.ravel()).reshape(v.shape)
    x, it, res = svd_deflated_gcr(apply, b, U, sig, V, tol=1e-11, maxiter=500, nkrylov=64)
    assert res <= 1e-11
    assert np.linalg.norm(x.ravel() - xs) <= 1e-8 * np.linalg.norm(xs)
    _, it_plain, _ = gcr(apply, b, tol=1e-11, maxiter=500, nkrylov=64)
    assert it <= it_plain


def test_chebyshev_ca_gcr_interval_only_conditions(coarse):
    """The Chebyshev interval changes the basis, not the space: two intervals
    (the exact [sigma_k, sigma_max] and a perturbed one) give the same
    minimum-residual correction."""
    S, Ad = coarse
    r = inputs.gaussian_field(S.lat.V, S.n, 50)
    sv = np.linalg.svd(Ad, compute_uv=False)
    apply = lambda v: (Ad @ v.ravel()).reshape(v.shape)
    e1 = ca_gcr_chebyshev(apply, r, 5, float(np.sort(sv)[3]), float(sv.max()))
    e2 = ca_gcr_chebyshev(apply, r, 5, 0.7 * float(np.sort(sv)[3]), 1.1 * float(sv.max()))
    assert np.linalg.norm(e1 - e2) <= 1e-9 * np.linalg.norm(e1)


def test_chebyshev_basis_is_chebyshev_polynomials(coarse):
    from numpy.polynomial import chebyshev as C
    S, Ad = coarse
    r = inputs.gaussian_field(S.lat.V, S.n, 48).ravel()
    lmin, lmax = 0.05, 3.0
    c, h = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    T = (Ad - c * np.eye(Ad.shape[0])) / h
    Q = chebyshev_basis(lambda v: (Ad @ v.ravel()).reshape(v.shape), r, 7, lmin, lmax)
    for k, q in enumerate(Q):
        coef = C.cheb2poly([0] * k + [1])          # T_k as a power series
        ref = np.zeros_like(r)
        Tp = r.copy()
        for a in coef:
            ref += a * Tp
            Tp = T @ Tp
        assert np.linalg.norm(q - ref) <= 1e-9 * max(1.0, np.linalg.norm(ref))


def test_block_preconditioned_stencil(coarse):
    """block_preconditioned(S) is the stencil of X^{-1} A_hat: identity self
    blocks, and it applies like the matrix-free block-preconditioned operator."""
    from oracle.coarse import block_preconditioned
    S, _ = coarse
    B = block_preconditioned(S)
    assert np.allclose(B.X, np.eye(S.n)[None], atol=1e-13)
    v = inputs.gaussian_field(S.lat.V, S.n, 49)
    np.testing.assert_allclose(B.apply(v), SchurCoarse(S).block_apply(v), rtol=0, atol=1e-11)


def test_block_coarse_three_level_solve():
    """Sec. 2.3's coarsening of X^{-1} A_hat (near-null vectors from A_hat)
    inside the K-cycle: the outer solve still reaches 1e-10 on M."""
    from oracle.mg import MGParams, MultigridSolver
    dims = (8, 8, 8, 8)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 1002)
    op = Staggered(lat, inputs.fat_links(thin, dims), inputs.naik_links(thin, dims), -1 / 24, 0.05)
    p = MGParams(agg=[(4, 4, 4, 4), (2, 2, 2, 2)], nvec=[4, 4], setup_maxiter=40, block_coarse=True)
    phi0 = [inputs.gaussian_fields(4, lat.V, 3, 3002), inputs.gaussian_fields(4, 16, 8, 3003)]
    mg = MultigridSolver(op, p, phi0)
    assert np.allclose(mg.levels[1].X, np.eye(8)[None], atol=1e-12)
    b = inputs.gaussian_field(lat.V, 3, 2002)
    x, it, res = mg.solve(b, tol=1e-10)
    assert res <= 1e-10
    assert np.linalg.norm(b - op.M(x)) <= 1e-10 * np.linalg.norm(b)


def test_deflated_coarsest_in_kcycle():
    """Table 1's coarsest solver inside the K-cycle (two levels, coarsest not
    dense): the outer solve reaches 1e-10 on M, and one coarsest solve meets
    the level's 0.25 rule or uses at most inner_maxiter CA-GCR steps."""
    from oracle.mg import MGParams, MultigridSolver
    from oracle.solvers import norm
    dims = (8, 8, 4, 4)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 1003)
    op = Staggered(lat, thin, None, 0.0, 0.1)
    p = MGParams(agg=[(4, 4, 4, 4)], nvec=[4], setup_maxiter=50, dense_max=0, coarsest_deflate=8,
                 coarsest_cheb_s=8)
    mg = MultigridSolver(op, p, [inputs.gaussian_fields(4, lat.V, 3, 3004)])
    assert mg.dense_lu is None and mg.defl is not None
    rc = inputs.gaussian_field(mg.levels[-1].lat.V, mg.levels[-1].n, 5)
    x = mg.deflated_coarsest(mg.levels[-1], rc)
    assert norm(rc - mg.levels[-1].apply(x)) < norm(rc)
    b = inputs.gaussian_field(lat.V, 3, 2003)
    xs, it, res = mg.solve(b, tol=1e-10)
    assert res <= 1e-10


def test_schur_deflated_coarsest_in_kcycle():
    """Table 1's level-3 form: the deflated Chebyshev-basis CA-GCR on the
    even/odd Schur complement of the block-preconditioned coarsest operator.
    One coarsest solve equals the Schur solve of the same deflated iteration
    done by hand, with all of S's triplets deflated it is the exact solution,
    and the outer solve reaches 1e-10 on M."""
    from oracle.mg import MGParams, MultigridSolver
    dims = (8, 8, 8, 8)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 1004)
    op = Staggered(lat, thin, None, 0.0, 0.1)
    kw = dict(agg=[(4, 4, 4, 4)], nvec=[4], setup_maxiter=30, dense_max=0, block_coarse=True,
              coarsest_deflate=8, coarsest_cheb_s=4)
    phi = [inputs.gaussian_fields(4, lat.V, 3, 3007)]
    mg = MultigridSolver(op, MGParams(coarsest_schur=True, **kw), phi)
    lev = mg.levels[-1]
    assert mg.schur is not None and mg.defl[0].shape == (len(mg.schur.even) * lev.n, 8)
    rc = inputs.gaussian_field(lev.lat.V, lev.n, 8)
    x = mg.coarse_solve(2, rc)
    rcx = np.einsum("xij,xj->xi", mg.xinv[-1], rc)   # block mode: the level solves X^{-1} A_hat x = X^{-1} rc
    sc = SchurCoarse(lev)
    rhs, c = sc.schur_rhs(rcx)
    xe = mg.deflated_coarsest_op(sc.schur_apply, rhs)
    assert np.linalg.norm(x - sc.reconstruct(xe, c)) <= 1e-13 * np.linalg.norm(x)
    Sd = mg.schur_dense()
    Ad = lev.dense()
    Ue, se, Ve = lowest_singular_triplets(Sd, Sd.shape[0])
    xe_full = (Ve @ ((Ue.conj().T @ rhs.ravel()) / se)).reshape(rhs.shape)
    xs = np.linalg.solve(Ad, rcx.ravel())
    assert np.linalg.norm(sc.reconstruct(xe_full, c).ravel() - xs) <= 1e-10 * np.linalg.norm(xs)
    b = inputs.gaussian_field(lat.V, 3, 2004)
    _, it, res = mg.solve(b, tol=1e-10)
    assert res <= 1e-10


def test_schur_level2_in_kcycle():
    """Table 1's level 2 in Schur form (GCR on S = 1 - K_eo K_oe preconditioned
    by the K-cycle on the embedded residual (r_e, 0)) inside the three-level
    K-cycle: the outer solve reaches 1e-10 on M, and one level-2 solve is an
    exact solution of the level's full system when the inner tolerance is
    tight (the reconstruction x_o = c_o - K_oe x_e closes the odd rows)."""
    from oracle.mg import MGParams, MultigridSolver
    dims = (8, 8, 8, 8)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 1005)
    op = Staggered(lat, thin, None, 0.0, 0.1)
    phi = [inputs.gaussian_fields(4, lat.V, 3, 3010), inputs.gaussian_fields(4, 16, 8, 3011)]
    kw = dict(agg=[(4, 4, 4, 4), (2, 2, 2, 2)], nvec=[4, 4], setup_maxiter=30, block_coarse=True,
              schur_coarse=True)
    mg = MultigridSolver(op, MGParams(inner_tol=1e-12, inner_maxiter=60, **kw), phi)
    lev = mg.levels[1]
    rc = inputs.gaussian_field(lev.lat.V, lev.n, 12)
    x = mg.coarse_solve(2, rc)
    rcx = np.einsum("xij,xj->xi", mg.xinv[1], rc)
    assert np.linalg.norm(rcx - lev.apply(x)) <= 1e-10 * np.linalg.norm(rcx)
    mg = MultigridSolver(op, MGParams(**kw), phi)
    b = inputs.gaussian_field(lat.V, 3, 2006)
    _, it, res = mg.solve(b, tol=1e-10)
    assert res <= 1e-10


def test_schur_spectrum_closed_form(coarse):
    """Independent of the Schur code's own formulas: for the bipartite
    A' = [[1, K_eo], [K_oe, 1]], A' (x_e, x_o) = lam (x_e, x_o) gives
    K_eo K_oe x_e = (lam - 1)^2 x_e, so every eigenvalue mu of
    S = 1 - K_eo K_oe belongs to the pair lam = 1 +- sqrt(1 - mu) of A' (the
    even and odd site counts are equal, so these pairs are all of A's
    spectrum)."""
    S, _ = coarse
    sc = SchurCoarse(S)
    ne, N = len(sc.even), S.n
    Sd = np.empty((ne * N, ne * N), dtype=np.complex128)
    for j in range(ne * N):
        e = np.zeros(ne * N, dtype=np.complex128)
        e[j] = 1.0
        Sd[:, j] = sc.schur_apply(e.reshape(ne, N)).ravel()
    V, n = S.lat.V, S.lat.V * N
    Bd = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        Bd[:, j] = sc.block_apply(e.reshape(V, N)).ravel()
    mu = np.linalg.eigvals(Sd)
    root = np.sqrt(1.0 - mu)
    pred = np.concatenate([1.0 + root, 1.0 - root])
    lam = np.linalg.eigvals(Bd)
    scale = np.abs(lam).max()
    # every predicted value has an eigenvalue of A' next to it, and vice versa
    d1 = np.abs(pred[:, None] - lam[None, :]).min(axis=1)
    d2 = np.abs(lam[:, None] - pred[None, :]).min(axis=1)
    assert d1.max() <= 1e-8 * scale and d2.max() <= 1e-8 * scale


@pytest.mark.parametrize("s", [3, 6, 10])
def test_shifted_power_basis_ca_gcr(coarse, s):
    """The shifted power basis is ((A - c)/h)^k r (matrix powers, not the
    recurrence), and CA-GCR(s) with it reaches the Arnoldi minimum residual
    over K_s(A, r), like the Chebyshev basis."""
    S, Ad = coarse
    r = inputs.gaussian_field(S.lat.V, S.n, 51)
    lmin, lmax = 0.05, 3.0
    c, h = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    apply = lambda v: (Ad @ v.ravel()).reshape(v.shape)
    Q = shifted_power_basis(apply, r, s, lmin, lmax)
    T = (Ad - c * np.eye(Ad.shape[0])) / h
    for k, q in enumerate(Q):
        ref = np.linalg.matrix_power(T, k) @ r.ravel()
        assert np.linalg.norm(q.ravel() - ref) <= 1e-10 * np.linalg.norm(ref)
    e = ca_gcr_basis(apply, r, s, lmin, lmax, "shifted").ravel()
    got = np.linalg.norm(r.ravel() - Ad @ e)
    assert abs(got - arnoldi_min_residual(Ad, r.ravel(), s)) <= 1e-9 * np.linalg.norm(r)
