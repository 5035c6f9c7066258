"""Pins of the oracle's Krylov solvers against dense linear algebra.

* GCR reaches the dense solution (numpy.linalg.solve) to its tolerance.
* CA-GCR(s) returns the minimum-residual correction over K_s(A, r): its
  residual equals that of an explicit least-squares solve over an orthonormal
  basis of the Krylov space (built by Arnoldi, independent of the power basis).
* CGNE (Craig's method) after k steps is the minimum-error iterate over
  x0 + A^dag K_k(A A^dag, r0), and converges to the dense solution.
"""
import numpy as np
import pytest

from oracle.dirac import KahlerDirac, Staggered
from oracle.lattice import Lattice
from oracle.solvers import ca_gcr, cgne, gcr
from paper_2212_12559_gb300 import inputs


@pytest.fixture(scope="module")
def small_system():
    dims = (4, 4, 4, 4)
    lat = Lattice(dims)
    op = Staggered(lat, inputs.random_su3_links(dims, 2), None, 0.0, 0.05)
    kd = KahlerDirac(op)
    n = 3 * lat.V
    Am = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128); e[j] = 1
        Am[:, j] = kd.A(e.reshape(-1, 3)).ravel()
    b = inputs.gaussian_field(lat.V, 3, 3)
    return kd, Am, b


def test_gcr_matches_dense_solve(small_system):
    kd, Am, b = small_system
    x, it, res = gcr(kd.A, b, tol=1e-11, maxiter=2000, nkrylov=400)
    xs = np.linalg.solve(Am, b.ravel())
    assert res <= 1e-11
    assert np.linalg.norm(x.ravel() - xs) <= 1e-8 * np.linalg.norm(xs)
    # preconditioned with an exact inverse: one iteration
    x1, it1, _ = gcr(kd.A, b, precond=lambda r: np.linalg.solve(Am, r.ravel()).reshape(r.shape),
                     tol=1e-11, maxiter=5)
    assert it1 == 1


@pytest.mark.parametrize("s", [1, 4, 8])
def test_ca_gcr_is_krylov_min_residual(small_system, s):
    kd, Am, b = small_system
    r = b.ravel()
    e = ca_gcr(lambda v: (Am @ v.ravel()).reshape(v.shape), b, s).ravel()
    # Arnoldi basis of K_s(A, r)
    Q = np.zeros((r.size, s), dtype=np.complex128)
    Q[:, 0] = r / np.linalg.norm(r)
    for j in range(1, s):
        w = Am @ Q[:, j - 1]
        for i in range(j):
            w -= np.vdot(Q[:, i], w) * Q[:, i]
        Q[:, j] = w / np.linalg.norm(w)
    y, *_ = np.linalg.lstsq(Am @ Q, r, rcond=None)
    best = np.linalg.norm(r - Am @ (Q @ y))
    got = np.linalg.norm(r - Am @ e)
    assert abs(got - best) <= 1e-9 * np.linalg.norm(r)
    assert got < np.linalg.norm(r)


def test_cgne_minimum_error_and_convergence(small_system):
    kd, Am, b = small_system
    x0 = inputs.gaussian_field(kd.lat.V, 3, 11)
    Ad = Am.conj().T
    xs = np.linalg.solve(Am, b.ravel())
    r0 = b.ravel() - Am @ x0.ravel()
    for k in (1, 3, 6):
        x, it, _ = cgne(kd.A, kd.Adag, b, x0, tol=0.0, maxiter=k)
        assert it == k
        # minimum of ||x - x*|| over x0 + A^dag span{(A A^dag)^j r0, j < k}
        K = [Ad @ r0]
        for _ in range(k - 1):
            K.append(Ad @ (Am @ K[-1]))
        K = np.linalg.qr(np.stack(K, axis=1))[0]
        y, *_ = np.linalg.lstsq(K, xs - x0.ravel(), rcond=None)
        best = x0.ravel() + K @ y
        assert np.linalg.norm(x.ravel() - best) <= 1e-8 * np.linalg.norm(xs)
    x, it, rel = cgne(kd.A, kd.Adag, b, x0, tol=1e-10, maxiter=5000)
    assert rel <= 1e-10
    assert np.linalg.norm(x.ravel() - xs) <= 1e-7 * np.linalg.norm(xs)


def test_multishift_cg_against_dense():
    """Every shifted system (A + sigma_i) x_i = b of a random Hermitian
    positive matrix, solved in one Krylov space, equals its dense solution;
    a single shift reduces to plain CG (same check), and the recomputed
    residuals meet the tolerance."""
    from oracle.solvers import multishift_cg
    rng = np.random.default_rng(5)
    n = 80
    X = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    A = X.conj().T @ X / n
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    for shifts in ([0.02, 0.1, 0.5, 2.0, 8.0], [0.3]):
        xs, it, res = multishift_cg(lambda v: A @ v, b, shifts, tol=1e-12)
        for s, x, r in zip(shifts, xs, res):
            xd = np.linalg.solve(A + s * np.eye(n), b)
            assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
            assert r <= 1e-11


def test_staggered_multishift_solves_each_mass():
    """x_i = M(m_i)^dag (D^dag D + m_i^2)^{-1} b solves M(m_i) x_i = b
    (dense solve of each M(m_i) on a small HISQ-shaped lattice)."""
    import scipy.linalg
    from oracle.dirac import Staggered
    from oracle.lattice import Lattice
    from oracle.solvers import staggered_multishift
    from paper_2212_12559_gb300 import inputs
    dims = (4, 4, 4, 4)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 1021)
    op = Staggered(lat, inputs.fat_links(thin, dims), inputs.naik_links(thin, dims), -1 / 24, 0.0)
    b = inputs.gaussian_field(lat.V, 3, 2021)
    masses = [0.05, 0.1, 0.3, 0.8]
    xs, it, res = staggered_multishift(op, b, masses, tol=1e-11)
    n = 3 * lat.V
    Dm = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128); e[j] = 1
        Dm[:, j] = op.D(e.reshape(-1, 3)).ravel()
    for m, x, r in zip(masses, xs, res):
        xd = scipy.linalg.solve(m * np.eye(n) + Dm, b.ravel())
        assert r <= 1e-10
        assert np.linalg.norm(x.ravel() - xd) <= 1e-9 / m * np.linalg.norm(xd)
