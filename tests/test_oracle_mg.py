"""Pins of the oracle's K-cycle multigrid solve: the recomputed residual
meets the paper's 1e-10 on the full operator (Sec. 3.2), and the solution
matches a dense LU solve within the bound ||x - x*|| <= tol * cond(M) ||x*||."""
import numpy as np
import pytest
import scipy.linalg

from oracle.dirac import Staggered
from oracle.lattice import Lattice
from oracle.mg import MGParams, MultigridSolver
from paper_2212_12559_gb300 import inputs


def dense_M(op):
    n = 3 * op.lat.V
    out = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128); e[j] = 1
        out[:, j] = op.M(e.reshape(-1, 3)).ravel()
    return out


@pytest.mark.parametrize("hisq", [False, True])
def test_two_level_solve_matches_dense(hisq):
    dims = (8, 4, 4, 4)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 1001)
    if hisq:
        op = Staggered(lat, inputs.fat_links(thin, dims), inputs.naik_links(thin, dims), -1 / 24, 0.1)
    else:
        op = Staggered(lat, thin, None, 0.0, 0.1)
    p = MGParams(agg=[(4, 4, 4, 4)], nvec=[4], setup_maxiter=50)
    phi0 = [inputs.gaussian_fields(4, lat.V, 3, 3001)]
    mg = MultigridSolver(op, p, phi0)
    assert mg.dense_lu is not None
    b = inputs.gaussian_field(lat.V, 3, 2001)
    x, it, res = mg.solve(b, tol=1e-10)
    assert res <= 1e-10
    assert np.linalg.norm(b - op.M(x)) <= 1e-10 * np.linalg.norm(b)
    xs = scipy.linalg.solve(dense_M(op), b.ravel())
    bound = 1e-10 * (op.mass + 4 * (1 + abs(op.c_naik))) / op.mass
    assert np.linalg.norm(x.ravel() - xs) <= bound * np.linalg.norm(xs)


def test_three_level_solve():
    dims = (8, 8, 8, 8)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 1002)
    op = Staggered(lat, inputs.fat_links(thin, dims), inputs.naik_links(thin, dims), -1 / 24, 0.05)
    p = MGParams(agg=[(4, 4, 4, 4), (2, 2, 2, 2)], nvec=[4, 4], setup_maxiter=40)
    phi0 = [inputs.gaussian_fields(4, lat.V, 3, 3002), inputs.gaussian_fields(4, 16, 8, 3003)]
    mg = MultigridSolver(op, p, phi0)
    assert len(mg.levels) == 3 and mg.levels[-1].lat.V == 1
    b = inputs.gaussian_field(lat.V, 3, 2002)
    x, it, res = mg.solve(b, tol=1e-10)
    assert res <= 1e-10
    assert np.linalg.norm(b - op.M(x)) <= 1e-10 * np.linalg.norm(b)


def test_truncated_pseudo_fine_operator():
    """Table 1's truncated level-1 operator (Sec. 3.1): the Naik hops are
    dropped from the pseudo-fine operator only.  (B+m)^{-1} is unchanged
    (the Naik reach of three never stays inside a 2^4 hypercube), A' differs
    from A by exactly (B+m)^{-1} applied to the Naik part of D, and the outer
    solve on the full HISQ M still reaches 1e-10 and the dense solution."""
    from oracle.dirac import KahlerDirac
    dims = (8, 4, 4, 4)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 1011)
    fat, naik = inputs.fat_links(thin, dims), inputs.naik_links(thin, dims)
    op = Staggered(lat, fat, naik, -1 / 24, 0.1)
    op_fat = Staggered(lat, fat, None, 0.0, 0.1)
    kd, kd_fat = KahlerDirac(op), KahlerDirac(op_fat)
    assert np.array_equal(kd.blocks, kd_fat.blocks)
    v = inputs.gaussian_field(lat.V, 3, 7)
    naik_only = Staggered(lat, np.zeros_like(fat), naik, -1 / 24, 0.0)
    np.testing.assert_allclose(kd.A(v) - kd_fat.A(v), kd.apply_inv(naik_only.M(v)), rtol=0, atol=1e-12)
    p = MGParams(agg=[(4, 4, 4, 4)], nvec=[4], setup_maxiter=50, truncate_naik=True)
    mg = MultigridSolver(op, p, [inputs.gaussian_fields(4, lat.V, 3, 3011)])
    w = inputs.gaussian_field(lat.V, 3, 8)
    np.testing.assert_allclose(mg.levels[0].apply(w), kd_fat.A(w), rtol=0, atol=1e-13)
    b = inputs.gaussian_field(lat.V, 3, 2011)
    x, it, res = mg.solve(b, tol=1e-10)
    assert res <= 1e-10
    xs = scipy.linalg.solve(dense_M(op), b.ravel())
    bound = 1e-10 * (op.mass + 4 * (1 + abs(op.c_naik))) / op.mass
    assert np.linalg.norm(x.ravel() - xs) <= bound * np.linalg.norm(xs)
