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
