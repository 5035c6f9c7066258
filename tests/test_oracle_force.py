"""Pins of the oracle's fermion action derivative: central finite
differences along random su(3) directions and in the mass, and the closed
form dS/dm = -2 m ||X||^2."""
import numpy as np
import pytest
import scipy.linalg

from oracle.dirac import Staggered
from oracle.force import action_vectors, link_gradient, mass_gradient
from oracle.lattice import Lattice
from paper_2212_12559_gb300 import inputs


def dense_solver(op):
    n = 3 * op.lat.V
    Mm = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128); e[j] = 1
        Mm[:, j] = op.M(e.reshape(-1, 3)).ravel()
    lu = scipy.linalg.lu_factor(Mm)
    return lambda b: scipy.linalg.lu_solve(lu, b.ravel()).reshape(b.shape)


def expm_i(eps, T):
    w, q = np.linalg.eigh(T)
    return (q * np.exp(1j * eps * w)[..., None, :]) @ np.conj(np.swapaxes(q, -1, -2))


@pytest.mark.parametrize("hisq", [False, True])
def test_force_finite_differences(hisq):
    dims = (4, 4, 4, 4)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 1005)
    fat = inputs.fat_links(thin, dims) if hisq else thin
    naik = inputs.naik_links(thin, dims) if hisq else None
    c = -1 / 24 if hisq else 0.0
    m = 0.2
    phi = inputs.gaussian_field(lat.V, 3, 2005)
    op = Staggered(lat, fat, naik, c, m)
    S, X, Y = action_vectors(op, dense_solver(op), phi)
    assert np.isclose(S, np.vdot(Y, Y).real, rtol=1e-12)
    G = link_gradient(op, X, Y)
    GN = link_gradient(op, X, Y, naik=True) if hisq else None
    Ts = inputs.lie_directions(3, lat.V, 4005)
    h = 1e-4
    for T in Ts:
        def S_at(e, which):
            f = expm_i(e, T) @ fat if which == "fat" else fat
            nk = (expm_i(e, T) @ naik if which == "naik" else naik) if hisq else None
            o = Staggered(lat, f, nk, c, m)
            return action_vectors(o, dense_solver(o), phi)[0]
        for which, grad in (("fat", G), ("naik", GN)):
            if grad is None:
                continue
            fd = (S_at(h, which) - S_at(-h, which)) / (2 * h)
            dU = 1j * T @ (fat if which == "fat" else naik)
            an = np.sum((np.conj(grad) * dU).real)
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
    dm = 1e-5
    Sp = action_vectors(Staggered(lat, fat, naik, c, m + dm), dense_solver(Staggered(lat, fat, naik, c, m + dm)), phi)[0]
    Sm = action_vectors(Staggered(lat, fat, naik, c, m - dm), dense_solver(Staggered(lat, fat, naik, c, m - dm)), phi)[0]
    assert np.isclose((Sp - Sm) / (2 * dm), mass_gradient(op, X), rtol=1e-6)
