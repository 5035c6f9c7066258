"""Pins of the oracle's antiperiodic time boundary (psi(x + L_t t) = -psi(x)).

Free-field closed forms with half-integer time momenta, anti- and
eps-Hermiticity with random links, the equivalence with negated boundary
time links (the form the GPU library applies), and the fermion-force
formula against the exact linear variation of D.
"""
import itertools

import numpy as np
import pytest

from oracle.dirac import KahlerDirac, Staggered
from oracle.force import link_gradient
from oracle.lattice import Lattice
from paper_2212_12559_gb300 import inputs


def unit_links(V):
    return np.broadcast_to(np.eye(3, dtype=np.complex128), (4, V, 3, 3)).copy()


def dense(op, V):
    n = 3 * V
    Dm = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1
        Dm[:, j] = op.D(e.reshape(V, 3)).ravel()
    return Dm


@pytest.mark.parametrize("c_naik", [0.0, -1.0 / 24])
def test_free_field_plane_wave_antiperiodic(c_naik):
    """Unit links, half-integer time momenta p_t = 2 pi (n + 1/2) / L_t:
    D^2 e^{ipx} chi = -sum_mu (sin p_mu + c_N sin 3p_mu)^2 e^{ipx} chi."""
    dims = (4, 6, 4, 8)
    lat = Lattice(dims)
    links = unit_links(lat.V)
    op = Staggered(lat, links, links if c_naik else None, c_naik, 0.0, bc_t=-1)
    g = np.random.default_rng(1)
    for _ in range(4):
        n = [g.integers(0, L) for L in dims]
        p = np.array([2 * np.pi * (n[m] + (0.5 if m == 3 else 0.0)) / dims[m] for m in range(4)])
        chi = g.standard_normal(3) + 1j * g.standard_normal(3)
        psi = np.exp(1j * lat.coords @ p)[:, None] * chi[None, :]
        lam = -np.sum((np.sin(p) + c_naik * np.sin(3 * p)) ** 2)
        assert np.allclose(op.D(op.D(psi)), lam * psi, atol=1e-12)


def test_free_field_dense_spectrum_antiperiodic():
    """Eigenvalues of D on 4^4 with unit links and the antiperiodic time
    boundary: +-i sqrt(sum sin^2 p_mu) with p_t half-integer; no zero mode."""
    dims = (4, 4, 4, 4)
    lat = Lattice(dims)
    ev = np.linalg.eigvals(dense(Staggered(lat, unit_links(lat.V), bc_t=-1), lat.V))
    assert np.max(np.abs(ev.real)) < 1e-12
    s = []
    for nn in itertools.product(range(4), repeat=4):
        p = 2 * np.pi * (np.asarray(nn) + np.array([0, 0, 0, 0.5])) / 4
        s += [np.sqrt(np.sum(np.sin(p) ** 2))] * 3
    assert np.allclose(np.sort(np.abs(ev.imag)), np.sort(s), atol=1e-10)
    assert np.min(np.abs(ev.imag)) > 0.5      # sin^2(pi/4) = 1/2 per direction at least


@pytest.mark.parametrize("hisq", [False, True])
def test_hermiticity_antiperiodic(hisq):
    """D^dag = -D and eps D eps = -D with random links."""
    dims = (4, 4, 4, 8)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 5)
    fat = inputs.fat_links(thin, dims) if hisq else thin
    naik = inputs.naik_links(thin, dims) if hisq else None
    op = Staggered(lat, fat, naik, -1 / 24 if hisq else 0.0, 0.0, bc_t=-1)
    u, v = inputs.gaussian_field(lat.V, 3, 11), inputs.gaussian_field(lat.V, 3, 12)
    assert abs(np.vdot(u, op.D(v)) + np.vdot(op.D(u), v)) < 1e-12 * np.linalg.norm(u) * np.linalg.norm(v) * 10
    eps = lat.eps()[:, None]
    assert np.allclose(eps * op.D(eps * v), -op.D(v), atol=1e-12)


@pytest.mark.parametrize("hisq", [False, True])
def test_antiperiodic_equals_negated_boundary_links(hisq):
    """The antiperiodic operator is the periodic one on links whose time
    component is negated where the hop wraps: fat links on the last time
    slice, Naik links on the last three; the KD blocks never contain a
    wrapping hop, so (B+m)^{-1} and A follow."""
    dims = (4, 4, 6, 8)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 6)
    fat = inputs.fat_links(thin, dims) if hisq else thin
    naik = inputs.naik_links(thin, dims) if hisq else None
    c = -1 / 24 if hisq else 0.0
    t = lat.coords[:, 3]
    fat_f = fat.copy()
    fat_f[3][t == dims[3] - 1] *= -1
    naik_f = None
    if hisq:
        naik_f = naik.copy()
        naik_f[3][t >= dims[3] - 3] *= -1
    ap = Staggered(lat, fat, naik, c, 0.07, bc_t=-1)
    pf = Staggered(lat, fat_f, naik_f, c, 0.07)
    v = inputs.gaussian_field(lat.V, 3, 13)
    assert np.allclose(ap.M(v), pf.M(v), atol=1e-13)
    assert np.allclose(ap.B(v), pf.B(v), atol=1e-13)
    assert np.allclose(KahlerDirac(ap).A(v), KahlerDirac(pf).A(v), atol=1e-12)
    assert not np.allclose(ap.M(v), Staggered(lat, fat, naik, c, 0.07).M(v))


@pytest.mark.parametrize("naik_links", [False, True])
def test_force_formula_antiperiodic(naik_links):
    """G of link_gradient is the exact derivative of the bilinear form
    -2 Re Y^dag D(U) X: D is linear in the links, so for any direction dU the
    variation is -2 Re Y^dag D_dU X with D_dU the operator built on dU (same
    phases and boundary), and it must equal Re <G, dU>."""
    dims = (4, 4, 4, 8)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 7)
    fat, naik = inputs.fat_links(thin, dims), inputs.naik_links(thin, dims)
    c = -1 / 24
    op = Staggered(lat, fat, naik, c, 0.05, bc_t=-1)
    x, y = inputs.gaussian_field(lat.V, 3, 21), inputs.gaussian_field(lat.V, 3, 22)
    g = np.random.default_rng(3)
    du = g.standard_normal((4, lat.V, 3, 3)) + 1j * g.standard_normal((4, lat.V, 3, 3))
    if naik_links:
        var = Staggered(lat, np.zeros_like(fat), du, c, 0.0, bc_t=-1)
    else:
        var = Staggered(lat, du, None, 0.0, 0.0, bc_t=-1)
    lhs = -2 * np.vdot(y, var.D(x)).real
    rhs = np.vdot(link_gradient(op, x, y, naik=naik_links), du).real
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
