"""Pins of the oracle's geometry, staggered operator and Kahler-Dirac split.

Each test checks the oracle against something other than itself: brute-force
loops, free-field closed forms (Sec. 2.2), Hermiticity identities, gauge
covariance, or the free-field KD algebra of Eq. 1 and Eq. 2.
"""
import itertools

import numpy as np
import pytest

from oracle.dirac import KahlerDirac, Staggered, gauge_transform_links
from oracle.lattice import Lattice, enumerate_sites
from paper_2212_12559_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore")


def unit_links(V):
    return np.broadcast_to(np.eye(3, dtype=np.complex128), (4, V, 3, 3)).copy()


def rand_spinor(V, seed):
    return inputs.gaussian_field(V, 3, seed)


# --------------------------------------------------------------------------- maps
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 4, 6, 2), (2, 6, 4, 8)])
def test_lexical_order_matches_nested_loops(dims):
    lat = Lattice(dims)
    assert np.array_equal(lat.coords, enumerate_sites(dims))
    assert np.array_equal(lat.index(lat.coords), np.arange(lat.V))


def test_phases_and_chirality_brute_force():
    lat = Lattice((4, 6, 4, 2))
    for i in range(lat.V):
        x = [int(c) for c in lat.coords[i]]
        for mu in range(4):
            assert lat.eta(mu)[i] == (-1) ** sum(x[:mu])
        assert lat.eps()[i] == (-1) ** sum(x)


def test_hypercubes_and_aggregates_brute_force():
    lat = Lattice((8, 4, 4, 8))
    sites = lat.kd_sites()
    for n in range(sites.shape[0]):
        cs = lat.coords[sites[n]]
        assert len(set(map(tuple, cs // 2))) == 1          # one hypercube
        for b in range(16):
            assert [(b >> mu) & 1 for mu in range(4)] == list(cs[b] % 2)
    aidx, apos = lat.aggregate((4, 4, 2, 4))
    cd = lat.coarse_dims((4, 4, 2, 4))
    assert cd == (2, 1, 2, 2)
    for i in range(lat.V):
        x = lat.coords[i]
        X = [x[0] // 4, x[1] // 4, x[2] // 2, x[3] // 4]
        assert aidx[i] == X[0] + cd[0] * (X[1] + cd[1] * (X[2] + cd[2] * X[3]))
        r = [x[0] % 4, x[1] % 4, x[2] % 2, x[3] % 4]
        assert apos[i] == r[0] + 4 * (r[1] + 4 * (r[2] + 2 * r[3]))


# ------------------------------------------------------------------- operator
def brute_force_D(dims, fat, naik, c_naik, psi, site):
    """(D psi)(site) with explicit coordinate arithmetic and 3x3 loops."""
    V = int(np.prod(dims))
    x = [site % dims[0], (site // dims[0]) % dims[1],
         (site // (dims[0] * dims[1])) % dims[2], site // (dims[0] * dims[1] * dims[2])]

    def idx(c):
        c = [c[m] % dims[m] for m in range(4)]
        return c[0] + dims[0] * (c[1] + dims[1] * (c[2] + dims[2] * c[3]))

    out = [0j, 0j, 0j]
    for mu in range(4):
        eta = (-1) ** sum(x[:mu])
        for links, k, coef in ((fat, 1, 0.5), (naik, 3, 0.5 * c_naik)):
            if links is None:
                continue
            fwd = list(x); fwd[mu] += k
            bwd = list(x); bwd[mu] -= k
            jf, jb = idx(fwd), idx(bwd)
            for a in range(3):
                for b in range(3):
                    out[a] += coef * eta * links[mu, site, a, b] * psi[jf, b]
                    out[a] -= coef * eta * np.conj(links[mu, jb, b, a]) * psi[jb, b]
    return np.asarray(out)


@pytest.mark.parametrize("hisq", [False, True])
def test_dslash_matches_brute_force(hisq):
    dims = (4, 4, 6, 8)
    V = int(np.prod(dims))
    thin = inputs.random_su3_links(dims, 11)
    fat = inputs.fat_links(thin, dims) if hisq else thin
    naik = inputs.naik_links(thin, dims) if hisq else None
    c = -1.0 / 24 if hisq else 0.0
    op = Staggered(Lattice(dims), fat, naik, c, mass=0.3)
    psi = rand_spinor(V, 5)
    d = op.D(psi)
    for site in [0, 1, 17, 100, V - 1, 321]:
        assert np.allclose(d[site], brute_force_D(dims, fat, naik, c, psi, site), atol=1e-13)
    assert np.allclose(op.M(psi), 0.3 * psi + d)


@pytest.mark.parametrize("c_naik", [0.0, -1.0 / 24])
def test_free_field_plane_wave(c_naik):
    """Unit links: D^2 e^{ipx} chi = -sum_mu (sin p_mu + c_N sin 3p_mu)^2 e^{ipx} chi."""
    dims = (8, 4, 6, 4)
    lat = Lattice(dims)
    links = unit_links(lat.V)
    op = Staggered(lat, links, links if c_naik else None, c_naik, 0.0)
    g = np.random.default_rng(0)
    for _ in range(4):
        n = [g.integers(0, L) for L in dims]
        p = np.array([2 * np.pi * n[m] / dims[m] for m in range(4)])
        chi = g.standard_normal(3) + 1j * g.standard_normal(3)
        psi = np.exp(1j * lat.coords @ p)[:, None] * chi[None, :]
        lam = -np.sum((np.sin(p) + c_naik * np.sin(3 * p)) ** 2)
        assert np.allclose(op.D(op.D(psi)), lam * psi, atol=1e-12)


def test_free_field_dense_spectrum():
    """Eigenvalues of D on 4^4 with unit links are +-i sqrt(sum sin^2 p_mu)."""
    dims = (4, 4, 4, 4)
    lat = Lattice(dims)
    op = Staggered(lat, unit_links(lat.V))
    n = 3 * lat.V
    Dm = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128); e[j] = 1
        Dm[:, j] = op.D(e.reshape(lat.V, 3)).ravel()
    ev = np.linalg.eigvals(Dm)
    assert np.max(np.abs(ev.real)) < 1e-12
    s = []
    for nn in itertools.product(range(4), repeat=4):
        p = 2 * np.pi * np.asarray(nn) / 4
        s += [np.sqrt(np.sum(np.sin(p) ** 2))] * 3
    assert np.allclose(np.sort(np.abs(ev.imag)), np.sort(s), atol=1e-10)
    assert abs(ev.imag.sum()) < 1e-9


@pytest.mark.parametrize("hisq", [False, True])
def test_anti_and_eps_hermiticity(hisq):
    dims = (4, 4, 4, 8)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 3)
    fat = inputs.fat_links(thin, dims) if hisq else thin
    naik = inputs.naik_links(thin, dims) if hisq else None
    op = Staggered(lat, fat, naik, -1 / 24 if hisq else 0.0, 0.05)
    u, v = rand_spinor(lat.V, 1), rand_spinor(lat.V, 2)
    assert np.isclose(np.vdot(u, op.D(v)), -np.vdot(op.D(u), v), rtol=1e-13)
    eps = lat.eps()[:, None]
    assert np.isclose(np.vdot(u, eps * op.M(eps * v)), np.vdot(op.M(u), v), rtol=1e-13)
    assert np.isclose(np.vdot(u, op.M(v)), np.vdot(op.Mdag(u), v), rtol=1e-13)


@pytest.mark.parametrize("hisq", [False, True])
def test_gauge_covariance(hisq):
    dims = (4, 4, 4, 4)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 7)
    fat = inputs.fat_links(thin, dims) if hisq else thin
    naik = inputs.naik_links(thin, dims) if hisq else None
    c = -1 / 24 if hisq else 0.0
    g = inputs.random_su3_field(dims, 99)
    fat_g = gauge_transform_links(lat, fat, g, 1)
    naik_g = None if naik is None else gauge_transform_links(lat, naik, g, 3)
    psi = rand_spinor(lat.V, 4)
    op = Staggered(lat, fat, naik, c, 0.2)
    op_g = Staggered(lat, fat_g, naik_g, c, 0.2)
    lhs = op_g.M(np.einsum("xab,xb->xa", g, psi))
    rhs = np.einsum("xab,xb->xa", g, op.M(psi))
    assert np.allclose(lhs, rhs, atol=1e-12)
    kd, kd_g = KahlerDirac(op), KahlerDirac(op_g)
    lhs = kd_g.A(np.einsum("xab,xb->xa", g, psi))
    rhs = np.einsum("xab,xb->xa", g, kd.A(psi))
    assert np.allclose(lhs, rhs, atol=1e-11)


# ------------------------------------------------------------------ KD algebra
def test_free_field_kd_algebra():
    """Unit links, 1/2 normalisation: B^2 = C^2 = -1, (B+m)^{-1} = (m - B)/(1 + m^2),
    and the spectrum of A = (B+m)^{-1} M lies on |lambda - 1| = 1/sqrt(1+m^2)."""
    dims = (4, 4, 4, 4)
    lat = Lattice(dims)
    m = 0.1
    op = Staggered(lat, unit_links(lat.V), mass=m)
    psi = rand_spinor(lat.V, 8)
    assert np.allclose(op.B(op.B(psi)), -psi, atol=1e-13)
    assert np.allclose(op.C(op.C(psi)), -psi, atol=1e-13)
    eps = lat.eps()[:, None]
    u = rand_spinor(lat.V, 9)
    for X in (op.B, op.C):   # anti-Hermitian and eps-Hermitian pieces
        assert np.isclose(np.vdot(u, X(psi)), -np.vdot(X(u), psi))
        assert np.allclose(eps * X(eps * psi), -X(psi))
    kd = KahlerDirac(op)
    Bblk = kd.blocks - m * np.eye(48)
    assert np.allclose(kd.inv, (m * np.eye(48) - Bblk) / (1 + m * m), atol=1e-13)
    n = 3 * lat.V
    Am = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128); e[j] = 1
        Am[:, j] = kd.A(e.reshape(lat.V, 3)).ravel()
    ev = np.linalg.eigvals(Am)
    assert np.allclose(np.abs(ev - 1.0), 1 / np.sqrt(1 + m * m), atol=1e-10)


@pytest.mark.parametrize("hisq", [False, True])
def test_kd_blocks_interacting(hisq):
    dims = (4, 4, 4, 8)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 21)
    fat = inputs.fat_links(thin, dims) if hisq else thin
    naik = inputs.naik_links(thin, dims) if hisq else None
    op = Staggered(lat, fat, naik, -1 / 24 if hisq else 0.0, 0.01)
    kd = KahlerDirac(op)
    eye = np.eye(48)
    assert np.allclose(kd.blocks @ kd.inv, eye, atol=1e-11)
    psi = rand_spinor(lat.V, 3)
    # B + m acting through the blocks equals the operator's B + m
    bl = kd.scatter(np.einsum("nij,nj->ni", kd.blocks, kd.gather(psi)))
    assert np.allclose(bl, op.B(psi) + 0.01 * psi, atol=1e-13)
    # every Naik hop is in C, and M = (B + m) + C (Eq. 1)
    assert np.allclose(op.M(psi), op.B(psi) + 0.01 * psi + op.C(psi), atol=1e-13)
    u = rand_spinor(lat.V, 4)
    assert np.isclose(np.vdot(u, kd.A(psi)), np.vdot(kd.Adag(u), psi), rtol=1e-12)


@pytest.mark.parametrize("agg", [(4, 4, 4, 4), (4, 4, 2, 4)])
def test_operator_parts_sum_to_M(agg):
    dims = (8, 4, 4, 8)
    lat = Lattice(dims)
    thin = inputs.random_su3_links(dims, 5)
    op = Staggered(lat, inputs.fat_links(thin, dims), inputs.naik_links(thin, dims), -1 / 24, 0.1)
    psi = rand_spinor(lat.V, 6)
    parts = op.M_parts(psi, agg)
    assert np.allclose(sum(parts.values()), op.M(psi), atol=1e-13)
    for k, v in parts.items():
        assert np.allclose(v, op.M_part(psi, agg, k), atol=1e-14)
