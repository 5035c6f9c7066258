"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds no arithmetic of the solver itself (no phases, no hopping
operator, no block maps): it only draws random numbers and turns them into the
gauge fields, sources and start vectors that the solver takes as inputs.  Both
the CUDA path (through the Python binding and ``bench.py``) and the CPU oracle
import it, so the two sides always see identical arrays.

Conventions (the paper fixes none of them, Sec. 2.2):

* A lattice has extents ``dims = (Lx, Ly, Lz, Lt)``; site ``i`` has lexical
  index ``x + Lx*(y + Ly*(z + Lz*t))`` (x fastest).  Boundaries are periodic.
* A colour vector field is a complex128 array of shape ``(V, 3)``.
* A link field is a complex128 array of shape ``(4, V, 3, 3)``; entry
  ``[mu, i, a, b]`` is row ``a``, column ``b`` of the link from site ``i`` to
  site ``i + mu``.

Link recipe (the paper's workloads are physical HISQ configurations that are
not available here; these seeded fields stand in for them):

* thin links ``U = Proj_SU3(exp(i * eps * H))``, ``H`` Gaussian traceless
  Hermitian (complex entries with unit-variance real and imaginary parts,
  Hermitised and made traceless);
* fat links ``V = Proj_SU3(U + alpha * staples)``, one APE-like smearing step;
* Naik (long) links ``W_mu(x) = U_mu(x) U_mu(x+mu) U_mu(x+2mu)``.

All randomness comes from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng", "volume", "site_coords", "shifted_index", "project_su3",
    "random_su3_links", "fat_links", "naik_links", "gaussian_field",
    "gaussian_fields", "random_su3_field", "log_masses", "lie_directions",
    "config_inputs",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def volume(dims) -> int:
    return int(np.prod(np.asarray(dims, dtype=np.int64)))


def site_coords(dims) -> np.ndarray:
    """(V, 4) int64 coordinates of every site in lexical order (x fastest)."""
    dims = tuple(int(d) for d in dims)
    idx = np.arange(volume(dims), dtype=np.int64)
    out = np.empty((idx.size, 4), dtype=np.int64)
    rem = idx
    for mu in range(4):
        out[:, mu] = rem % dims[mu]
        rem = rem // dims[mu]
    return out


def shifted_index(dims, mu: int, k: int) -> np.ndarray:
    """Lexical index of site x + k*mu_hat (periodic) for every site x."""
    dims = tuple(int(d) for d in dims)
    c = site_coords(dims)
    c[:, mu] = (c[:, mu] + k) % dims[mu]
    stride = [1, dims[0], dims[0] * dims[1], dims[0] * dims[1] * dims[2]]
    return c @ np.asarray(stride, dtype=np.int64)


def _gaussian_complex(g: np.random.Generator, shape) -> np.ndarray:
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def _random_traceless_hermitian(g: np.random.Generator, n: int) -> np.ndarray:
    a = _gaussian_complex(g, (n, 3, 3))
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)
    return h


def project_su3(m: np.ndarray) -> np.ndarray:
    """Nearest unitary matrix (polar factor) with the determinant phase removed.

    ``W = M (M^dag M)^{-1/2}``, then ``W / det(W)^{1/3}``.  Both steps commute
    with ``M -> g M h^dag`` for g, h in SU(3), so smearing built from it stays
    gauge covariant.
    """
    u, _, vh = np.linalg.svd(m)
    w = u @ vh
    det = np.linalg.det(w)
    phase = np.exp(-1j * np.angle(det) / 3.0)
    return w * phase[..., None, None]


def random_su3_links(dims, seed: int, eps: float = 0.3) -> np.ndarray:
    """Thin links Proj_SU3(exp(i*eps*H)), shape (4, V, 3, 3)."""
    g = rng(seed)
    V = volume(dims)
    h = _random_traceless_hermitian(g, 4 * V)
    w, q = np.linalg.eigh(h)
    ex = (q * np.exp(1j * eps * w)[:, None, :]) @ np.conj(np.swapaxes(q, -1, -2))
    return project_su3(ex).reshape(4, V, 3, 3)


def random_su3_field(dims, seed: int, eps: float = 1.0) -> np.ndarray:
    """One random SU(3) matrix per site, shape (V, 3, 3) (gauge transforms)."""
    g = rng(seed)
    V = volume(dims)
    h = _random_traceless_hermitian(g, V)
    w, q = np.linalg.eigh(h)
    ex = (q * np.exp(1j * eps * w)[:, None, :]) @ np.conj(np.swapaxes(q, -1, -2))
    return project_su3(ex)


def _dag(m: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(m, -1, -2))


def fat_links(thin: np.ndarray, dims, alpha: float = 0.1) -> np.ndarray:
    """One APE-like step: Proj_SU3(U_mu + alpha * sum of the six staples)."""
    out = np.empty_like(thin)
    for mu in range(4):
        fwd_mu = shifted_index(dims, mu, 1)
        staple = np.zeros_like(thin[mu])
        for nu in range(4):
            if nu == mu:
                continue
            fwd_nu = shifted_index(dims, nu, 1)
            bwd_nu = shifted_index(dims, nu, -1)
            # upper staple U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
            staple += thin[nu] @ thin[mu][fwd_nu] @ _dag(thin[nu][fwd_mu])
            # lower staple U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
            x_m_nu_p_mu = fwd_mu[bwd_nu]
            staple += _dag(thin[nu][bwd_nu]) @ thin[mu][bwd_nu] @ thin[nu][x_m_nu_p_mu]
        out[mu] = project_su3(thin[mu] + alpha * staple)
    return out


def naik_links(thin: np.ndarray, dims) -> np.ndarray:
    """Long links W_mu(x) = U_mu(x) U_mu(x+mu) U_mu(x+2mu)."""
    out = np.empty_like(thin)
    for mu in range(4):
        f1 = shifted_index(dims, mu, 1)
        f2 = shifted_index(dims, mu, 2)
        out[mu] = thin[mu] @ thin[mu][f1] @ thin[mu][f2]
    return out


def gaussian_field(dims_or_V, n: int, seed: int) -> np.ndarray:
    """Complex Gaussian field of shape (V, n), unit-variance real/imag parts."""
    V = dims_or_V if isinstance(dims_or_V, (int, np.integer)) else volume(dims_or_V)
    return _gaussian_complex(rng(seed), (int(V), int(n)))


def gaussian_fields(count: int, V: int, n: int, seed: int) -> np.ndarray:
    """``count`` Gaussian fields, shape (count, V, n), from one stream."""
    return _gaussian_complex(rng(seed), (int(count), int(V), int(n)))


def log_masses(m_lo: float = 0.001, m_hi: float = 0.05, n: int = 8) -> np.ndarray:
    """Log-spaced masses m_i = m_lo * (m_hi/m_lo)^(i/(n-1))."""
    i = np.arange(n, dtype=np.float64)
    return m_lo * (m_hi / m_lo) ** (i / (n - 1))


def lie_directions(count: int, V: int, seed: int) -> np.ndarray:
    """Random traceless Hermitian 3x3 matrices per link, shape (count, 4, V, 3, 3)."""
    g = rng(seed)
    t = _random_traceless_hermitian(g, count * 4 * V)
    return t.reshape(count, 4, V, 3, 3)


# ----------------------------------------------------------------------------
# The five benchmark workloads, as seeded recipes.
# ----------------------------------------------------------------------------

CONFIGS = {
    1: dict(dims=(8, 8, 8, 8), hisq=False, mass=0.1, agg=[(4, 4, 4, 4)], nvec=[24],
            precision="double", nrhs=1, masses=None, seeds=(1001, 2001, 3001)),
    2: dict(dims=(16, 16, 16, 16), hisq=True, mass=0.01, agg=[(4, 4, 4, 4), (2, 2, 2, 2)],
            nvec=[24, 32], precision="mixed", nrhs=1, masses=None, seeds=(1002, 2002, 3002)),
    3: dict(dims=(32, 32, 32, 32), hisq=False, mass=0.001, agg=[(4, 4, 4, 4), (2, 2, 2, 2)], nvec=[64, 32],
            precision="mixed", nrhs=12, masses=None, seeds=(1003, 2003, 3003)),
    4: dict(dims=(24, 24, 24, 48), hisq=True, mass=0.001, agg=[(4, 4, 4, 4), (2, 2, 2, 2)],
            nvec=[64, 32], precision="mixed", nrhs=4, masses="log8", seeds=(1004, 2004, 3004)),
    5: dict(dims=(16, 16, 16, 16), hisq=False, mass=0.02, agg=[(4, 4, 4, 4)], nvec=[24],
            precision="double", nrhs=1, masses=None, seeds=(1005, 2005, 3005)),
}


def config_inputs(cfg: int, dims=None):
    """Gauge fields and sources of one workload (optionally on other extents).

    Returns a dict with ``fat``, ``naik`` (None for the naive operator),
    ``c_naik``, ``sources`` (nrhs, V, 3) and ``nullvec_seed``.
    """
    c = dict(CONFIGS[cfg])
    if dims is not None:
        c["dims"] = tuple(dims)
    dims = c["dims"]
    s_link, s_src, s_nv = c["seeds"]
    thin = random_su3_links(dims, s_link, 0.3)
    if c["hisq"]:
        fat = fat_links(thin, dims, 0.1)
        naik = naik_links(thin, dims)
        c_naik = -1.0 / 24.0
    else:
        fat, naik, c_naik = thin, None, 0.0
    V = volume(dims)
    src = np.stack([gaussian_field(V, 3, s_src + r) for r in range(c["nrhs"])])
    c.update(fat=fat, naik=naik, c_naik=c_naik, sources=src, nullvec_seed=s_nv)
    return c
