"""Fermion force through torch.autograd and the C ABI.

Pins: the library's X, Y agree with the oracle's (dense solves); the
autograd link gradient equals the oracle's formula on those vectors; central
finite differences (eps = 1e-4) of S along random su(3) directions
U -> exp(i eps T) U match the gradient; dS/dm matches -2 m |X|^2 and its own
finite difference (configuration 5 shape on a smaller lattice).
"""
import numpy as np
import pytest
import scipy.linalg

from oracle.dirac import Staggered
from oracle.force import action_vectors, link_gradient, mass_gradient
from oracle.lattice import Lattice
from paper_2212_12559_gb300 import inputs

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("prec", [0, 2])
def test_fermion_force_autograd(lib, prec):
    import torch
    from paper_2212_12559_gb300 import binding
    from paper_2212_12559_gb300.force import fermion_action
    dims = (8, 4, 4, 8)
    m = 0.02
    thin = inputs.random_su3_links(dims, 1005)
    lat = Lattice(dims)
    V = lat.V
    phi = inputs.gaussian_field(V, 3, 2005)
    s = binding.Solver(dims)
    s.set_gauge(thin)
    s.set_mass(m)
    s.mg_setup(binding.default_params(nvec=[6], setup_maxiter=100, precision=prec),
               [inputs.gaussian_fields(6, V, 3, 3005)])
    dev = torch.device("cuda")
    U = torch.from_numpy(thin).to(dev).requires_grad_(True)
    mt = torch.tensor(m, dtype=torch.float64, requires_grad=True)
    ph = torch.from_numpy(phi).to(dev)
    S = fermion_action(U, mt, ph, s, tol=1e-12)
    S.backward()
    G = U.grad.cpu().numpy()
    op = Staggered(lat, thin, None, 0.0, m)
    S_o, X_o, Y_o = action_vectors(op, dense_solver(op), phi)
    assert abs(S.item() - S_o) <= 1e-9 * abs(S_o)
    G_o = link_gradient(op, X_o, Y_o)
    assert np.linalg.norm(G - G_o) <= 1e-8 * np.linalg.norm(G_o)
    assert abs(mt.grad.item() - mass_gradient(op, X_o)) <= 1e-8 * abs(mass_gradient(op, X_o))
    # central finite differences along random su(3) directions through the GPU
    # action, eps = 1e-4 and eps/2 combined (Richardson) to cancel the O(eps^2)
    # term, which at m = 0.02 is ~3e-5 of the derivative
    h = 1e-4
    Ts = inputs.lie_directions(16, V, 4005)

    def central(T, e):
        vals = []
        for sg in (1, -1):
            Ue = torch.from_numpy(expm_i(sg * e, T) @ thin).to(dev)
            vals.append(fermion_action(Ue, mt.detach(), ph, s, tol=1e-12).item())
        return (vals[0] - vals[1]) / (2 * e)

    for T in Ts:
        d1, d2 = central(T, h), central(T, h / 2)
        fd = (4 * d2 - d1) / 3
        an = np.sum((np.conj(G) * (1j * T @ thin)).real)
        assert abs(d1 - an) <= 1e-4 * abs(an) + 1e-6 * abs(S_o), (d1, an)
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-7 * abs(S_o), (fd, an)

    def central_m(e):
        sp = fermion_action(torch.from_numpy(thin).to(dev), m + e, ph, s, tol=1e-12).item()
        sm = fermion_action(torch.from_numpy(thin).to(dev), m - e, ph, s, tol=1e-12).item()
        return (sp - sm) / (2 * e)

    dm = 1e-5
    fdm = (4 * central_m(dm / 2) - central_m(dm)) / 3
    assert abs(fdm - mt.grad.item()) <= 1e-6 * abs(mt.grad.item())


@pytest.mark.parametrize("prec", [0, 2])
def test_fermion_force_16x4_64_directions(lib, prec):
    """The force workload at its own shape: 16^4 naive, m = 0.02, Gaussian
    phi, 64 random su(3) directions with central differences at eps = 1e-4
    with the mixed-precision preconditioner (8 with the FP64 one).  At this size there is no dense solve: the
    oracle checks the library's X, Y through its own operator (M X = Y,
    M^dag Y = phi), the link gradient is the oracle's formula on those
    vectors, dS/dm = -2 m |X|^2, and each directional difference matches the
    gradient to its O(eps^2) term (about 3e-5 relative at this mass)."""
    import torch
    from paper_2212_12559_gb300 import binding
    from paper_2212_12559_gb300.force import fermion_action
    dims, m = (16, 16, 16, 16), 0.02
    lat = Lattice(dims)
    V = lat.V
    thin = inputs.random_su3_links(dims, 1005)
    phi = inputs.gaussian_field(V, 3, 2005)
    s = binding.Solver(dims)
    s.set_gauge(thin)
    s.set_mass(m)
    s.mg_setup(binding.default_params(nvec=[24], setup_maxiter=300, precision=prec),
               [inputs.gaussian_fields(24, V, 3, 3005)])
    dev = torch.device("cuda")
    U = torch.from_numpy(thin).to(dev).requires_grad_(True)
    mt = torch.tensor(m, dtype=torch.float64, requires_grad=True)
    ph = torch.from_numpy(phi).to(dev)
    S = fermion_action(U, mt, ph, s, tol=1e-12)
    S.backward()
    G = U.grad.cpu().numpy()
    _, _, X, Y, infos = s.fermion_action(ph, 1e-12)
    X, Y = X.cpu().numpy(), Y.cpu().numpy()
    op = Staggered(lat, thin, None, 0.0, m)
    # M X = Y and M^dag Y = phi (M^dag = eps M eps) by the oracle's operator
    assert np.linalg.norm(op.M(X) - Y) <= 1e-11 * np.linalg.norm(Y)
    eps = lat.eps()[:, None]
    assert np.linalg.norm(eps * op.M(eps * Y) - phi) <= 1e-11 * np.linalg.norm(phi)
    S_o = float(np.vdot(Y, Y).real)
    assert abs(S.item() - S_o) <= 1e-12 * S_o
    G_o = link_gradient(op, X, Y)
    assert np.linalg.norm(G - G_o) <= 1e-12 * np.linalg.norm(G_o)
    assert abs(mt.grad.item() - mass_gradient(op, X)) <= 1e-12 * abs(mass_gradient(op, X))
    h = 1e-4
    # 64 directions with the mixed-precision preconditioner; 8 with the FP64
    # one (each direction rebuilds the coarse operators twice)
    Ts = inputs.lie_directions(64 if prec == 2 else 8, V, 4005)
    for T in Ts:
        vals = []
        for sg in (1, -1):
            Ue = torch.from_numpy(expm_i(sg * h, T) @ thin).to(dev)
            vals.append(fermion_action(Ue, mt.detach(), ph, s, tol=1e-12).item())
        fd = (vals[0] - vals[1]) / (2 * h)
        an = np.sum((np.conj(G) * (1j * T @ thin)).real)
        assert abs(fd - an) <= 1e-4 * abs(an) + 1e-7 * S_o, (fd, an)
    dm = 1e-5
    sp = fermion_action(torch.from_numpy(thin).to(dev), m + dm, ph, s, tol=1e-12).item()
    sm = fermion_action(torch.from_numpy(thin).to(dev), m - dm, ph, s, tol=1e-12).item()
    assert abs((sp - sm) / (2 * dm) - mt.grad.item()) <= 1e-5 * abs(mt.grad.item())
