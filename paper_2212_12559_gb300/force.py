"""The fermion action S = phi^dag (M^dag M)^{-1} phi as a torch.autograd.Function.

Forward: two multigrid solves in libsmg (smg_fermion_action).  Backward: the
link derivative from the library's outer-product kernel (smg_force) and
dS/dm = -2 m |X|^2, both scaled by the incoming gradient.  The gradient with
respect to a complex link follows PyTorch's convention for real functions of
complex tensors: dS/dRe U + i dS/dIm U.

Between calls with new links the near-null vectors are kept and the Galerkin
operators rebuilt from them (the paper reuses near-null vectors across
solves, Sec. 3.2; evolving them under HMC is future work there, Sec. 4).
"""
from __future__ import annotations

import torch

from . import binding


def _refresh(solver: binding.Solver, fat, naik, c_naik, mass):
    params = solver.params
    if params is None:
        raise RuntimeError("run mg_setup on the solver once before using FermionAction")
    vecs = [solver.null_vectors(l) for l in range(params.n_coarse)]
    solver.set_gauge(fat, naik, c_naik)
    solver.set_mass(mass)
    p = binding.MGParams.from_buffer_copy(params)
    p.setup_maxiter = 0
    solver.mg_setup(p, vecs)
    solver.params = params


class FermionAction(torch.autograd.Function):
    """S(U, m) for a fixed pseudofermion phi; differentiable in the fat links
    (and Naik links when given) and in the mass."""

    @staticmethod
    def forward(ctx, fat, mass, phi, solver, naik=None, c_naik=0.0, tol=1e-10):
        m = float(mass.detach().cpu()) if isinstance(mass, torch.Tensor) else float(mass)
        _refresh(solver, fat.detach().contiguous(), None if naik is None else naik.detach().contiguous(),
                 c_naik, m)
        S, dSdm, X, Y, infos = solver.fermion_action(phi.detach().contiguous(), tol)
        if not all(i.converged for i in infos):
            raise RuntimeError("fermion action: a multigrid solve did not converge")
        ctx.solver = solver
        ctx.has_naik = naik is not None
        ctx.dSdm = dSdm
        ctx.save_for_backward(X, Y)
        return torch.tensor(S, dtype=torch.float64, device=fat.device)

    @staticmethod
    def backward(ctx, grad):
        X, Y = ctx.saved_tensors
        g = grad.to(torch.float64)
        F = ctx.solver.force(X, Y, 0) * g
        FN = ctx.solver.force(X, Y, 1) * g if ctx.has_naik else None
        dm = torch.as_tensor(ctx.dSdm, dtype=torch.float64) * g.cpu()
        return F, dm, None, None, FN, None, None


def fermion_action(fat, mass, phi, solver, naik=None, c_naik=0.0, tol=1e-10):
    return FermionAction.apply(fat, mass, phi, solver, naik, c_naik, tol)
