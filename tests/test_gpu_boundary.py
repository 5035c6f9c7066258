"""The antiperiodic time boundary on the GPU against the oracle (bc_t = -1).

smg_set_boundary(SMG_BC_T_ANTIPERIODIC) before smg_set_gauge: the fine
operator in every storage precision, the KD block inverse and A per element
against the oracle's antiperiodic operator; a multigrid solve to 1e-10 with
the residual recomputed by the oracle; the force kernel for fat and Naik
links; and the switch back to the periodic boundary.  Bars as in
test_gpu_ops: FP64 1e-12, FP32 1e-6, FP16 storage 5e-3 (the larger of the
relative 2-norm error and max |error| / max |ref|).
"""
import numpy as np
import pytest

from oracle.dirac import KahlerDirac, Staggered
from oracle.force import link_gradient
from oracle.lattice import Lattice
from paper_2212_12559_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6, 2: 5e-3}


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    d = np.abs(a - b)
    return max(np.linalg.norm(d) / np.linalg.norm(b), d.max() / np.abs(b).max())


@pytest.fixture(scope="module")
def binding(lib):
    from paper_2212_12559_gb300 import binding as b
    return b


def hisq_problem(dims, seed, mass):
    thin = inputs.random_su3_links(dims, seed)
    fat, naik, c = inputs.fat_links(thin, dims), inputs.naik_links(thin, dims), -1.0 / 24
    return fat, naik, c, Staggered(Lattice(dims), fat, naik, c, mass, bc_t=-1)


def test_antiperiodic_operators(binding):
    dims, mass = (8, 4, 6, 8), 0.07
    fat, naik, c, op = hisq_problem(dims, 1071, mass)
    kd = KahlerDirac(op)
    s = binding.Solver(dims)
    s.set_boundary(True)
    s.set_gauge(fat, naik, c)
    s.set_mass(mass)
    v = inputs.gaussian_fields(2, op.lat.V, 3, 71)
    for prec in (0, 1, 2):
        m = s.apply(binding.OP_M, v, prec)
        for k in range(2):
            assert rel(m[k], op.M(v[k])) <= TOL[prec], ("M", prec, k)
    a = s.apply(binding.OP_A, v, binding.PREC_DOUBLE)
    binv = s.apply(binding.OP_KD, v, binding.PREC_DOUBLE)
    for k in range(2):
        assert rel(a[k], kd.A(v[k])) <= 1e-12
        assert rel(binv[k], kd.apply_inv(v[k])) <= 1e-12
    X, Y = inputs.gaussian_field(op.lat.V, 3, 72), inputs.gaussian_field(op.lat.V, 3, 73)
    assert rel(s.force(X, Y, 0), link_gradient(op, X, Y)) <= 1e-14
    assert rel(s.force(X, Y, 1), link_gradient(op, X, Y, naik=True)) <= 1e-14
    # back to periodic: the same links give the periodic operator again
    s.set_boundary(False)
    s.set_gauge(fat, naik, c)
    per = Staggered(op.lat, fat, naik, c, mass)
    m = s.apply(binding.OP_M, v, binding.PREC_DOUBLE)
    assert rel(m[0], per.M(v[0])) <= 1e-12
    assert rel(m[0], op.M(v[0])) > 1e-3


def test_antiperiodic_mg_solve(binding):
    """Two-level mixed-precision solve on 8^4 with the antiperiodic boundary:
    converged, and the residual recomputed by the oracle's operator is below
    1e-10."""
    dims, mass = (8, 8, 8, 8), 0.05
    fat, naik, c, op = hisq_problem(dims, 1072, mass)
    s = binding.Solver(dims)
    s.set_boundary(True)
    s.set_gauge(fat, naik, c)
    s.set_mass(mass)
    V = op.lat.V
    s.mg_setup(binding.default_params(nvec=[8], setup_maxiter=100, precision=binding.PREC_HALF),
               [inputs.gaussian_fields(8, V, 3, 3072)])
    b = inputs.gaussian_field(V, 3, 2072)
    x, info = s.solve(b, 1e-10)
    assert info.converged == 1 and info.true_residual <= 1e-10
    assert np.linalg.norm(b - op.M(x)) / np.linalg.norm(b) <= 1e-10
