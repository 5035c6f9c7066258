"""GPU multigrid solves through the C ABI, judged by the oracle.

Every solve must meet ||b - M x|| <= 1e-10 ||b|| with the residual recomputed
by the oracle's FP64 operator (Sec. 3.2: tolerance on the full operator), and
its solution must agree with an independent oracle solution within the
bound ||x - x*|| <= (tol_gpu + tol_ref) * ||M|| ||M^-1|| ||x*||, with
||M|| <= m + 4 (1 + |c_N|) and ||M^-1|| <= 1/m (D is anti-Hermitian).
"""
import numpy as np
import pytest
import scipy.linalg

from oracle.dirac import Staggered
from oracle.lattice import Lattice
from oracle.solvers import gcr
from paper_2212_12559_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding(lib):
    from paper_2212_12559_gb300 import binding as b
    return b


def problem(dims, hisq, mass, seed=1001):
    thin = inputs.random_su3_links(dims, seed)
    if hisq:
        fat, naik, c = inputs.fat_links(thin, dims), inputs.naik_links(thin, dims), -1 / 24
    else:
        fat, naik, c = thin, None, 0.0
    return fat, naik, c, Staggered(Lattice(dims), fat, naik, c, mass)


def bound(op, tol):
    return tol * (op.mass + 4 * (1 + abs(op.c_naik))) / op.mass


def check_solution(op, b, x, x_ref, tol_ref):
    r = np.linalg.norm(b - op.M(x)) / np.linalg.norm(b)
    assert r <= 1e-10, r
    err = np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)
    assert err <= bound(op, 1e-10 + tol_ref), err


def dense_solution(op, b):
    n = 3 * op.lat.V
    Mm = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128); e[j] = 1
        Mm[:, j] = op.M(e.reshape(-1, 3)).ravel()
    return scipy.linalg.solve(Mm, b.ravel()).reshape(b.shape)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("hisq", [False, True])
def test_two_level_small_vs_dense(binding, prec, hisq):
    dims = (8, 4, 4, 4)
    fat, naik, c, op = problem(dims, hisq, 0.1)
    s = binding.Solver(dims)
    s.set_gauge(fat, naik, c)
    s.set_mass(0.1)
    p = binding.default_params(nvec=[4], setup_maxiter=50, precision=prec)
    s.mg_setup(p, [inputs.gaussian_fields(4, op.lat.V, 3, 3001)])
    b = inputs.gaussian_field(op.lat.V, 3, 2001)
    x, info = s.solve(b, 1e-10)
    assert info.converged == 1 and info.true_residual <= 1e-10
    check_solution(op, b, x, dense_solution(op, b), 1e-13)


@pytest.mark.parametrize("prec", [0, 2])
def test_config1_shape(binding, prec):
    """8^4 naive, m = 0.1, 24 near-null vectors, 4^4 aggregates, full setup."""
    dims = (8, 8, 8, 8)
    fat, naik, c, op = problem(dims, False, 0.1)
    s = binding.Solver(dims)
    s.set_gauge(fat, naik, c)
    s.set_mass(0.1)
    p = binding.default_params(nvec=[24], precision=prec)
    s.mg_setup(p, [inputs.gaussian_fields(24, op.lat.V, 3, 3001)])
    assert 0 < s.setup_iterations(0) <= 2000
    b = inputs.gaussian_field(op.lat.V, 3, 2001)
    x, info = s.solve(b, 1e-10)
    assert info.converged == 1
    x_ref, _, res = gcr(op.M, b, tol=1e-12, maxiter=3000, nkrylov=300)
    check_solution(op, b, x, x_ref, res)


@pytest.mark.parametrize("use_graph", [0, 1])
def test_three_level_hisq_mixed(binding, use_graph):
    dims = (8, 8, 8, 8)
    fat, naik, c, op = problem(dims, True, 0.05, seed=1002)
    s = binding.Solver(dims)
    s.set_gauge(fat, naik, c)
    s.set_mass(0.05)
    p = binding.default_params(n_coarse=2, agg=[(4, 4, 4, 4), (2, 2, 2, 2)], nvec=[8, 8], setup_maxiter=200,
                               precision=binding.PREC_HALF, use_graph=use_graph)
    s.mg_setup(p, [inputs.gaussian_fields(8, op.lat.V, 3, 3002), inputs.gaussian_fields(8, 16, 16, 3003)])
    b = inputs.gaussian_field(op.lat.V, 3, 2002)
    x, info = s.solve(b, 1e-10)
    assert info.converged == 1
    x2, info2 = s.solve(b, 1e-10)          # a second solve reuses the engine (and graph)
    assert info2.converged == 1
    x_ref, _, res = gcr(op.M, b, tol=1e-12, maxiter=3000, nkrylov=300)
    check_solution(op, b, x, x_ref, res)
    check_solution(op, b, x2, x_ref, res)


def test_three_level_coarsest_gcr(binding):
    """Coarsest level solved by GCR(0.25, 8) instead of the dense inverse."""
    dims = (8, 8, 8, 8)
    fat, naik, c, op = problem(dims, False, 0.1)
    s = binding.Solver(dims)
    s.set_gauge(fat, naik, c)
    s.set_mass(0.1)
    p = binding.default_params(n_coarse=2, agg=[(4, 4, 4, 4), (2, 1, 1, 1)], nvec=[6, 6], setup_maxiter=100,
                               dense_max=0, precision=binding.PREC_SINGLE)
    s.mg_setup(p, [inputs.gaussian_fields(6, op.lat.V, 3, 1), inputs.gaussian_fields(6, 16, 12, 2)])
    b = inputs.gaussian_field(op.lat.V, 3, 3)
    x, info = s.solve(b, 1e-10)
    assert info.converged == 1
    x_ref, _, res = gcr(op.M, b, tol=1e-12, maxiter=3000, nkrylov=300)
    check_solution(op, b, x, x_ref, res)


@pytest.mark.parametrize("prec", [0, 2])
def test_multi_solve_shifts(binding, prec):
    """2 sources x 3 masses in one batch; coarse operators from the lightest mass."""
    dims = (8, 4, 4, 8)
    masses = np.array([0.02, 0.05, 0.2])
    fat, naik, c, op0 = problem(dims, True, masses[0])
    s = binding.Solver(dims)
    s.set_gauge(fat, naik, c)
    s.set_mass(masses[0])
    p = binding.default_params(nvec=[6], setup_maxiter=100, precision=prec)
    s.mg_setup(p, [inputs.gaussian_fields(6, op0.lat.V, 3, 5)])
    b = inputs.gaussian_fields(2, op0.lat.V, 3, 6)
    x, infos = s.multi_solve(b, masses, 1e-10)
    assert x.shape == (3, 2, op0.lat.V, 3)
    for i, m in enumerate(masses):
        op = Staggered(op0.lat, fat, naik, c, m)
        for r in range(2):
            assert infos[i * 2 + r].converged == 1
            x_ref = dense_solution(op, b[r])
            check_solution(op, b[r], x[i, r], x_ref, 1e-13)


def test_error_paths(binding):
    dims = (8, 4, 4, 4)
    fat, naik, c, op = problem(dims, False, 0.1)
    s = binding.Solver(dims)
    b = inputs.gaussian_field(op.lat.V, 3, 1)
    with pytest.raises(binding.SmgError) as e:
        s.solve(b)
    assert e.value.code == -4          # solve before setup
    s.set_gauge(fat, naik, c)
    s.set_mass(0.1)
    with pytest.raises(binding.SmgError) as e:
        s.mg_setup(binding.default_params(agg=[(3, 4, 4, 4)], nvec=[4]), [inputs.gaussian_fields(4, op.lat.V, 3, 1)])
    assert e.value.code == -1          # aggregate does not tile
    p = binding.default_params(nvec=[4], setup_maxiter=10, max_outer=1)
    s.mg_setup(p, [inputs.gaussian_fields(4, op.lat.V, 3, 1)])
    x, info = s.solve(b, 1e-10)        # one outer iteration cannot reach 1e-10
    assert info.converged == 0 and info.iterations == 1
    r = np.linalg.norm(b - op.M(x)) / np.linalg.norm(b)
    assert abs(r - info.true_residual) <= 1e-6 * r
    with pytest.raises(binding.SmgError) as e:
        s.solve(b, 2.0)
    assert e.value.code == -1


def test_iteration_count_matches_oracle(binding):
    """Same near-null vectors on both sides (oracle CGNE output fed to the GPU
    with setup_maxiter = 0): the FP64 GPU K-cycle needs the oracle's number of
    outer iterations (rounding may move an inner stop by one step)."""
    from oracle.coarse import FineLevelOp, near_null_vectors
    from oracle.dirac import KahlerDirac
    from oracle.mg import MGParams, MultigridSolver
    dims = (8, 8, 8, 8)
    fat, naik, c, op = problem(dims, False, 0.05, seed=1003)
    phi0 = inputs.gaussian_fields(8, op.lat.V, 3, 77)
    raw, _ = near_null_vectors(FineLevelOp(KahlerDirac(op)), phi0, 1e-6, 40)
    mg = MultigridSolver(op, MGParams(agg=[(4, 4, 4, 4)], nvec=[8], setup_maxiter=0), [raw])
    b = inputs.gaussian_field(op.lat.V, 3, 78)
    x_o, it_o, res_o = mg.solve(b, 1e-10)
    s = binding.Solver(dims)
    s.set_gauge(fat, naik, c)
    s.set_mass(0.05)
    s.mg_setup(binding.default_params(nvec=[8], setup_maxiter=0), [raw])
    x, info = s.solve(b, 1e-10)
    assert info.converged == 1 and res_o <= 1e-10
    assert abs(info.iterations - it_o) <= max(2, 0.15 * it_o), (info.iterations, it_o)
    check_solution(op, b, x, x_o, res_o)


@pytest.mark.parametrize("nrhs", [1, 3])
def test_persistent_coarse_solver_matches_launch_path(binding, nrhs):
    """The cooperative single-launch coarse GCR and the launch-per-kernel path
    run the same algorithm: both converge with (nearly) the same outer count."""
    dims = (8, 8, 8, 8)
    fat, naik, c, op = problem(dims, True, 0.05, seed=1002)
    b = inputs.gaussian_fields(nrhs, op.lat.V, 3, 2002)
    its = {}
    for pers in (0, 1):
        s = binding.Solver(dims)
        s.set_gauge(fat, naik, c)
        s.set_mass(0.05)
        p = binding.default_params(n_coarse=2, agg=[(4, 4, 4, 4), (2, 2, 2, 2)], nvec=[8, 8], setup_maxiter=200,
                                   precision=binding.PREC_HALF, persistent=pers, use_graph=1)
        s.mg_setup(p, [inputs.gaussian_fields(8, op.lat.V, 3, 3002), inputs.gaussian_fields(8, 16, 16, 3003)])
        if nrhs == 1:
            x, info = s.solve(b[0], 1e-10)
            infos, xs = [info], x[None]
        else:
            x, infos = s.multi_solve(b, [0.05], 1e-10)
            xs = x[0]
        its[pers] = infos[0].iterations
        for r in range(nrhs):
            assert infos[r].converged == 1
            assert np.linalg.norm(b[r] - op.M(xs[r])) <= 1e-10 * np.linalg.norm(b[r])
    assert abs(its[0] - its[1]) <= max(2, 0.25 * max(its.values())), its


@pytest.mark.parametrize("prec", [0, 2])
def test_truncated_pseudo_fine_operator(binding, prec):
    """Table 1's truncated level-1 operator (Naik hops dropped from the
    pseudo-fine operator only, Sec. 3.1): the outer solve on the full HISQ M
    still meets 1e-10 and the dense solution; in FP64 the iteration count
    follows the oracle's solve with the same option."""
    from oracle.mg import MGParams, MultigridSolver
    dims = (8, 4, 4, 4)
    fat, naik, c, op = problem(dims, True, 0.1, seed=1011)
    phi = inputs.gaussian_fields(4, op.lat.V, 3, 3011)
    s = binding.Solver(dims)
    s.set_gauge(fat, naik, c)
    s.set_mass(0.1)
    s.mg_setup(binding.default_params(nvec=[4], setup_maxiter=50, precision=prec, truncate_naik=1), [phi])
    b = inputs.gaussian_field(op.lat.V, 3, 2011)
    x, info = s.solve(b, 1e-10)
    assert info.converged == 1 and info.true_residual <= 1e-10
    check_solution(op, b, x, dense_solution(op, b), 1e-13)
    if prec == 0:
        mg = MultigridSolver(op, MGParams(nvec=[4], setup_maxiter=50, truncate_naik=True), [phi])
        _, it_ref, _ = mg.solve(b, tol=1e-10)
        assert abs(info.iterations - it_ref) <= max(2, 0.15 * it_ref), (info.iterations, it_ref)


def test_truncated_coarse_operator(binding):
    """With the truncated option the Galerkin stencil is R A' P with
    A' = (B+m)^{-1}(m + D_fat): same raw near-null vectors on both sides."""
    from oracle.coarse import FineLevelOp, Transfer, galerkin
    from oracle.dirac import KahlerDirac
    dims = (8, 8, 8, 8)
    fat, naik, c, op = problem(dims, True, 0.1, seed=1012)
    op_fat = Staggered(op.lat, fat, None, 0.0, 0.1)
    phi = inputs.gaussian_fields(4, op.lat.V, 3, 3012)
    lop = FineLevelOp(KahlerDirac(op_fat))
    T = Transfer(op.lat, 3, lop.chirality(), (4, 4, 4, 4), phi)
    S = galerkin(lop, T)
    s = binding.Solver(dims)
    s.set_gauge(fat, naik, c)
    s.set_mass(0.1)
    s.mg_setup(binding.default_params(nvec=[4], setup_maxiter=0, precision=binding.PREC_HALF,
                                      truncate_naik=1), [phi])
    got = s.coarse_op(0)
    Vc, N = S.X.shape[0], S.X.shape[1]
    ref = np.empty((Vc, N, 9, N), dtype=np.complex128)
    ref[:, :, 0, :] = S.X
    for mu in range(4):
        ref[:, :, 1 + 2 * mu, :] = S.Yf[mu]
        ref[:, :, 2 + 2 * mu, :] = S.Yb[mu]
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)


def test_multishift_cg(binding):
    """Sec. 4's multi-shift CG: every mass of an unsorted list is solved to
    1e-10 on the full HISQ-shaped M (recomputed by the oracle) and matches the
    dense solution; the shared iteration count follows the oracle's
    multi-shift CG run to the same stopping rule."""
    from oracle.solvers import staggered_multishift
    dims = (8, 4, 4, 4)
    fat, naik, c, op = problem(dims, True, 0.1, seed=1021)
    s = binding.Solver(dims)
    s.set_gauge(fat, naik, c)
    b = inputs.gaussian_field(op.lat.V, 3, 2021)
    masses = [0.4, 0.05, 0.1, 0.2]
    x, infos = s.multishift_cg(b, masses, 1e-10)
    for m, xi, inf in zip(masses, x, infos):
        assert inf.converged == 1 and inf.true_residual <= 1e-10
        op_m = Staggered(op.lat, fat, naik, c, m)
        check_solution(op_m, b, xi, dense_solution(op_m, b), 1e-13)
    _, it_ref, res_ref = staggered_multishift(op, b, masses, tol=0.5e-10)
    assert max(res_ref) <= 1e-10
    assert abs(infos[0].iterations - it_ref) <= 2, (infos[0].iterations, it_ref)


def test_propagator_split(binding):
    """The workflow split of Sec. 4: the two lightest masses by MG (setup at
    the lightest mass, coarse operators reused), the rest by multi-shift CG;
    every result in the caller's mass order solves its own M to 1e-10."""
    dims = (8, 4, 4, 4)
    fat, naik, c, op = problem(dims, True, 0.02, seed=1022)
    s = binding.Solver(dims)
    s.set_gauge(fat, naik, c)
    s.set_mass(0.02)
    s.mg_setup(binding.default_params(nvec=[4], setup_maxiter=50, precision=binding.PREC_HALF),
               [inputs.gaussian_fields(4, op.lat.V, 3, 3022)])
    b = inputs.gaussian_field(op.lat.V, 3, 2022)
    masses = [0.2, 0.02, 0.1, 0.03, 0.4, 0.05]
    x, infos = s.propagators(b, masses, n_mg=2)
    for m, xi, inf in zip(masses, x, infos):
        assert inf.converged == 1 and inf.true_residual <= 1e-10, (m, inf.true_residual)
        op_m = Staggered(op.lat, fat, naik, c, m)
        check_solution(op_m, b, xi, dense_solution(op_m, b), 1e-13)
