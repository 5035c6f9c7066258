"""Checkpoint of the multigrid setup through the C ABI (smg_save_setup /
smg_load_setup): Sec. 3.2 generates the near-null and singular vectors once
and reuses them for later solves.  A setup saved and loaded into a fresh
context with the same gauge field and mass gives bit-identical near-null
vectors, coarse stencils and deflation, and the same solve; damaged or
mismatched files are refused."""
import numpy as np
import pytest

from paper_2212_12559_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding(lib):
    from paper_2212_12559_gb300 import binding as b
    return b


def hisq(dims, seed):
    thin = inputs.random_su3_links(dims, seed)
    return inputs.fat_links(thin, dims), inputs.naik_links(thin, dims), -1.0 / 24


def fresh(binding, dims, links, mass):
    s = binding.Solver(dims)
    s.set_gauge(*links)
    s.set_mass(mass)
    return s


def test_save_load_three_level_mixed(binding, tmp_path):
    """Three levels, FP16 storage, near-null vectors from 40 CGNE iterations:
    the reloaded context holds the same vectors and stencils bit for bit and
    solves the same system in the same iterations to the same bits."""
    dims, mass = (8, 8, 8, 8), 0.05
    links = hisq(dims, 1041)
    V = int(np.prod(dims))
    p = dict(n_coarse=2, agg=[(4, 4, 4, 4), (2, 2, 2, 2)], nvec=[6, 6], setup_maxiter=40,
             precision=2, use_graph=1)
    s = fresh(binding, dims, links, mass)
    s.mg_setup(binding.default_params(**p), [inputs.gaussian_fields(6, V, 3, 3041),
                                             inputs.gaussian_fields(6, 16, 12, 3042)])
    b = inputs.gaussian_field(V, 3, 2041)
    x0, i0 = s.solve(b, 1e-10)
    path = tmp_path / "setup.smg"
    s.save_setup(path)
    t = fresh(binding, dims, links, mass)
    t.load_setup(path)
    for l in range(2):
        assert np.array_equal(t.null_vectors(l), s.null_vectors(l))
        assert np.array_equal(t.coarse_op(l), s.coarse_op(l))
        assert t.setup_iterations(l) == s.setup_iterations(l)
    x1, i1 = t.solve(b, 1e-10)
    assert i1.converged == 1 and i1.iterations == i0.iterations
    assert np.array_equal(x1, x0)


def test_save_load_deflated_coarsest(binding, tmp_path):
    """With Table 1's deflated coarsest level the singular values and vectors
    come back as saved (no subspace iteration on load) and the FP64 solve
    repeats bit for bit."""
    from oracle.coarse import FineLevelOp, near_null_vectors
    from oracle.dirac import KahlerDirac, Staggered
    from oracle.lattice import Lattice
    dims, mass = (8, 8, 4, 4), 0.1
    thin = inputs.random_su3_links(dims, 1003)
    op = Staggered(Lattice(dims), thin, None, 0.0, mass)
    raw, _ = near_null_vectors(FineLevelOp(KahlerDirac(op)), inputs.gaussian_fields(4, op.lat.V, 3, 3004), 1e-6, 50)
    k = 8
    start = inputs.gaussian_fields(binding.deflation_block(k), 4, 8, 3005)
    prm = binding.default_params(nvec=[4], setup_maxiter=0, dense_max=0, coarsest_deflate=k)
    s = fresh(binding, dims, (thin, None, 0.0), mass)
    s.mg_setup(prm, [raw, start])
    b = inputs.gaussian_field(op.lat.V, 3, 2003)
    x0, i0 = s.solve(b, 1e-10)
    path = tmp_path / "defl.smg"
    s.save_setup(path)
    t = fresh(binding, dims, (thin, None, 0.0), mass)
    t.load_setup(path)
    sig0, inf0 = s.deflation()
    sig1, inf1 = t.deflation()
    assert np.array_equal(sig0, sig1) and inf0 == inf1
    assert np.array_equal(t.coarse_op(0), s.coarse_op(0))
    x1, i1 = t.solve(b, 1e-10)
    assert i1.iterations == i0.iterations and np.array_equal(x1, x0)


def test_load_refuses_bad_files(binding, tmp_path):
    """A file for other extents, a flipped byte (hash), a truncated file and
    a missing file are refused with SMG_ERR_ARG; a save before any setup is
    SMG_ERR_STATE."""
    dims, mass = (8, 4, 4, 8), 0.1
    V = int(np.prod(dims))
    links = (inputs.random_su3_links(dims, 1051), None, 0.0)
    s = fresh(binding, dims, links, mass)
    with pytest.raises(binding.SmgError) as e:
        s.save_setup(tmp_path / "none.smg")
    assert e.value.code == -4
    s.mg_setup(binding.default_params(nvec=[4], setup_maxiter=5), [inputs.gaussian_fields(4, V, 3, 3051)])
    good = tmp_path / "good.smg"
    s.save_setup(good)
    data = good.read_bytes()
    flipped = tmp_path / "flipped.smg"
    mid = len(data) // 2          # inside the near-null vectors
    flipped.write_bytes(data[:mid] + bytes([data[mid] ^ 1]) + data[mid + 1:])
    short = tmp_path / "short.smg"
    short.write_bytes(data[:-100])
    other = fresh(binding, (8, 8, 4, 4), (inputs.random_su3_links((8, 8, 4, 4), 1052), None, 0.0), mass)
    for ctx, path, msg in ((s, flipped, "checksum"), (s, short, "truncated"), (other, good, "extents"),
                           (s, tmp_path / "missing.smg", "cannot open")):
        with pytest.raises(binding.SmgError) as e:
            ctx._check(ctx.lib.smg_load_setup(ctx.ctx, str(path).encode(), None))
        assert e.value.code == -1 and msg in str(e.value), str(e.value)
    s.load_setup(good)
    # other solver settings on the same vectors; another level structure is refused
    s.load_setup(good, binding.default_params(nvec=[4], precision=binding.PREC_HALF, inner_tol=0.1))
    with pytest.raises(binding.SmgError) as e:
        s.load_setup(good, binding.default_params(nvec=[6]))
    assert e.value.code == -1 and "level structure" in str(e.value)
