"""The autotuner's candidates all compute the same operator.

For each kernel family with several launch shapes (systems per CTA of the
dslash and the KD block apply; kernel and systems per CTA of restriction
and prolongation; the coarse apply's
kernels are checked one by one in test_gpu_coarse_shapes), a first call lets the tuner time the candidates and record its
choice; then every candidate in turn is forced through the table
(smg_tune_load of "key<TAB>id") and its output compared with the oracle's
operator, per system, at the storage precision's bar.  Bars as in
test_gpu_ops: FP32 arithmetic on FP16 storage within 5e-3 of the relative
2-norm and of max |error| / max |ref|.
"""
import numpy as np
import pytest

from oracle.coarse import FineLevelOp, Transfer, galerkin
from oracle.dirac import KahlerDirac, Staggered
from oracle.lattice import Lattice
from paper_2212_12559_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 5e-3


@pytest.fixture(scope="module")
def binding(lib):
    from paper_2212_12559_gb300 import binding as b
    return b


def err(a, b):
    d = np.abs(a - b)
    return max(np.linalg.norm(d) / np.linalg.norm(b), d.max() / np.abs(b).max())


def forced(binding, tmp_path, family, run, check, want=None):
    """run() once with tuning on, take the key the family recorded, then run
    and check every candidate of that key forced through the table (`want`:
    a candidate id that must be among them)."""
    binding.tune_clear()
    binding.tune_mode(1)
    run()
    rows = [r for r in binding.tune_table() if r[0].startswith(family + " ")]
    assert rows, (family, binding.tune_table())
    key, chosen, _, times = rows[0]
    ids = {"1 system/CTA": 1, "2 systems/CTA": 2, "4 systems/CTA": 4, "8 systems/CTA": 8, "16 systems/CTA": 16,
           "aggregate CTA, 1 system": 17, "aggregate CTA, 2 systems": 18, "aggregate CTA, 4 systems": 20,
           "aggregate CTA, 8 systems": 24, "tensor cores, 16 systems/CTA": 32,
           "2 rows/thread, 1 system/CTA": 33, "2 rows/thread, 2 systems/CTA": 34,
           "2 rows/thread, 4 systems/CTA": 36, "2 rows/thread, 8 systems/CTA": 40,
           "2 rows/thread, 16 systems/CTA": 48}
    cands = [ids[n] for n in times]
    assert len(cands) >= 2 and chosen in cands, (key, times)
    assert want is None or want in cands, (key, times)
    f = tmp_path / "t.txt"
    for cid in cands:
        binding.tune_clear()
        f.write_text(f"{key}\t{cid}\n")
        binding.tune_load(f)
        check(run(), cid)
        assert [r[1] for r in binding.tune_table() if r[0] == key] == [cid]
    binding.tune_clear()


@pytest.mark.parametrize("hisq,nsys", [(False, 5), (True, 5), (False, 12), (True, 12)])
def test_fine_kernels_every_candidate(binding, tmp_path, hisq, nsys):
    """12 systems bring the 16-systems-per-CTA candidates in (one group)."""
    dims, mass = (8, 4, 6, 10), 0.05
    thin = inputs.random_su3_links(dims, 7)
    if hisq:
        fat, naik, c = inputs.fat_links(thin, dims), inputs.naik_links(thin, dims), -1 / 24
    else:
        fat, naik, c = thin, None, 0.0
    op = Staggered(Lattice(dims), fat, naik, c, mass)
    kd = KahlerDirac(op)
    s = binding.Solver(dims)
    s.set_gauge(fat, naik, c)
    s.set_mass(mass)
    v = inputs.gaussian_fields(nsys, op.lat.V, 3, 11)
    for fam, opid, ref in (("hop_dslash", binding.OP_M, op.M), ("kd_apply", binding.OP_KD, kd.apply_inv)):
        want = [ref(v[k]) for k in range(nsys)]

        def check(out, cid, want=want, fam=fam):
            for k in range(nsys):
                assert err(out[k], want[k]) <= TOL, (fam, cid, k)
        forced(binding, tmp_path, fam, lambda opid=opid: s.apply(opid, v, binding.PREC_HALF), check)


def test_transfer_every_candidate(binding, tmp_path):
    dims, mass, nsys = (8, 8, 8, 8), 0.1, 5
    thin = inputs.random_su3_links(dims, 8)
    op = Staggered(Lattice(dims), thin, None, 0.0, mass)
    lat = op.lat
    phi = inputs.gaussian_fields(8, lat.V, 3, 31)
    lop = FineLevelOp(KahlerDirac(op))
    T = Transfer(lat, 3, lop.chirality(), (4, 4, 4, 4), phi)
    s = binding.Solver(dims)
    s.set_gauge(thin)
    s.set_mass(mass)
    s.mg_setup(binding.default_params(nvec=[8], setup_maxiter=0, precision=binding.PREC_HALF), [phi])
    v = inputs.gaussian_fields(nsys, lat.V, 3, 5)
    vc = inputs.gaussian_fields(nsys, 16, 16, 6)
    wr = [T.restrict(v[k]) for k in range(nsys)]
    wp = [T.prolong(vc[k]) for k in range(nsys)]

    def check_r(out, cid):
        for k in range(nsys):
            assert err(out[k], wr[k]) <= TOL, ("restrict", cid, k)

    def check_p(out, cid):
        for k in range(nsys):
            assert err(out[k], wp[k]) <= TOL, ("prolong", cid, k)
    forced(binding, tmp_path, "restrict", lambda: s.restrict(0, v, binding.PREC_HALF), check_r)
    forced(binding, tmp_path, "prolong", lambda: s.prolong(0, vc, binding.PREC_HALF), check_p)


@pytest.mark.parametrize("nsys", [5, 18])
def test_transfer_mma_every_candidate(binding, tmp_path, nsys):
    """With 32 near-null vectors the transfers of both coarsenings offer the
    tensor-core kernel: the fine one (4^4 aggregates, chirality = site
    parity) and the second one (2^4 aggregates of the 2^4 level-1 lattice,
    chirality = upper or lower half of the 64 components).  18 systems take
    two 16-system groups.  Every candidate matches the oracle's transfer of
    the same block-orthonormalised vectors at the FP16 bar."""
    dims, mass, nv = (8, 8, 8, 8), 0.1, 32
    thin = inputs.random_su3_links(dims, 9)
    op = Staggered(Lattice(dims), thin, None, 0.0, mass)
    lat = op.lat
    phi0 = inputs.gaussian_fields(nv, lat.V, 3, 41)
    phi1 = inputs.gaussian_fields(nv, 16, 2 * nv, 42)
    T0 = Transfer(lat, 3, FineLevelOp(KahlerDirac(op)).chirality(), (4, 4, 4, 4), phi0)
    clat = Lattice((2, 2, 2, 2))
    chi1 = np.broadcast_to((np.arange(2 * nv) >= nv).astype(np.int64), (clat.V, 2 * nv)).copy()
    T1 = Transfer(clat, 2 * nv, chi1, (2, 2, 2, 2), phi1)
    s = binding.Solver(dims)
    s.set_gauge(thin)
    s.set_mass(mass)
    s.mg_setup(binding.default_params(n_coarse=2, agg=[(4, 4, 4, 4), (2, 2, 2, 2)], nvec=[nv, nv], setup_maxiter=0,
                                      precision=binding.PREC_HALF), [phi0, phi1])
    for lvl, T in ((0, T0), (1, T1)):
        v = inputs.gaussian_fields(nsys, T.lat.V, T.n, 50 + lvl)
        vc = inputs.gaussian_fields(nsys, T.coarse_lat.V, T.N, 60 + lvl)
        v[1] *= 1e-7          # a system far from unit scale
        vc[2] *= 3e5
        wr = [T.restrict(v[k]) for k in range(nsys)]
        wp = [T.prolong(vc[k]) for k in range(nsys)]

        def check_r(out, cid, wr=wr, lvl=lvl):
            for k in range(nsys):
                assert err(out[k], wr[k]) <= TOL, ("restrict", lvl, cid, k)

        def check_p(out, cid, wp=wp, lvl=lvl):
            for k in range(nsys):
                assert err(out[k], wp[k]) <= TOL, ("prolong", lvl, cid, k)

        def run_r(lvl=lvl, v=v):
            return s.restrict(lvl, v, binding.PREC_HALF)

        def run_p(lvl=lvl, vc=vc):
            return s.prolong(lvl, vc, binding.PREC_HALF)
        forced(binding, tmp_path, "restrict", run_r, check_r, want=32)
        forced(binding, tmp_path, "prolong", run_p, check_p, want=32)
