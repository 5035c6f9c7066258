"""The coarse apply (Sec. 3.1) at the shapes the benchmark launches, every
kernel the autotuner can pick, against the oracle's 9-point stencil.

The stencil and vectors are seeded Gaussian data of the coarse level's shape
(N = 128 as on the 32^4 workload's coarse level, N = 48 as on the 24^3 x 48
and 16^4 ones); the lattices give the persistent tcgen05 kernel two or more
sites per CTA (4 x 4 x 4 x 10 = 640 sites against 304 or 152 CTAs), so the
walk from one site to the next (scale pass, stencil ring, epilogue) is
checked, not only a single site.  Bars: per element, max |out - ref| /
max |ref|, and per system, the relative 2-norm error: FP64 1e-12, FP32 1e-6,
FP16 storage 5e-3.
"""
import numpy as np
import pytest

from oracle.coarse import CoarseStencil
from oracle.lattice import Lattice
from paper_2212_12559_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6, 2: 5e-3}


@pytest.fixture(scope="module")
def binding(lib):
    from paper_2212_12559_gb300 import binding as b
    return b


def oracle_apply(cdims, S, v):
    """CoarseStencil.apply per system; the stencil blocks are taken from the
    [site][row][direction][column] layout."""
    lat = Lattice(cdims)
    st = CoarseStencil(lat, S[:, :, 0, :], np.stack([S[:, :, 1 + 2 * mu, :] for mu in range(4)]),
                       np.stack([S[:, :, 2 + 2 * mu, :] for mu in range(4)]))
    return np.stack([st.apply(v[k]) for k in range(v.shape[0])])


@pytest.mark.parametrize("cdims,N,nsys", [((4, 4, 4, 10), 128, 12), ((4, 4, 4, 10), 128, 1),
                                          ((4, 4, 4, 6), 48, 12), ((4, 4, 4, 6), 48, 1)])
def test_coarse_apply_every_kernel(binding, cdims, N, nsys):
    import torch
    Vc = int(np.prod(cdims))
    g = inputs.rng(4000 + N + nsys)
    S = (g.standard_normal((Vc, N, 9, N)) + 1j * g.standard_normal((Vc, N, 9, N))) / np.sqrt(9 * N)
    v = g.standard_normal((nsys, Vc, N)) + 1j * g.standard_normal((nsys, Vc, N))
    ref = oracle_apply(cdims, S, v)
    dev = torch.device("cuda")
    Sd = torch.from_numpy(S).to(dev)
    vd = torch.from_numpy(v).to(dev)
    del S
    s = binding.Solver((4, 4, 4, 4))
    seen = []
    for prec in (0, 1, 2):
        paths = binding.coarse_paths(N, nsys, prec)
        for path in paths + [binding.COARSE_AUTO]:
            out = s.coarse_apply_stencil(cdims, Sd, vd, prec, path).cpu().numpy()
            d = np.abs(out - ref)
            elem = d.max() / np.abs(ref).max()
            assert elem <= TOL[prec], (prec, path, elem)
            for k in range(nsys):
                r = np.linalg.norm(out[k] - ref[k]) / np.linalg.norm(ref[k])
                assert r <= TOL[prec], (prec, path, k, r)
            seen.append((prec, path))
    if N == 128 and nsys > 1:
        assert (2, binding.COARSE_TC_2x4) in seen and (2, binding.COARSE_TC_1x6) in seen
    # the tuner recorded a choice for the multi-kernel shape
    if nsys > 1:
        keys = [row[0] for row in binding.tune_table()]
        assert any(f"V={Vc} N={N} nsys={nsys}" in k for k in keys), keys
