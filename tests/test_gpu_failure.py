"""Failure paths on the GPU without a GPU fault: a bounded device wait that
runs out returns an error status, and the context stays usable.

The persistent coarse-level solver's grid barriers wait at most a set time;
the test hook makes every barrier expect one arrival that never comes (a flag
nothing sets) and shortens the limit to 200 microseconds.  The solve must
return SMG_ERR_TIMEOUT, and the next solve with the normal settings must
converge on the full M as usual."""
import numpy as np
import pytest

from oracle.dirac import Staggered
from oracle.lattice import Lattice
from paper_2212_12559_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_persistent_barrier_expiry_returns_timeout(lib):
    from paper_2212_12559_gb300 import binding
    dims, mass = (8, 8, 8, 8), 0.05
    thin = inputs.random_su3_links(dims, 1061)
    fat, naik, c = inputs.fat_links(thin, dims), inputs.naik_links(thin, dims), -1.0 / 24
    V = int(np.prod(dims))
    s = binding.Solver(dims)
    s.set_gauge(fat, naik, c)
    s.set_mass(mass)
    p = binding.default_params(n_coarse=2, agg=[(4, 4, 4, 4), (2, 2, 2, 2)], nvec=[6, 6], setup_maxiter=30,
                               precision=binding.PREC_HALF, persistent=1)
    s.mg_setup(p, [inputs.gaussian_fields(6, V, 3, 3061), inputs.gaussian_fields(6, 16, 12, 3062)])
    b = inputs.gaussian_field(V, 3, 2061)
    s.debug_persist_barrier(200_000, 1)
    with pytest.raises(binding.SmgError) as e:
        s.solve(b, 1e-10)
    assert e.value.code == -7 and "timeout" in str(e.value)
    with pytest.raises(binding.SmgError):
        s.debug_persist_barrier(10, 0)       # below the 1 us floor: refused
    s.debug_persist_barrier(2_000_000_000, 0)
    x, info = s.solve(b, 1e-10)
    assert info.converged == 1
    op = Staggered(Lattice(dims), fat, naik, c, mass)
    assert np.linalg.norm(b - op.M(x)) / np.linalg.norm(b) <= 1e-10
