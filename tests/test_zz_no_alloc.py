"""The inner-product entry point that allocates nothing (smg_dot_noalloc).

Callers whose device heap is owned by another allocator, or whose inner loops
cannot take cudaMalloc's implicit synchronisation, use it.  Checked here
through the C ABI against the existing entry point that reduces with the
context's allocated scratch: smg_fermion_action returns S = <Y, Y> and
dS/dm = -2 m <X, X>; the same sums from smg_dot_noalloc, on two calls in a
row, must agree to rounding (1e-12 relative).  Collected after the solver tests.
"""
import numpy as np
import pytest

from paper_2212_12559_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_dot_noalloc_matches_fermion_action(lib):
    import torch
    from paper_2212_12559_gb300 import binding
    dims = (8, 4, 4, 8)
    m = 0.05
    V = int(np.prod(dims))
    s = binding.Solver(dims)
    s.set_gauge(inputs.random_su3_links(dims, 1005))
    s.set_mass(m)
    s.mg_setup(binding.default_params(nvec=[4], setup_maxiter=30), [inputs.gaussian_fields(4, V, 3, 3005)])
    dev = torch.device("cuda")
    phi = torch.from_numpy(inputs.gaussian_field(V, 3, 2005)).to(dev)
    S, dSdm, X, Y, infos = s.fermion_action(phi, 1e-10)
    assert all(i.converged for i in infos)
    out = torch.zeros(2, dtype=torch.complex128, device=dev)
    s.dot_noalloc(Y[None], Y[None], out[0:1])     # first call: <Y, Y>
    s.dot_noalloc(X[None], X[None], out[1:2])     # second call: <X, X>
    torch.cuda.synchronize()
    yy, xx = out.cpu().numpy()
    assert abs(yy.real - S) <= 1e-12 * abs(S) and abs(yy.imag) <= 1e-12 * abs(S)
    assert abs(-2 * m * xx.real - dSdm) <= 1e-12 * abs(dSdm)
    # batched form: both sums in one call, twice in a row, same answer
    XY = torch.stack([Y, X])
    for _ in range(2):
        out2 = torch.zeros(2, dtype=torch.complex128, device=dev)
        s.dot_noalloc(XY, XY, out2)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out2.cpu().numpy(), [yy, xx], rtol=1e-12)
    # sizes beyond the fixed scratch are refused with a clear error
    with pytest.raises(binding.SmgError) as e:
        s._check(s.lib.smg_dot_noalloc(s.ctx, Y.data_ptr(), Y.data_ptr(), 1, 8193, out.data_ptr()))
    assert e.value.code == -1 and "8192" in str(e.value)
