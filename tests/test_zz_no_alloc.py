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


@pytest.mark.parametrize("nsys,n", [(1, 1 << 20), (64, 1 << 16)])
def test_dot_noalloc_block_caps(lib, nsys, n):
    """The two caps on the CTAs per system: 304 CTAs for one long system
    (2^20 entries), 8192 / 64 = 128 CTAs for 64 systems, where the partial
    sums fill the fixed array to its end.  Every row agrees with torch.vdot to
    1e-12 and two calls in a row give identical bits (fixed summation order,
    arrival counter back at zero after each call)."""
    import torch
    from paper_2212_12559_gb300 import binding
    dev = torch.device("cuda")
    s = binding.Solver((4, 4, 4, 4))
    g = torch.Generator(device="cpu").manual_seed(nsys)
    x = torch.randn(nsys, n, dtype=torch.complex128, generator=g).to(dev)
    y = torch.randn(nsys, n, dtype=torch.complex128, generator=g).to(dev)
    ref = torch.stack([torch.vdot(x[i], y[i]) for i in range(nsys)]).cpu().numpy()
    outs = []
    for _ in range(2):
        out = torch.zeros(nsys, dtype=torch.complex128, device=dev)
        s.dot_noalloc(x, y, out)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    # rounding of a sum of n products is bounded by a multiple of eps |x_i| |y_i|
    for i in range(nsys):
        assert abs(outs[0][i] - ref[i]) <= 1e-12 * float(torch.linalg.norm(x[i]) * torch.linalg.norm(y[i]))
    assert np.array_equal(outs[0], outs[1])


def test_dot_noalloc_refuses_misaligned(lib):
    """A pointer that is not 16-byte aligned (a view starting at an imaginary
    part) is refused with SMG_ERR_ARG before anything is launched."""
    import torch
    from paper_2212_12559_gb300 import binding
    dev = torch.device("cuda")
    s = binding.Solver((4, 4, 4, 4))
    x = torch.zeros(2, 64, dtype=torch.complex128, device=dev)
    out = torch.zeros(2, dtype=torch.complex128, device=dev)
    with pytest.raises(binding.SmgError) as e:
        s._check(s.lib.smg_dot_noalloc(s.ctx, x.data_ptr() + 8, x.data_ptr(), 32, 1, out.data_ptr()))
    assert e.value.code == -1 and "16-byte" in str(e.value)

