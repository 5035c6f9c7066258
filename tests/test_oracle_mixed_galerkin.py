"""The FP16 bar of the mixed-precision Galerkin product, derived on the CPU.

In mixed precision the GPU builds A_hat = R A P from the FP16 prolongator
the K-cycle applies, with A P rounded to FP16 inside the tensor-core
restriction (FP32 sums).  Here the oracle's FP64 product is recomputed with
the prolongator rounded to FP16 (|P| <= 1 after block orthonormalisation,
so no scale is needed): the stencil moves by about 1e-4 relative, per
element and in norm.  The rounding of A P adds an error of the same order,
so the GPU test's bar of 5e-3 leaves a margin of more than ten.
"""
import numpy as np

from oracle.coarse import FineLevelOp, Transfer, galerkin
from oracle.dirac import KahlerDirac, Staggered
from oracle.lattice import Lattice
from paper_2212_12559_gb300 import inputs


def layout(S):
    return np.stack([S.X] + [S.Yf[m] for m in range(4)] + [S.Yb[m] for m in range(4)])


def test_fp16_prolongator_moves_the_stencil_by_about_1e_4():
    dims, nv = (8, 8, 8, 8), 32
    thin = inputs.random_su3_links(dims, 21)
    fat, naik, c = inputs.fat_links(thin, dims), inputs.naik_links(thin, dims), -1 / 24
    op = Staggered(Lattice(dims), fat, naik, c, 0.1)
    lop = FineLevelOp(KahlerDirac(op))
    phi = inputs.gaussian_fields(nv, op.lat.V, 3, 71)
    T = Transfer(op.lat, 3, lop.chirality(), (4, 4, 4, 4), phi)
    assert np.abs(T.P).max() <= 1.0 + 1e-12
    T16 = Transfer(op.lat, 3, lop.chirality(), (4, 4, 4, 4), phi)
    T16.P = T.P.real.astype(np.float16).astype(np.float64) + 1j * T.P.imag.astype(np.float16).astype(np.float64)
    a, b = layout(galerkin(lop, T16)), layout(galerkin(lop, T))
    d = np.abs(a - b)
    norm_err = np.linalg.norm(d) / np.linalg.norm(b)
    elem_err = d.max() / np.abs(b).max()
    assert 1e-6 < norm_err < 5e-4 and elem_err < 5e-4, (norm_err, elem_err)
