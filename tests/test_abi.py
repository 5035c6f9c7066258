"""Host-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point that include/smg.h declares (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "smg.h")).read()
    return sorted(set(re.findall(r"SMG_API\s+[\w\s\*]+?\b(smg_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2212_12559_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["smg_create", "smg_set_gauge", "smg_set_mass", "smg_mg_setup", "smg_solve",
                 "smg_multi_solve", "smg_destroy", "smg_last_error"]:
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2212_12559_gb300 import binding
    assert sorted(binding.EXPORTS) == declared_symbols()


def test_params_struct_layout(libpath):
    """ctypes mirror of smg_mg_params agrees with the library's defaults."""
    from paper_2212_12559_gb300 import binding
    p = binding.default_params()
    assert p.n_coarse == 1 and list(p.agg[0]) == [4, 4, 4, 4] and p.nvec[0] == 24
    assert p.setup_tol == 1e-6 and p.setup_maxiter == 2000
    assert p.inner_tol == 0.25 and p.inner_maxiter == 8 and p.smoother_s == 8
    assert p.nkrylov == 16 and p.dense_max == 4096 and p.use_graph == 0
    assert p.persistent == 1 and p.truncate_naik == 0 and p.block_coarse == 0
    assert p.coarsest_deflate == 0 and p.coarsest_cheb_s == 8 and p.coarsest_schur == 0
    assert p.schur_coarse == 0 and p.coarsest_basis == 0


def test_create_rejects_bad_extents(libpath):
    from paper_2212_12559_gb300 import binding
    lib = binding.load()
    ctx = ctypes.c_void_p()
    for dims in [(3, 4, 4, 4), (4, 4, 4, 2), (0, 4, 4, 4)]:
        assert lib.smg_create((ctypes.c_int * 4)(*dims), ctypes.byref(ctx)) == -1
    assert lib.smg_destroy(None) == -1


def test_setup_input_sizes(libpath):
    """The start arrays smg_mg_setup reads, by level (host logic of the
    binding, which refuses short arrays before the call)."""
    from paper_2212_12559_gb300 import binding
    p = binding.default_params(n_coarse=2, agg=[(4, 4, 4, 4), (2, 2, 2, 2)], nvec=[24, 32])
    assert binding.setup_input_sizes((16, 16, 16, 16), p) == [24 * 65536 * 3, 32 * 256 * 48]
    p.coarsest_deflate = 16
    assert binding.setup_input_sizes((16, 16, 16, 16), p)[2] == (16 + 4) * 16 * 64
    p.coarsest_deflate = 40
    assert binding.deflation_block(40) == 50
    assert binding.setup_input_sizes((16, 16, 16, 16), p)[2] == 50 * 16 * 64
