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
    assert p.coarse_inner_tol == 0.0 and p.coarse_inner_maxiter == 0 and p.galerkin_tc == 1
    assert ctypes.sizeof(p) == ctypes.sizeof(binding.MGParams)


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


C_CLIENT = r"""
#include <stdio.h>
#include "smg.h"
int main(void) {
  smg_mg_params p;
  long long plan[10];
  smg_default_params(&p);
  if (smg_persist_plan(256, 48, 1, 32, SMG_PREC_HALF, 152, 232448, plan) != SMG_OK) return 2;
  printf("%d %d %d %d %d %d %lld %lld %lld %d\n", p.n_coarse, p.nvec[0], p.inner_maxiter, p.coarsest_cheb_s,
         p.block_coarse, p.coarsest_basis, plan[0], plan[1], plan[2], (int)sizeof(smg_mg_params));
  return 0;
}
"""


def test_plain_c_client(libpath, tmp_path):
    """The boundary is a C ABI: a C99 program built against include/smg.h and
    linked to libsmg.so reads the defaults and a persistent launch plan (host
    only, no GPU call) exactly as the Python binding does."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(libpath)
    cudalib = "/usr/local/cuda/lib64"
    cmd = [cc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"), str(src),
           "-o", str(exe), f"-L{libdir}", "-lsmg", f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{cudalib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    from paper_2212_12559_gb300 import binding
    p = binding.default_params()
    q = binding.persist_plan(256, 48, 1, 32, binding.PREC_HALF, 152, 232448)
    want = [p.n_coarse, p.nvec[0], p.inner_maxiter, p.coarsest_cheb_s, p.block_coarse, p.coarsest_basis,
            q["grid"], q["per"], q["nslot"], ctypes.sizeof(binding.MGParams)]
    assert [int(v) for v in r.stdout.split()] == want


def test_dot_noalloc_argument_checks():
    """The binding refuses, before any pointer reaches the library, the
    tensors that would make the no-allocation reduction read or write outside
    the caller's buffers: a narrower dtype, a strided view, a y of another
    shape, an out shorter than nsys, host memory (host-only checks)."""
    import torch
    from paper_2212_12559_gb300.binding import check_dot_noalloc_args
    x = torch.zeros(2, 8, dtype=torch.complex128)
    out = torch.zeros(2, dtype=torch.complex128)
    cases = [
        (x.to(torch.complex64), x, out, "complex128"),
        (x, x, out.to(torch.complex64), "complex128"),
        (torch.zeros(8, 2, dtype=torch.complex128).t(), x, out, "contiguous"),
        (x, torch.zeros(2, 7, dtype=torch.complex128), out, "shape"),
        (x, x, torch.zeros(1, dtype=torch.complex128), "nsys entries"),
        (x, x, out, "CUDA"),
        (x.numpy(), x, out, "torch tensor"),
        (torch.zeros(0, 8, dtype=torch.complex128), torch.zeros(0, 8, dtype=torch.complex128), out, "non-empty"),
    ]
    for a, b, o, msg in cases:
        with pytest.raises(ValueError, match=msg):
            check_dot_noalloc_args(a, b, o)
