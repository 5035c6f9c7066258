"""Python binding of libsmg's C ABI (argument marshalling only).

Every numeric step runs inside the CUDA library; this module converts
numpy arrays (host memory) or torch CUDA tensors (device memory) into
pointers and back.  There is no fallback: if libsmg.so cannot be loaded the
calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsmg.so")

SMG_HOST, SMG_DEVICE = 0, 1
PREC_DOUBLE, PREC_SINGLE, PREC_HALF = 0, 1, 2
OP_M, OP_MDAG, OP_KD, OP_KDDAG, OP_A, OP_ADAG = range(6)
K_DSLASH, K_KD, K_RESTRICT, K_PROLONG, K_COARSE, K_A, K_COARSE_SOLVE = range(7)
BC_T_ANTIPERIODIC = 1
MAX_COARSE = 3
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_OOM", -4: "ERR_STATE",
          -5: "ERR_NOT_CONVERGED", -6: "ERR_BREAKDOWN", -7: "ERR_TIMEOUT"}

EXPORTS = ["smg_default_params", "smg_create", "smg_destroy", "smg_last_error", "smg_set_stream",
           "smg_set_gauge", "smg_set_mass", "smg_mg_setup", "smg_solve", "smg_multi_solve",
           "smg_apply_fine", "smg_get_maps", "smg_get_kd_inverse", "smg_get_null_vectors",
           "smg_get_coarse_op", "smg_restrict", "smg_prolong", "smg_coarse_apply", "smg_force",
           "smg_setup_iterations", "smg_time_kernel", "smg_kernel_launches", "smg_fermion_action", "smg_dot_noalloc",
           "smg_bench_coarse_apply", "smg_multishift_cg", "smg_propagators", "smg_persist_plan",
           "smg_get_coarse_xinv", "smg_get_deflation", "smg_coarse_solve", "smg_save_setup", "smg_load_setup",
           "smg_coarse_apply_stencil", "smg_coarse_paths", "smg_tune_mode", "smg_tune_table", "smg_tune_save",
           "smg_tune_load", "smg_tune_clear", "smg_debug_persist_barrier", "smg_setup_times",
           "smg_set_boundary"]


class MGParams(ctypes.Structure):
    _fields_ = [
        ("n_coarse", ctypes.c_int),
        ("agg", (ctypes.c_int * 4) * MAX_COARSE),
        ("nvec", ctypes.c_int * MAX_COARSE),
        ("setup_tol", ctypes.c_double),
        ("setup_maxiter", ctypes.c_int),
        ("inner_tol", ctypes.c_double),
        ("inner_maxiter", ctypes.c_int),
        ("smoother_s", ctypes.c_int),
        ("dense_max", ctypes.c_int),
        ("nkrylov", ctypes.c_int),
        ("max_outer", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("persistent", ctypes.c_int),
        ("truncate_naik", ctypes.c_int),
        ("block_coarse", ctypes.c_int),
        ("coarsest_deflate", ctypes.c_int),
        ("coarsest_cheb_s", ctypes.c_int),
        ("coarsest_schur", ctypes.c_int),
        ("schur_coarse", ctypes.c_int),
        ("coarsest_basis", ctypes.c_int),
        ("coarse_inner_tol", ctypes.c_double),
        ("coarse_inner_maxiter", ctypes.c_int),
        ("galerkin_tc", ctypes.c_int),
    ]


class SolveInfo(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("true_residual", ctypes.c_double), ("seconds", ctypes.c_double)]


class SmgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libsmg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libsmg.so not found at {path}; build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    ip = ctypes.POINTER(ctypes.c_int)
    sig = {
        "smg_default_params": (None, [ctypes.POINTER(MGParams)]),
        "smg_create": (i, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(vp)]),
        "smg_destroy": (i, [vp]),
        "smg_last_error": (ctypes.c_char_p, [vp]),
        "smg_set_stream": (i, [vp, vp]),
        "smg_set_gauge": (i, [vp, vp, vp, d, i]),
        "smg_set_mass": (i, [vp, d]),
        "smg_mg_setup": (i, [vp, ctypes.POINTER(MGParams), ctypes.POINTER(vp), i]),
        "smg_solve": (i, [vp, vp, vp, d, i, ctypes.POINTER(SolveInfo)]),
        "smg_coarse_apply_stencil": (i, [vp, ctypes.POINTER(ctypes.c_int), i, i, i, vp, i, vp, vp, i]),
        "smg_coarse_paths": (i, [i, i, i, ip, i]),
        "smg_tune_mode": (i, [i]),
        "smg_debug_persist_barrier": (i, [vp, ctypes.c_longlong, i]),
        "smg_tune_table": (ctypes.c_longlong, [ctypes.c_char_p, ctypes.c_longlong]),
        "smg_tune_save": (i, [ctypes.c_char_p]),
        "smg_tune_load": (i, [ctypes.c_char_p]),
        "smg_tune_clear": (i, []),
        "smg_save_setup": (i, [vp, ctypes.c_char_p]),
        "smg_load_setup": (i, [vp, ctypes.c_char_p, ctypes.POINTER(MGParams)]),
        "smg_multi_solve": (i, [vp, i, vp, i, ctypes.POINTER(d), vp, d, i, ctypes.POINTER(SolveInfo)]),
        "smg_multishift_cg": (i, [vp, vp, i, ctypes.POINTER(d), vp, d, i, i, ctypes.POINTER(SolveInfo)]),
        "smg_persist_plan": (i, [i, i, i, i, i, i, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]),
        "smg_propagators": (i, [vp, vp, i, ctypes.POINTER(d), i, vp, d, i, i, ctypes.POINTER(SolveInfo)]),
        "smg_apply_fine": (i, [vp, i, i, i, vp, vp, i]),
        "smg_get_maps": (i, [vp, ip, ip, ip, ip, ip, ip, i]),
        "smg_get_kd_inverse": (i, [vp, vp, i]),
        "smg_get_null_vectors": (i, [vp, i, vp, i]),
        "smg_get_coarse_op": (i, [vp, i, vp, i]),
        "smg_get_coarse_xinv": (i, [vp, i, vp, i]),
        "smg_get_deflation": (i, [vp, vp, vp]),
        "smg_coarse_solve": (i, [vp, i, i, vp, vp, i]),
        "smg_restrict": (i, [vp, i, i, i, vp, vp, i]),
        "smg_prolong": (i, [vp, i, i, i, vp, vp, i]),
        "smg_coarse_apply": (i, [vp, i, i, i, vp, vp, i]),
        "smg_force": (i, [vp, vp, vp, i, vp, i]),
        "smg_setup_iterations": (i, [vp, i, ip]),
        "smg_setup_times": (i, [vp, i, ctypes.POINTER(d)]),
        "smg_set_boundary": (i, [vp, i]),
        "smg_time_kernel": (i, [vp, i, i, i, i, ctypes.POINTER(d)]),
        "smg_kernel_launches": (ctypes.c_longlong, []),
        "smg_fermion_action": (i, [vp, vp, vp, vp, d, i, ctypes.POINTER(d), ctypes.POINTER(d),
                                   ctypes.POINTER(SolveInfo)]),
        "smg_dot_noalloc": (i, [vp, vp, vp, ctypes.c_longlong, i, vp]),
        "smg_bench_coarse_apply": (i, [vp, ctypes.POINTER(ctypes.c_int), i, i, i, i, ctypes.POINTER(d)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def kernel_launches() -> int:
    return int(load().smg_kernel_launches())


(COARSE_AUTO, COARSE_CORES, COARSE_MMA, COARSE_TC_1x4, COARSE_TC_2x4, COARSE_TC_1x6, COARSE_ROWS,
 COARSE_ROWS_MULTI) = range(8)


def coarse_paths(N, nsys, prec):
    """Coarse-apply kernels (COARSE_*) that serve a shape, the untuned default first (host only)."""
    out = (ctypes.c_int * 8)()
    n = load().smg_coarse_paths(int(N), int(nsys), int(prec), out, 8)
    if n < 0:
        raise SmgError(n, "coarse_paths: bad arguments")
    return list(out)[:n]


def tune_mode(mode):
    rc = load().smg_tune_mode(int(mode))
    if rc != 0:
        raise SmgError(rc, "tune_mode: 0 or 1")


def tune_table():
    """The autotuner's table: list of (key, path id, name, {candidate: ms})."""
    lib = load()
    need = lib.smg_tune_table(None, 0)
    buf = ctypes.create_string_buffer(int(need))
    lib.smg_tune_table(buf, need)
    rows = []
    for line in buf.value.decode().splitlines():
        f = line.split("\t")
        times = {}
        for t in f[3:]:
            k, _, v = t.rpartition("=")
            times[k] = float(v)
        rows.append((f[0], int(f[1]), f[2] if len(f) > 2 else "", times))
    return rows


def tune_save(path):
    rc = load().smg_tune_save(os.fsencode(path))
    if rc != 0:
        raise SmgError(rc, f"tune_save: cannot write {path}")


def tune_load(path):
    rc = load().smg_tune_load(os.fsencode(path))
    if rc != 0:
        raise SmgError(rc, f"tune_load: cannot read {path}")


def tune_clear():
    load().smg_tune_clear()


def persist_plan(V, N, nsys, nvec_next, prec, sms, smem_cap):
    """Launch plan of the persistent coarse solver (host only): dict of grid,
    per, nslot, resident, sg, smem, off_S, off_sc, off_P, off_stg."""
    out = (ctypes.c_longlong * 10)()
    rc = load().smg_persist_plan(V, N, nsys, nvec_next, prec, sms, smem_cap, out)
    if rc != 0:
        raise SmgError(rc, "persist_plan: bad shape")
    keys = ("grid", "per", "nslot", "resident", "sg", "smem", "off_S", "off_sc", "off_P", "off_stg")
    return dict(zip(keys, list(out)))


def deflation_block(k: int) -> int:
    """Fields in the start block of a k-vector coarsest deflation (k + guard)."""
    return k + max(4, k // 4)


def setup_input_sizes(dims, params: MGParams):
    """Complex entries each smg_mg_setup start array must hold: nvec[l] fields
    of coarsening l's fine side, then (coarsest_deflate = k > 0) the
    deflation start block of k + guard fields on the coarsest level."""
    sizes = []
    d, ndof = tuple(int(x) for x in dims), 3
    for l in range(params.n_coarse):
        sizes.append(params.nvec[l] * int(np.prod(d)) * ndof)
        d = tuple(x // a for x, a in zip(d, params.agg[l]))
        ndof = 2 * params.nvec[l]
    if params.coarsest_deflate > 0:
        sizes.append(deflation_block(params.coarsest_deflate) * int(np.prod(d)) * ndof)
    return sizes


def default_params(**kw) -> MGParams:
    p = MGParams()
    load().smg_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "agg":
            for l, a in enumerate(v):
                for mu in range(4):
                    p.agg[l][mu] = int(a[mu])
        elif k == "nvec":
            for l, n in enumerate(v):
                p.nvec[l] = int(n)
        else:
            setattr(p, k, v)
    return p


def _ptr(a):
    """(pointer, where) for a complex128 numpy array or torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            if a.is_cuda:
                return ctypes.c_void_p(a.data_ptr()), SMG_DEVICE
            return ctypes.c_void_p(a.data_ptr()), SMG_HOST
    except ImportError:
        pass
    if not isinstance(a, np.ndarray) or not a.flags.c_contiguous:
        raise ValueError("expected a C-contiguous numpy array or a torch tensor")
    return ctypes.c_void_p(a.ctypes.data), SMG_HOST


class Solver:
    """One lattice context of libsmg."""

    def __init__(self, dims):
        self.lib = load()
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.ctx = ctypes.c_void_p()
        arr = (ctypes.c_int * 4)(*self.dims)
        rc = self.lib.smg_create(arr, ctypes.byref(self.ctx))
        if rc != 0:
            raise SmgError(rc, f"smg_create failed for {self.dims}")
        self.params = None

    def close(self):
        if self.ctx:
            self.lib.smg_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != 0 and rc not in allow:
            raise SmgError(rc, self.lib.smg_last_error(self.ctx).decode())
        return rc

    # -- problem ---------------------------------------------------------------
    def set_gauge(self, fat, naik=None, c_naik=0.0):
        fat = _prep(fat)
        pf, where = _ptr(fat)
        if naik is not None:
            naik = _prep(naik)
            pn, _ = _ptr(naik)
        else:
            pn = None
        self._check(self.lib.smg_set_gauge(self.ctx, pf, pn, float(c_naik), where))

    def set_mass(self, m):
        self._check(self.lib.smg_set_mass(self.ctx, float(m)))

    def set_boundary(self, antiperiodic_t=False):
        """Time boundary of the fermion field (periodic or antiperiodic); call
        set_gauge (and mg_setup) again afterwards."""
        self._check(self.lib.smg_set_boundary(self.ctx, BC_T_ANTIPERIODIC if antiperiodic_t else 0))

    def set_stream(self, stream_handle):
        self._check(self.lib.smg_set_stream(self.ctx, ctypes.c_void_p(stream_handle)))

    def mg_setup(self, params: MGParams, phi0):
        # the library reads these host or device arrays by the sizes the
        # parameters imply; a short array is refused here, before the call
        need = setup_input_sizes(self.dims, params)
        for l, (a, n) in enumerate(zip(phi0, need)):
            if int(np.prod(tuple(a.shape))) < n:
                raise SmgError(-1, f"mg_setup: start array {l} holds {int(np.prod(tuple(a.shape)))} "
                                   f"complex entries, needs {n}")
        arrs = [_prep(a) for a in phi0]
        ptrs = [_ptr(a) for a in arrs]
        where = ptrs[0][1]
        # a trailing NULL: the library reads phi0[n_coarse] (the deflation start
        # block) only with coarsest_deflate > 0 and reports a missing one
        arr = (ctypes.c_void_p * (len(arrs) + 1))(*([p for p, _ in ptrs] + [None]))
        self._check(self.lib.smg_mg_setup(self.ctx, ctypes.byref(params), arr, where))
        self.params = params
        self._keep = arrs

    def save_setup(self, path):
        """Writes the current setup (parameters, near-null vectors, deflation) to `path`."""
        self._check(self.lib.smg_save_setup(self.ctx, os.fsencode(path)))

    def load_setup(self, path, params=None):
        """Rebuilds the hierarchy from a file of save_setup for the current gauge
        field and mass, with the saved parameters or `params` (same level structure)."""
        self._check(self.lib.smg_load_setup(self.ctx, os.fsencode(path),
                                            None if params is None else ctypes.byref(params)))
        self.params = self._read_params(path) if params is None else params

    @staticmethod
    def _read_params(path):
        """The smg_mg_params block of a saved setup (binding bookkeeping: the
        level shapes the array getters need)."""
        with open(path, "rb") as f:
            head = f.read(8 + 4 + 4 + 16 + 8 + 4)
            if head[:8] != b"SMGSETUP":
                raise SmgError(-1, f"{path} is not a saved setup")
            p = MGParams()
            raw = f.read(ctypes.sizeof(MGParams))
            ctypes.memmove(ctypes.byref(p), raw, ctypes.sizeof(MGParams))
        return p

    def solve(self, b, tol=1e-10, x=None):
        b = _prep(b)
        x = _like(b) if x is None else x
        pb, where = _ptr(b)
        px, _ = _ptr(x)
        info = SolveInfo()
        self._check(self.lib.smg_solve(self.ctx, pb, px, float(tol), where, ctypes.byref(info)), allow=(-5,))
        return x, info

    def multi_solve(self, b, masses, tol=1e-10, x=None):
        """b: (nrhs, V, 3); returns x: (nshift, nrhs, V, 3) and a list of infos."""
        b = _prep(b)
        nrhs = b.shape[0]
        masses = np.ascontiguousarray(masses, dtype=np.float64)
        nshift = masses.size
        if x is None:
            x = _like(b, (nshift,) + tuple(b.shape))
        pb, where = _ptr(b)
        px, _ = _ptr(x)
        infos = (SolveInfo * (nrhs * nshift))()
        mp = masses.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self._check(self.lib.smg_multi_solve(self.ctx, nrhs, pb, nshift, mp, px, float(tol), where, infos),
                    allow=(-5,))
        return x, list(infos)

    def multishift_cg(self, b, masses, tol=1e-10, maxiter=10000):
        """M(m_i) x_i = b for every mass with one multi-shift CG; b: (V, 3);
        returns x: (nshift, V, 3) and a list of infos."""
        b = _prep(b)
        masses = np.ascontiguousarray(masses, dtype=np.float64)
        x = _like(b, (masses.size,) + tuple(b.shape))
        pb, where = _ptr(b)
        px, _ = _ptr(x)
        infos = (SolveInfo * masses.size)()
        mp = masses.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self._check(self.lib.smg_multishift_cg(self.ctx, pb, masses.size, mp, px, float(tol), int(maxiter), where,
                                               infos), allow=(-5,))
        return x, list(infos)

    def propagators(self, b, masses, n_mg, tol=1e-10, cg_maxiter=10000):
        """The workflow split: the n_mg lightest masses by MG, the rest by
        multi-shift CG; b: (V, 3); returns x: (nmass, V, 3) in the order of
        `masses` and a list of infos."""
        b = _prep(b)
        masses = np.ascontiguousarray(masses, dtype=np.float64)
        x = _like(b, (masses.size,) + tuple(b.shape))
        pb, where = _ptr(b)
        px, _ = _ptr(x)
        infos = (SolveInfo * masses.size)()
        mp = masses.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self._check(self.lib.smg_propagators(self.ctx, pb, masses.size, mp, int(n_mg), px, float(tol),
                                             int(cg_maxiter), where, infos), allow=(-5,))
        return x, list(infos)

    # -- hooks -------------------------------------------------------------------
    def apply(self, op, v, prec=PREC_DOUBLE):
        v = _prep(v)
        nsys = v.shape[0] if v.ndim == 3 else 1
        out = _like(v)
        pi, where = _ptr(v)
        po, _ = _ptr(out)
        self._check(self.lib.smg_apply_fine(self.ctx, op, prec, nsys, pi, po, where))
        return out

    def maps(self, agg):
        outs = [np.empty(self.V, dtype=np.int32) for _ in range(5)]
        a = (ctypes.c_int * 4)(*agg)
        ptrs = [o.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) for o in outs]
        self._check(self.lib.smg_get_maps(self.ctx, a, *ptrs, SMG_HOST))
        return outs

    def kd_inverse(self):
        out = np.empty((self.V // 16, 48, 48), dtype=np.complex128)
        self._check(self.lib.smg_get_kd_inverse(self.ctx, ctypes.c_void_p(out.ctypes.data), SMG_HOST))
        return out

    def _level_shape(self, l):
        p = self.params
        dims = self.dims
        ndof = 3
        for k in range(l):
            dims = tuple(d // a for d, a in zip(dims, p.agg[k]))
            ndof = 2 * p.nvec[k]
        cdims = tuple(d // a for d, a in zip(dims, p.agg[l]))
        return int(np.prod(dims)), ndof, int(np.prod(cdims)), 2 * p.nvec[l]

    def null_vectors(self, l):
        Vf, ndof, _, _ = self._level_shape(l)
        out = np.empty((self.params.nvec[l], Vf, ndof), dtype=np.complex128)
        self._check(self.lib.smg_get_null_vectors(self.ctx, l, ctypes.c_void_p(out.ctypes.data), SMG_HOST))
        return out

    def coarse_op(self, l):
        _, _, Vc, N = self._level_shape(l)
        out = np.empty((Vc, N, 9, N), dtype=np.complex128)
        self._check(self.lib.smg_get_coarse_op(self.ctx, l, ctypes.c_void_p(out.ctypes.data), SMG_HOST))
        return out

    def coarse_xinv(self, l):
        _, _, Vc, N = self._level_shape(l)
        out = np.empty((Vc, N, N), dtype=np.complex128)
        self._check(self.lib.smg_get_coarse_xinv(self.ctx, l, ctypes.c_void_p(out.ctypes.data), SMG_HOST))
        return out

    def deflation(self):
        """(sigma, info) of the deflated coarsest level: the k lowest singular
        values and {lmin, lmax, iterations, residual}."""
        k = self.params.coarsest_deflate
        sig = np.empty(k, dtype=np.float64)
        info = np.empty(4, dtype=np.float64)
        self._check(self.lib.smg_get_deflation(self.ctx, ctypes.c_void_p(sig.ctypes.data),
                                               ctypes.c_void_p(info.ctypes.data)))
        return sig, dict(lmin=info[0], lmax=info[1], iterations=int(info[2]), residual=info[3])

    def coarse_solve(self, l, v):
        """One solve of the level coarsening l produces, as the K-cycle runs it."""
        _, _, Vc, N = self._level_shape(l)
        v = _prep(v)
        nsys = v.shape[0]
        out = _like(v, (nsys, Vc, N))
        pi, where = _ptr(v)
        po, _ = _ptr(out)
        self._check(self.lib.smg_coarse_solve(self.ctx, l, nsys, pi, po, where))
        return out

    def _xfer(self, fn, l, v, prec, out_shape):
        v = _prep(v)
        nsys = v.shape[0]
        out = _like(v, (nsys,) + out_shape)
        pi, where = _ptr(v)
        po, _ = _ptr(out)
        self._check(fn(self.ctx, l, prec, nsys, pi, po, where))
        return out

    def restrict(self, l, v, prec=PREC_DOUBLE):
        _, _, Vc, N = self._level_shape(l)
        return self._xfer(self.lib.smg_restrict, l, v, prec, (Vc, N))

    def prolong(self, l, v, prec=PREC_DOUBLE):
        Vf, ndof, _, _ = self._level_shape(l)
        return self._xfer(self.lib.smg_prolong, l, v, prec, (Vf, ndof))

    def coarse_apply(self, l, v, prec=PREC_DOUBLE):
        _, _, Vc, N = self._level_shape(l)
        return self._xfer(self.lib.smg_coarse_apply, l, v, prec, (Vc, N))

    def force(self, X, Y, which=0):
        X, Y = _prep(X), _prep(Y)
        F = _like(X, (4, self.V, 3, 3))
        px, where = _ptr(X)
        py, _ = _ptr(Y)
        pf, _ = _ptr(F)
        self._check(self.lib.smg_force(self.ctx, px, py, int(which), pf, where))
        return F

    def time_kernel(self, kernel, l=0, nsys=1, nrep=100):
        """Average milliseconds per launch of one library kernel (CUDA events)."""
        v = ctypes.c_double()
        self._check(self.lib.smg_time_kernel(self.ctx, kernel, l, nsys, nrep, ctypes.byref(v)))
        return v.value

    def fermion_action(self, phi, tol=1e-10):
        """S, dS/dm, X, Y for S = phi^dag (M^dag M)^{-1} phi (two MG solves in the library)."""
        phi = _prep(phi)
        X, Y = _like(phi), _like(phi)
        pp, where = _ptr(phi)
        px, _ = _ptr(X)
        py, _ = _ptr(Y)
        S, dm = ctypes.c_double(), ctypes.c_double()
        infos = (SolveInfo * 2)()
        self._check(self.lib.smg_fermion_action(self.ctx, pp, px, py, float(tol), where, ctypes.byref(S),
                                                ctypes.byref(dm), infos), allow=(-5,))
        return S.value, dm.value, X, Y, list(infos)

    def dot_noalloc(self, x, y, out):
        """out[s] = <x_s, y_s> for device tensors x, y ([nsys, ...] complex128) into
        the caller's device tensor out (nsys complex128); enqueued on the
        context's stream, no allocation inside the library.  The library
        cannot tell host from device pointers, so the tensors are checked here
        (ValueError) before any pointer reaches it."""
        nsys, n = check_dot_noalloc_args(x, y, out)
        self._check(self.lib.smg_dot_noalloc(self.ctx, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                             n, nsys, ctypes.c_void_p(out.data_ptr())))
        return out

    def coarse_apply_stencil(self, cdims, stencil, v, prec=PREC_HALF, path=0):
        """The coarse apply of a caller's FP64 stencil [Vc][N][9][N] on v [nsys][Vc][N]
        through kernel `path` (COARSE_*; 0 = the autotuner's choice)."""
        stencil = _prep(stencil)
        v = _prep(v)
        N = int(stencil.shape[1])
        out = _like(v)
        ps, where = _ptr(stencil)
        pi, _ = _ptr(v)
        po, _ = _ptr(out)
        arr = (ctypes.c_int * 4)(*[int(c) for c in cdims])
        self._check(self.lib.smg_coarse_apply_stencil(self.ctx, arr, N, int(prec), int(path), ps, int(v.shape[0]),
                                                      pi, po, where))
        return out

    def bench_coarse_apply(self, cdims, N, nsys=1, prec=PREC_HALF, nrep=20):
        """ms per launch of the coarse apply on a synthetic stencil of this shape."""
        v = ctypes.c_double()
        arr = (ctypes.c_int * 4)(*cdims)
        self._check(self.lib.smg_bench_coarse_apply(self.ctx, arr, int(N), int(nsys), int(prec), int(nrep),
                                                    ctypes.byref(v)))
        return v.value

    def debug_persist_barrier(self, limit_ns=2000000000, extra_arrivals=0):
        """Test hook: grid-barrier wait limit of the persistent coarse solver and
        an extra expected arrival that never comes (extra_arrivals = 1)."""
        self._check(self.lib.smg_debug_persist_barrier(self.ctx, int(limit_ns), int(extra_arrivals)))

    def setup_iterations(self, l):
        v = ctypes.c_int()
        self._check(self.lib.smg_setup_iterations(self.ctx, l, ctypes.byref(v)))
        return v.value

    def setup_times(self, l):
        """Seconds the last setup spent on coarsening l: dict of the phases
        cgne, orthonormalise, galerkin, other."""
        v = (ctypes.c_double * 4)()
        self._check(self.lib.smg_setup_times(self.ctx, l, v))
        return dict(zip(("cgne", "orthonormalise", "galerkin", "other"), [float(x) for x in v]))


def check_dot_noalloc_args(x, y, out):
    """(nsys, n) of a dot_noalloc call on torch tensors x, y of shape
    [nsys, ...] and out of at least nsys entries; ValueError unless all three
    are contiguous complex128 CUDA tensors on one device with y shaped like x.
    A host tensor, a narrower dtype or a short y / out would make the kernel
    read or write outside the caller's buffers."""
    import torch
    for name, t in (("x", x), ("y", y), ("out", out)):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"dot_noalloc: {name} must be a torch tensor")
        if t.dtype != torch.complex128:
            raise ValueError(f"dot_noalloc: {name} must be complex128")
        if not t.is_contiguous():
            raise ValueError(f"dot_noalloc: {name} must be contiguous")
    if x.dim() < 1 or x.shape[0] < 1 or x.numel() == 0:
        raise ValueError("dot_noalloc: x must hold at least one non-empty system")
    if tuple(y.shape) != tuple(x.shape):
        raise ValueError("dot_noalloc: y must have the shape of x")
    nsys = int(x.shape[0])
    if out.numel() < nsys:
        raise ValueError("dot_noalloc: out must hold nsys entries")
    for name, t in (("x", x), ("y", y), ("out", out)):
        if not t.is_cuda:
            raise ValueError(f"dot_noalloc: {name} must be a CUDA tensor")
    if not (x.device == y.device == out.device):
        raise ValueError("dot_noalloc: x, y and out must be on one device")
    return nsys, x.numel() // nsys


def _prep(a):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.complex128:
                raise ValueError("tensors must be complex128")
            return a.contiguous()
    except ImportError:
        pass
    return np.ascontiguousarray(a, dtype=np.complex128)


def _like(a, shape=None):
    shape = tuple(a.shape) if shape is None else tuple(shape)
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return torch.empty(shape, dtype=torch.complex128, device=a.device)
    except ImportError:
        pass
    return np.empty(shape, dtype=np.complex128)
