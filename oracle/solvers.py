"""Krylov solvers of the oracle (test infrastructure only).

* GCR, flexible and right-preconditioned (Sec. 2.1: the K-cycle preconditions
  an outer flexible GCR; Table 1: every level's solver is GCR).
* CA-GCR(s), the s-step smoother of Sec. 3.2 / Table 1: one Krylov basis of
  s vectors built from powers of the operator, then a single least-squares
  solve for the minimum-residual combination.  In exact arithmetic this is
  the minimum-residual correction over the Krylov space K_s(A, r).
* CGNE, the setup solver of Table 1, used on the homogeneous system
  A phi = 0 from a random start (Sec. 2.1): conjugate gradients on
  A A^dag y = b with x = A^dag y (Craig's method), which minimises the error
  norm; for b = 0 the iterate decays slowest along the low modes.

Vectors are numpy arrays of any shape; inner products are over all entries.
"""
from __future__ import annotations

import numpy as np


def dot(a, b) -> complex:
    return complex(np.vdot(a, b))


def norm(a) -> float:
    return float(np.sqrt(np.vdot(a, a).real))


def gcr(apply, b, x0=None, precond=None, tol=1e-10, maxiter=1000, nkrylov=16,
        true_residual=True):
    """Flexible GCR with right preconditioning and restarts.

    Iteration k: z_k = K(r), w_k = A z_k, w_k made orthogonal to w_0..w_{k-1}
    (modified Gram-Schmidt), then x += alpha z-combination with
    alpha = <w_k, r>/<w_k, w_k>.  The search directions p_k (A p_k = w_k) are
    kept explicitly.  Stops when ||r|| <= tol ||b|| (with the residual
    recomputed as b - A x at each restart and at the end when
    ``true_residual``) or after ``maxiter`` iterations.

    Returns (x, iterations, ||b - A x|| / ||b||).
    """
    bnorm = norm(b)
    x = np.zeros_like(b) if x0 is None else x0.astype(np.complex128, copy=True)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    r = b - apply(x) if x0 is not None else b.copy()
    it = 0
    while True:
        ps, ws = [], []
        rnorm = norm(r)
        while it < maxiter and rnorm > tol * bnorm and len(ws) < nkrylov:
            z = precond(r) if precond is not None else r.copy()
            w = apply(z)
            for p_j, w_j in zip(ps, ws):
                beta = dot(w_j, w) / dot(w_j, w_j).real
                w = w - beta * w_j
                z = z - beta * p_j
            alpha = dot(w, r) / dot(w, w).real
            x = x + alpha * z
            r = r - alpha * w
            ps.append(z)
            ws.append(w)
            rnorm = norm(r)
            it += 1
        if not true_residual:
            return x, it, rnorm / bnorm
        r = b - apply(x)
        rnorm = norm(r)
        if rnorm <= tol * bnorm or it >= maxiter:
            return x, it, rnorm / bnorm


def ca_gcr(apply, r, s: int):
    """s-step minimum-residual correction e with the power basis.

    V = [r, A r, ..., A^{s-1} r], W = A V, alpha = argmin ||r - W alpha||,
    e = V alpha.
    """
    vs = [r]
    for _ in range(s - 1):
        vs.append(apply(vs[-1]))
    ws = vs[1:] + [apply(vs[-1])]
    Vm = np.stack([v.ravel() for v in vs], axis=1)
    Wm = np.stack([w.ravel() for w in ws], axis=1)
    alpha, *_ = np.linalg.lstsq(Wm, r.ravel(), rcond=None)
    return (Vm @ alpha).reshape(r.shape)


def cgne(apply, apply_dag, b, x0, tol: float, maxiter: int):
    """Craig's method (CG on A A^dag) from x0.  Stops when
    ||b - A x|| <= tol * ||b - A x0|| or after ``maxiter`` iterations.

    Returns (x, iterations, final ||r|| / ||r0||).
    """
    x = x0.astype(np.complex128, copy=True)
    r = b - apply(x)
    rr = dot(r, r).real
    r0 = np.sqrt(rr)
    if r0 == 0.0:
        return x, 0, 0.0
    p = apply_dag(r)
    it = 0
    while it < maxiter and np.sqrt(rr) > tol * r0:
        alpha = rr / dot(p, p).real
        x = x + alpha * p
        r = r - alpha * apply(p)
        rr_new = dot(r, r).real
        beta = rr_new / rr
        rr = rr_new
        p = apply_dag(r) + beta * p
        it += 1
    return x, it, float(np.sqrt(rr) / r0)
