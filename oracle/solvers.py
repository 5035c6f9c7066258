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


def multishift_cg(apply, b, shifts, tol: float = 1e-10, maxiter: int = 10000):
    """Conjugate gradients for (A + sigma_i) x_i = b, all shifts at once.

    A is Hermitian positive (semi)definite and every sigma_i >= 0.  The
    shifted systems share one Krylov space: CG runs on the base system
    A + sigma_0 (sigma_0 = min sigma) with one product by A per iteration, and
    shift i carries a scalar zeta_i with its residual r_i = zeta_i r.  From the
    three-term recurrence of the Lanczos polynomials (Jegerlehner 1996,
    "Krylov space solvers for shifted linear systems"), with d_i = sigma_i -
    sigma_0, base step alpha and base beta:

      zeta_i' = zeta_i zeta_i^- a^- / (a b^- (zeta_i^- - zeta_i)
                                        + zeta_i^- a^- (1 + d_i a)),
      alpha_i = a zeta_i' / zeta_i,   beta_i = b (zeta_i' / zeta_i)^2,
      x_i += alpha_i p_i,             p_i = zeta_i' r' + beta_i p_i.

    Shift i stops updating x_i once |zeta_i| ||r|| <= tol ||b||; the loop stops
    when every shift has.  Returns (xs, iterations, residuals) with xs[i]
    the solution of shift i and residuals[i] = ||b - (A + sigma_i) x_i|| / ||b||
    recomputed.
    """
    shifts = np.asarray(shifts, dtype=np.float64)
    ns = len(shifts)
    s0 = float(shifts.min())
    d = shifts - s0
    bn = norm(b)
    xs = np.zeros((ns,) + b.shape, dtype=np.complex128)
    ps = np.repeat(b[None].astype(np.complex128), ns, axis=0)
    r = b.astype(np.complex128).copy()
    rr = dot(r, r).real
    zeta = np.ones(ns)
    zeta_prev = np.ones(ns)
    a_prev, b_prev = 1.0, 0.0
    active = np.ones(ns, dtype=bool)
    base = int(np.argmin(shifts))
    it = 0
    while it < maxiter and active.any() and bn > 0:
        w = apply(ps[base]) + s0 * ps[base]
        a = rr / dot(ps[base], w).real
        zeta_new = np.empty(ns)
        for i in range(ns):
            den = a * b_prev * (zeta_prev[i] - zeta[i]) + zeta_prev[i] * a_prev * (1.0 + d[i] * a)
            zeta_new[i] = zeta[i] * zeta_prev[i] * a_prev / den if den != 0 else 0.0
            if active[i]:
                xs[i] += (a * zeta_new[i] / zeta[i]) * ps[i]
        r = r - a * w
        rr_new = dot(r, r).real
        beta = rr_new / rr
        for i in range(ns):
            bi = beta * (zeta_new[i] / zeta[i]) ** 2 if zeta[i] != 0 else 0.0
            ps[i] = zeta_new[i] * r + bi * ps[i]
        zeta_prev, zeta = zeta, zeta_new
        a_prev, b_prev, rr = a, beta, rr_new
        it += 1
        active &= np.abs(zeta) * np.sqrt(rr) > tol * bn
    res = [norm(b - (apply(xs[i]) + shifts[i] * xs[i])) / bn if bn > 0 else 0.0 for i in range(ns)]
    return xs, it, res


def staggered_multishift(op, b, masses, tol: float = 1e-10, maxiter: int = 10000):
    """M(m_i) x_i = b for several masses with one Krylov space (the paper's
    multi-shift CG for the heavier masses of a propagator workflow, Sec. 4):
    M(m) = m + D with D anti-Hermitian is normal, M(m)^dag M(m) = m^2 + D^dag D,
    so CG on (D^dag D + m_i^2) y_i = b with shifts m_i^2, then x_i = M(m_i)^dag y_i
    = m_i y_i - D y_i.  `op` supplies D (its own mass is not used).
    Returns (xs, iterations, residuals ||b - M(m_i) x_i|| / ||b||)."""
    ys, it, _ = multishift_cg(lambda v: -op.D(op.D(v)), b, [m * m for m in masses], tol, maxiter)
    xs = np.stack([m * y - op.D(y) for m, y in zip(masses, ys)])
    bn = norm(b)
    res = [norm(b - (m * x + op.D(x))) / bn for m, x in zip(masses, xs)]
    return xs, it, res


def chebyshev_basis(apply, r, s: int, lmin: float, lmax: float):
    """q_k = T_k((A - c)/h) r for k < s by the three-term recurrence of the
    Chebyshev polynomials, c = (lmax + lmin)/2, h = (lmax - lmin)/2."""
    c = 0.5 * (lmax + lmin)
    h = 0.5 * (lmax - lmin)
    Q = [r]
    if s > 1:
        Q.append((apply(r) - c * r) / h)
    while len(Q) < s:
        Q.append(2.0 * (apply(Q[-1]) - c * Q[-1]) / h - Q[-2])
    return Q


def ca_gcr_chebyshev(apply, r, s: int, lmin: float, lmax: float):
    """CA-GCR(s) with a Chebyshev basis (Table 1, coarsest level): the basis
    q_0 = r, q_1 = T q_0, q_{k+1} = 2 T q_k - q_{k-1} with T = (A - c)/h,
    c = (lmax + lmin)/2, h = (lmax - lmin)/2, spans the same Krylov space
    K_s(A, r) as the power basis but stays far better conditioned when the
    spectrum lies near [lmin, lmax]; the correction is the minimum-residual
    combination sum_k a_k q_k over that space (one least-squares solve)."""
    Q = chebyshev_basis(apply, r, s, lmin, lmax)
    W = np.stack([apply(q).ravel() for q in Q], axis=1)
    a, *_ = np.linalg.lstsq(W, r.ravel(), rcond=None)
    return sum(ak * q for ak, q in zip(a, Q))


def shifted_power_basis(apply, r, s: int, lmin: float, lmax: float):
    """q_k = ((A - c)/h)^k r for k < s, c = (lmax + lmin)/2, h = (lmax - lmin)/2:
    the Faber (power) basis of the disk |z - c| <= h, which stays well
    conditioned when the spectrum fills a disk around c rather than lying on
    the real interval [lmin, lmax]."""
    c = 0.5 * (lmax + lmin)
    h = 0.5 * (lmax - lmin)
    Q = [r]
    while len(Q) < s:
        Q.append((apply(Q[-1]) - c * Q[-1]) / h)
    return Q


def ca_gcr_basis(apply, r, s: int, lmin: float, lmax: float, basis: str = "chebyshev"):
    """CA-GCR(s) with the Chebyshev basis of [lmin, lmax] (Table 1) or the
    shifted power basis of the disk around its centre; both span K_s(A, r), so
    in exact arithmetic the minimum-residual correction is the same."""
    if basis == "chebyshev":
        return ca_gcr_chebyshev(apply, r, s, lmin, lmax)
    Q = shifted_power_basis(apply, r, s, lmin, lmax)
    W = np.stack([apply(q).ravel() for q in Q], axis=1)
    a, *_ = np.linalg.lstsq(W, r.ravel(), rcond=None)
    return sum(ak * q for ak, q in zip(a, Q))


def lowest_singular_triplets(dense, k: int):
    """The k smallest singular values of a (small) dense operator with their
    left (U) and right (V) singular vectors: A V = U diag(sigma)."""
    U, sig, Vh = np.linalg.svd(dense)
    idx = np.argsort(sig)[:k]
    return U[:, idx], sig[idx], Vh[idx].conj().T


def svd_deflated_gcr(apply, b, U, sigma, V, tol=1e-10, maxiter=1000, nkrylov=16):
    """GCR from the deflated start x0 = V diag(1/sigma) U^dag b (Table 1's
    SVD-deflated coarsest solve): the residual b - A x0 = (1 - U U^dag) b has
    no component along the deflated left singular vectors, which removes the
    slowest directions before the iteration starts.  Fields are flattened."""
    shape = b.shape
    x0 = (V @ ((U.conj().T @ b.ravel()) / sigma)).reshape(shape)
    return gcr(apply, b, x0=x0, tol=tol, maxiter=maxiter, nkrylov=nkrylov)
