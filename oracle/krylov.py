"""Krylov solvers of the oracle: flexible GCR, minimal-residual relaxation, and
the comparison solvers BiCGStab and CGNR.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper uses GCR as the outer solver because the Wilson operator is
non-Hermitian and the multigrid cycle is non-stationary ("Adaptive
multigrid"), and GCR again at every coarse level, preconditioned by the next
cycle, down to an unpreconditioned GCR on the coarsest lattice
("Implementation").  Restart length and orthogonalisation are not given;
the reading here is textbook flexible GCR(m) with modified Gram-Schmidt on
the ``w_j = A z_j`` (the ``z_j`` follow the same combination), both scaled by
``1/||w||``, and the true residual recomputed at every restart.

The smoother ("relaxation ... stationary or Krylov") is minimal-residual
relaxation, i.e. GCR(1) without restarts.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .dirac import inner, norm2


@dataclass
class SolveInfo:
    iterations: int = 0
    restarts: int = 0
    residual: float = float("nan")
    history: list = field(default_factory=list)
    converged: bool = False


def fgcr(A, b, precond=None, x0=None, tol_abs: float = 0.0, maxiter: int = 1000, restart: int = 16,
         true_residual: bool = True, stop=None):
    """Flexible GCR(restart) for ``A x = b``.

    Stops when ``||r|| <= tol_abs`` (or ``stop(x, r)`` returns True) or after
    ``maxiter`` iterations.  ``precond(r)`` gives ``z``; ``None`` means
    ``z = r``.  Returns ``(x, SolveInfo)``.
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b.copy() if x0 is None else b - A(x)
    info = SolveInfo()
    rn = math.sqrt(norm2(r))
    info.history.append(rn)
    if rn <= tol_abs:
        info.residual, info.converged = rn, True
        return x, info
    while info.iterations < maxiter:
        Z, W = [], []
        for _ in range(restart):
            z = precond(r) if precond is not None else r.copy()
            w = A(z)
            for zj, wj in zip(Z, W):
                beta = inner(wj, w)
                w = w - beta * wj
                z = z - beta * zj
            g = math.sqrt(norm2(w))
            if g == 0.0:
                break
            w = w / g
            z = z / g
            alpha = inner(w, r)
            x = x + alpha * z
            r = r - alpha * w
            Z.append(z)
            W.append(w)
            info.iterations += 1
            rn = math.sqrt(norm2(r))
            info.history.append(rn)
            if rn <= tol_abs or info.iterations >= maxiter:
                break
        if true_residual:
            r = b - A(x)
            rn = math.sqrt(norm2(r))
        info.restarts += 1
        if rn <= tol_abs or (stop is not None and stop(x, r)):
            break
        if not Z:
            break
    info.residual = rn
    info.converged = rn <= tol_abs
    return x, info


def mr(A, r, nu: int):
    """``nu`` steps of minimal-residual relaxation on ``A e = r`` from ``e = 0``."""
    e = np.zeros_like(r)
    r = r.copy()
    for _ in range(nu):
        w = A(r)
        ww = norm2(w)
        if ww == 0.0:
            break
        alpha = inner(w, r) / ww
        e = e + alpha * r
        r = r - alpha * w
    return e


# ----------------------------------------------------------------------------- comparison solvers
# The paper times multigrid against the Krylov solvers in use ("Results"):
# BiCGStab, CG on the normal residual (CGNR) and a mixed-precision version by
# iterative refinement.  The oracle restates the textbook methods; their
# solutions are D^{-1} b like every other solve, so the GPU solvers are
# checked by their true residuals with the oracle's D.

def bicgstab(A, b, x0=None, tol_abs: float = 0.0, maxiter: int = 1000):
    """BiCGStab (van der Vorst) for ``A x = b``: shadow residual ``r_hat = r_0``,
    two applications of A per iteration, stop on ``||r|| <= tol_abs``."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    info = SolveInfo(residual=math.sqrt(norm2(r)))
    if info.residual <= tol_abs:
        info.converged = True
        return x, info
    rh = r.copy()
    rho = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for it in range(maxiter):
        rho_new = inner(rh, r)
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = A(p)
        alpha = rho_new / inner(rh, v)
        s = r - alpha * v
        t = A(s)
        omega = inner(t, s) / inner(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho = rho_new
        info.iterations = it + 1
        info.residual = math.sqrt(norm2(r))
        info.history.append(info.residual)
        if info.residual <= tol_abs:
            info.converged = True
            break
    return x, info


def cgnr(A, Adag, b, x0=None, tol_abs: float = 0.0, maxiter: int = 1000):
    """CG on the normal equations ``A^dag A x = A^dag b`` (CGLS: the residual
    ``r = b - A x`` is carried along and tested, ``||r|| <= tol_abs``)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    z = Adag(r)
    p = z.copy()
    zz = norm2(z)
    info = SolveInfo(residual=math.sqrt(norm2(r)))
    for it in range(maxiter):
        if info.residual <= tol_abs or zz == 0.0:
            break
        w = A(p)
        a = zz / norm2(w)
        x = x + a * p
        r = r - a * w
        z = Adag(r)
        zz_new = norm2(z)
        p = z + (zz_new / zz) * p
        zz = zz_new
        info.iterations = it + 1
        info.residual = math.sqrt(norm2(r))
        info.history.append(info.residual)
    info.converged = info.residual <= tol_abs
    return x, info
