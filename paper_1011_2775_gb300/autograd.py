"""``torch.autograd`` Function for the solve ``psi = D(U)^{-1} eta``.

The paper solves the Dirac equation; differentiating the solve is an
extension.  Forward: one multigrid solve (``mg_solve``).  Backward, for the
incoming gradient ``g`` of ``psi`` (torch's convention for complex tensors,
``dL/dRe + i dL/dIm``):

* ``lam = D^{-dag} g``: one adjoint solve with the same multigrid through
  ``D^dag = gamma_5 D gamma_5`` (``mg_solve_dagger``);
* ``grad_eta = lam``;
* ``grad_U``: the derivative of ``-Re<lam, D(U) psi>`` with respect to the
  complex links (``mg_force`` with ``MG_FORCE_WIRTINGER``), hop and clover
  terms.

Only ``psi`` is kept between forward and backward -- the Krylov vectors of
either solve are not stored.  Marshalling only: both solves and the force run
in libmgclover.
"""
from __future__ import annotations

import torch

from . import binding as B


class DiracSolve(torch.autograd.Function):
    """``psi = DiracSolve.apply(eta, U, solver, tol)``.

    ``solver`` (a :class:`~paper_1011_2775_gb300.solver.Solver`) must hold ``U``:
    loaded with ``solver.load_gauge(U)`` (the same tensor, unmodified since),
    clover and mass set and, for the multigrid mode, set up.  ``eta`` and ``U``
    are complex128 CUDA tensors in the ABI layouts.
    """

    @staticmethod
    def forward(ctx, eta, U, solver, tol=1e-10, mode=B.MG_MODE_MG):
        if U is not None and (solver.gauge_ref is not U or solver.gauge_version != U._version):
            raise ValueError("the solver does not hold this gauge field: call solver.load_gauge(U) "
                             "(and set the clover, mass and setup) first")
        psi, info = solver.solve(eta.contiguous(), tol, mode)
        ctx.save_for_backward(psi)
        ctx.solver, ctx.tol, ctx.mode = solver, tol, mode
        ctx.info = info
        return psi

    @staticmethod
    def backward(ctx, g):
        (psi,) = ctx.saved_tensors
        lam, _ = ctx.solver.solve_dagger(g.contiguous(), ctx.tol, ctx.mode)
        grad_eta = lam if ctx.needs_input_grad[0] else None
        grad_U = None
        if ctx.needs_input_grad[1]:
            grad_U = ctx.solver.force(lam, psi, kind=B.MG_FORCE_WIRTINGER)
        return grad_eta, grad_U, None, None, None


def dirac_solve(solver, eta, U=None, tol: float = 1e-10, mode: int = B.MG_MODE_MG):
    """Differentiable ``D(U)^{-1} eta`` (see :class:`DiracSolve`)."""
    return DiracSolve.apply(eta, U, solver, tol, mode)


def su3_force(solver, lam, psi):
    """The su(3) force ``sum_a F^a T_a`` of ``-Re<lam, D(U) psi>`` (``MG_FORCE_SU3``)."""
    return solver.force(lam, psi, kind=B.MG_FORCE_SU3)
