"""GPU parity of the comparison Krylov solvers, through the C ABI.

* D_r^dag (mg_apply MG_OP_DR_DAG, the operator of CGNR) against the conjugate
  transpose of the oracle's D_r, built column by column as a dense matrix on
  4^4 (FP64 <= 1e-12, FP32 <= 1e-5).
* BiCGStab, CGNR and the mixed-precision BiCGStab (iterative refinement) reach
  ||eta - D psi|| / ||eta|| <= 1e-10 with the oracle's D, agree with the
  multigrid solution, and solve the dagger system through gamma_5.
* Bad modes and a coarse-level D_r^dag are rejected.
"""
import numpy as np
import pytest

from gpu_common import TOL32, TOL64, lib_built, rel
from oracle.dirac import WilsonClover, norm2
from paper_1011_2775_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _solver(dims, U, csw, m0):
    lib_built()
    from paper_1011_2775_gb300.solver import Solver
    S = Solver(dims)
    S.load_gauge(U)
    S.set_clover(csw, m0)
    return S


def _res(W, psi, eta):
    r = eta.reshape(W.shape + (12,)) - W.D(psi.reshape(W.shape + (12,)))
    return float(np.sqrt(norm2(r) / norm2(eta)))


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_dr_dagger_is_the_adjoint_of_the_oracle_dr(prec):
    from paper_1011_2775_gb300 import binding as B
    dims = (4, 4, 4, 4)
    U = I.make_gauge(dims, 0.5, 1, 0.5, 9001)
    W = WilsonClover(U, 1.2, -0.3)
    even = np.broadcast_to(W.even, W.shape + (12,)).astype(bool)
    idx = np.flatnonzero(even.ravel())
    n = idx.size
    Dr = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(W.shape + (12,), dtype=np.complex128)
    for j in range(n):
        e.ravel()[idx[j]] = 1.0
        Dr[:, j] = W.Dr(e).ravel()[idx]
        e.ravel()[idx[j]] = 0.0
    S = _solver(dims, U, 1.2, -0.3)
    u = I.gaussian_source(dims, 9002)
    got = S.apply(B.MG_OP_DR_DAG, u, prec=prec)
    ref = np.zeros(W.shape + (12,), dtype=np.complex128)
    ref.ravel()[idx] = Dr.conj().T @ u.reshape(W.shape + (12,)).ravel()[idx]
    assert rel(got, ref.reshape(u.shape)) <= (TOL64 if prec == 0 else TOL32)
    assert not got.reshape(W.shape + (12,))[~even].any()       # odd sites zeroed
    S.close()


@pytest.fixture(scope="module")
def system():
    dims = (8, 8, 8, 16)
    U = I.make_gauge(dims, 1.0, 5, 0.5, 9101)
    W = WilsonClover(U, 1.0, -0.3)
    S = _solver(dims, U, 1.0, -0.3)
    S.set_params(levels=2, blocks=[(4, 4, 4, 4)], nv=[12], seed=9102, maxit_fine=20000)
    S.setup()
    eta = I.gaussian_source(dims, 9103)
    from paper_1011_2775_gb300 import binding as B
    ref, _ = S.solve(eta, 1e-10, B.MG_MODE_MG)
    yield dims, W, S, eta, ref
    S.close()


@pytest.mark.parametrize("mode", ["BICGSTAB", "CGNR", "BICGSTAB_MP"])
def test_comparison_solvers_reach_the_tolerance(system, mode):
    from paper_1011_2775_gb300 import binding as B
    dims, W, S, eta, ref = system
    psi, info = S.solve(eta, 1e-10, getattr(B, "MG_MODE_" + mode))
    assert info.true_residual <= 1e-10
    assert _res(W, psi, eta) <= 1e-10
    assert np.linalg.norm((psi - ref).ravel()) / np.linalg.norm(ref.ravel()) < 1e-7
    assert info.outer_iterations > 0
    if mode == "BICGSTAB_MP":
        assert info.restarts >= 2          # several refinement steps for 1e-10 from 1e-4 inner solves


@pytest.mark.parametrize("mode", ["BICGSTAB", "BICGSTAB_MP"])
def test_comparison_solvers_dagger(system, mode):
    from paper_1011_2775_gb300 import binding as B
    dims, W, S, eta, ref = system
    lam, info = S.solve_dagger(eta, 1e-10, getattr(B, "MG_MODE_" + mode))
    lv = lam.reshape(W.shape + (12,))
    r = eta.reshape(W.shape + (12,)) - W.gamma5(W.D(W.gamma5(lv)))
    assert np.sqrt(norm2(r) / norm2(eta)) <= 1e-10


def test_iteration_cap_and_bad_arguments(system):
    from paper_1011_2775_gb300 import binding as B
    dims, W, S, eta, ref = system
    S.set_params(maxit_fine=5)
    psi = np.zeros_like(eta)
    st, info = B.mg_solve(S.ctx, psi, eta, 1, 1e-10, B.MG_MODE_BICGSTAB, allow_not_converged=True)
    assert st == B.MG_ERR_NOT_CONVERGED and info.true_residual > 1e-10
    S.set_params(maxit_fine=20000)
    with pytest.raises(B.MGError) as e:
        B.mg_solve(S.ctx, psi, eta, 1, 1e-10, 5)
    assert e.value.status == B.MG_ERR_ARG
    with pytest.raises(B.MGError) as e:
        S.apply(B.MG_OP_DR_DAG, np.zeros((2, 2, 2, 4, 24), dtype=np.complex128), level=1)
    assert e.value.status == B.MG_ERR_ARG


@pytest.mark.parametrize("mode", ["bicgstab", "cgnr"])
def test_krylov_iterations_and_solution_match_the_oracle(mode):
    """The GPU's FP64 BiCGStab and CGNR against the oracle's textbook solvers
    on the same reduced system (config 1: 4^4, eps = 0.3, csw = 1, m0 = -0.1):
    both stop at ||r_r|| <= 0.5e-10 ||eta||; the iteration counts agree within
    two (the GPU also tests the half-step residual of BiCGStab) and the
    solutions agree to the conditioning of that residual."""
    from oracle.krylov import bicgstab, cgnr
    from paper_1011_2775_gb300 import binding as B
    dims = (4, 4, 4, 4)
    U = I.make_gauge(dims, 0.3, 0, 0.5, 1001)
    W = WilsonClover(U, 1.0, -0.1)
    eta = I.gaussian_source(dims, 1002)
    b = eta.reshape(W.shape + (12,))
    tol_abs = 0.5e-10 * np.sqrt(norm2(b))
    br = W.b_r(b)
    if mode == "bicgstab":
        y, oinfo = bicgstab(lambda v: W.Dr(v * W.even), br, tol_abs=tol_abs, maxiter=5000)
    else:
        even = np.broadcast_to(W.even, W.shape + (12,)).astype(bool)
        idx = np.flatnonzero(even.ravel())
        Dr = np.empty((idx.size, idx.size), dtype=np.complex128)
        e = np.zeros(W.shape + (12,), dtype=np.complex128)
        for j in range(idx.size):
            e.ravel()[idx[j]] = 1.0
            Dr[:, j] = W.Dr(e).ravel()[idx]
            e.ravel()[idx[j]] = 0.0

        def dag(v):
            out = np.zeros_like(v)
            out.ravel()[idx] = Dr.conj().T @ v.ravel()[idx]
            return out
        y, oinfo = cgnr(lambda v: W.Dr(v * W.even), dag, br, tol_abs=tol_abs, maxiter=5000)
    assert oinfo.converged
    x = W.reconstruct(y, b)
    S = _solver(dims, U, 1.0, -0.1)
    S.set_params(maxit_fine=5000)
    psi, info = S.solve(eta, 1e-10, B.MG_MODE_BICGSTAB if mode == "bicgstab" else B.MG_MODE_CGNR)
    assert _res(W, psi, eta) <= 1e-10
    assert abs(info.outer_iterations - oinfo.iterations) <= 2, (info.outer_iterations, oinfo.iterations)
    assert np.linalg.norm(psi.ravel() - x.ravel()) <= 1e-7 * np.linalg.norm(x)
    S.close()
