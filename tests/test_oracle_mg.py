"""Pins of the oracle's multigrid, Krylov solvers and random start vectors.

Checked against: dense linear algebra (LU, eig) on small lattices, the
definition ``P^dag D_p P`` assembled densely, the complete-basis two-grid
(unitary P makes the coarse correction exact), published known-answer
vectors of Philox4x32-10, and structural identities (P^dag P = I,
gamma_5 P = P gamma_5c, R = P^dag gamma_5 equivalence).
"""
import math
import os

import numpy as np
import pytest

from oracle.dirac import WilsonClover, inner, norm2
from oracle.krylov import fgcr, mr
from oracle.multigrid import (GSBreakdown, MGParams, Multigrid, Transfer, block_gram_schmidt,
                              build_coarse, eo_solve, setup_null_vectors)
from oracle.philox import gaussian_vector, philox4x32_10
from paper_1011_2775_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _vec(dims, seed):
    return I.gaussian_source(dims, seed).reshape(I.lattice_shape(dims) + (12,))


def _random_vectors(level, nv, seed):
    return [gaussian_vector(seed, 0, k, level.shape, level.ndof) for k in range(nv)]


# ----------------------------------------------------------------------------- RNG
def test_philox_known_answers():
    n = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            out = philox4x32_10(w[0:4], w[4:6])
            assert [int(o) for o in out] == w[6:10]
            n += 1
    assert n == 3


def test_gaussian_vector_statistics():
    v = gaussian_vector(12345, 0, 0, (8, 8, 8, 8), 12)
    assert abs(v.real.mean()) < 0.01 and abs(v.imag.mean()) < 0.01
    assert abs(v.real.var() - 0.5) < 0.01 and abs(v.imag.var() - 0.5) < 0.01
    assert abs(np.mean(v.real * v.imag)) < 0.01
    w = gaussian_vector(12345, 0, 1, (8, 8, 8, 8), 12)
    assert abs(np.vdot(v, w)) / v.size < 0.02


# ----------------------------------------------------------------------------- Krylov
def test_fgcr_matches_dense_solve():
    rng = np.random.default_rng(3)
    n = 60
    A = np.eye(n) * 3 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, info = fgcr(lambda v: A @ v, b, tol_abs=1e-13 * np.linalg.norm(b), restart=8, maxiter=500)
    assert info.converged
    assert np.allclose(x, np.linalg.solve(A, b), atol=1e-11)
    # flexible: a varying preconditioner still converges
    k = [0]

    def pre(r):
        k[0] += 1
        return r * (1.0 + 0.3 * np.sin(k[0]))
    x2, info2 = fgcr(lambda v: A @ v, b, precond=pre, tol_abs=1e-13 * np.linalg.norm(b), restart=8)
    assert info2.converged and np.allclose(x2, x, atol=1e-11)


def test_mr_reduces_residual_monotonically():
    rng = np.random.default_rng(4)
    n = 40
    A = np.eye(n) * 2 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(4 * n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    prev = np.linalg.norm(b)
    for nu in range(1, 6):
        e = mr(lambda v: A @ v, b, nu)
        cur = np.linalg.norm(b - A @ e)
        assert cur <= prev + 1e-14
        prev = cur
    assert prev < 0.2 * np.linalg.norm(b)


# ----------------------------------------------------------------------------- transfer
@pytest.fixture(scope="module")
def two_grid_44():
    """Config 1 shape: 4^4, 2^4 blocks, Nv = 8."""
    dims = (4, 4, 4, 4)
    W = WilsonClover(I.make_gauge(dims, 0.3, 0, 0.5, 1001), 1.0, -0.1)
    P = block_gram_schmidt(W, (2, 2, 2, 2), _random_vectors(W, 8, 77))
    T = Transfer(W, (2, 2, 2, 2), P)
    return W, T


def _dense_P(T):
    nc = 2 * T.nv
    cols = []
    for j in range(int(np.prod(T.cshape)) * nc):
        e = np.zeros(int(np.prod(T.cshape)) * nc, dtype=complex)
        e[j] = 1
        cols.append(T.prolong(e.reshape(T.cshape + (nc,))).ravel())
    return np.stack(cols, axis=1)


def test_P_orthonormal_per_block_and_chirality(two_grid_44):
    """P7: P^dag P = I (the blocks and chiralities make P's columns orthonormal)."""
    W, T = two_grid_44
    Pd = _dense_P(T)
    assert np.abs(Pd.conj().T @ Pd - np.eye(Pd.shape[1])).max() < 1e-13


def test_P_commutes_with_gamma5(two_grid_44):
    """P7: gamma_5 P = P gamma_5c and R is the adjoint of P."""
    W, T = two_grid_44
    nc = 2 * T.nv
    rng = np.random.default_rng(5)
    vc = rng.standard_normal(T.cshape + (nc,)) + 1j * rng.standard_normal(T.cshape + (nc,))
    g5c = np.concatenate([np.ones(T.nv), -np.ones(T.nv)])
    assert np.abs(W.gamma5(T.prolong(vc)) - T.prolong(vc * g5c)).max() < 1e-14
    v = _vec(W.dims, 6)
    assert abs(inner(T.restrict(v), vc) - inner(v, T.prolong(vc))) < 1e-12 * abs(inner(v, T.prolong(vc)))


def test_block_gs_breakdown_detected():
    dims = (4, 4, 4, 4)
    W = WilsonClover(I.unit_gauge(dims), 1.0, 0.0)
    V = _random_vectors(W, 4, 8)
    V.append(0.5 * V[1] - 2.0 * V[3])
    with pytest.raises(GSBreakdown):
        block_gram_schmidt(W, (2, 2, 2, 2), V)


@pytest.mark.parametrize("dims,block,op", [((4, 4, 4, 4), (2, 2, 2, 2), "Dp"),
                                           ((4, 4, 4, 4), (2, 2, 2, 2), "D"),
                                           ((4, 4, 4, 4), (4, 2, 2, 2), "Dp"),
                                           ((6, 2, 2, 4), (2, 2, 1, 2), "Dp")])
def test_coarse_operator_equals_dense_galerkin(dims, block, op):
    """P8: the coarse links (X, Y_d) as an operator equal dense P^dag D_p P (or
    P^dag D P), including coarse extent 2 (+mu and -mu hit the same block),
    extent 1 (all hops intra-block) and extent 3."""
    W = WilsonClover(I.make_gauge(dims, 0.4, 0, 0.5, 51), 1.0, -0.15)
    nv = 4
    P = block_gram_schmidt(W, block, _random_vectors(W, nv, 52))
    T = Transfer(W, block, P)
    C = build_coarse(W, T, op)
    Pd = _dense_P(T)
    Dd = W.as_dense(W.Dp if op == "Dp" else W.D)
    ref = Pd.conj().T @ Dd @ Pd
    got = C.as_dense(C.D)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_restriction_with_gamma5_gives_same_correction(two_grid_44):
    """R = P^dag gamma_5 and R = P^dag give the same coarse correction."""
    W, T = two_grid_44
    Pd = _dense_P(T)
    Dp = W.as_dense(W.Dp)
    g5 = np.tile(np.concatenate([np.ones(6), -np.ones(6)]), int(np.prod(W.shape)))
    r = _vec(W.dims, 9).ravel()
    R1 = Pd.conj().T * g5[None, :]
    c1 = Pd @ np.linalg.solve(R1 @ Dp @ Pd, R1 @ r)
    c0 = Pd @ np.linalg.solve(Pd.conj().T @ Dp @ Pd, Pd.conj().T @ r)
    assert np.abs(c1 - c0).max() < 1e-11 * np.abs(c0).max()


def test_coarse_even_odd_solve_matches_dense():
    """Coarse even-odd algebra: reduced solve + reconstruction = dense solve of D_hat."""
    dims = (4, 4, 4, 4)
    W = WilsonClover(I.make_gauge(dims, 0.3, 0, 0.5, 61), 1.0, -0.1)
    T = Transfer(W, (2, 2, 2, 2), block_gram_schmidt(W, (2, 2, 2, 2), _random_vectors(W, 4, 62)))
    C = build_coarse(W, T)
    rng = np.random.default_rng(1)
    b = rng.standard_normal(C.shape + (C.ndof,)) + 1j * rng.standard_normal(C.shape + (C.ndof,))
    ref = np.linalg.solve(C.as_dense(C.D), b.ravel()).reshape(b.shape)
    x, info = eo_solve(C, b, tol=1e-13)
    assert info.converged and np.abs(x - ref).max() < 1e-10 * np.abs(ref).max()


# ----------------------------------------------------------------------------- solver
def test_complete_basis_two_grid_converges_in_one_iteration():
    """P9: with Nv = 6 * 16 on 2^4 blocks P is unitary, D_hat is unitarily
    similar to D_p and an exact coarse solve makes MG-GCR converge in 1 step."""
    dims = (4, 4, 4, 4)
    W = WilsonClover(I.make_gauge(dims, 0.3, 0, 0.5, 71), 1.0, -0.1)
    nv = 96
    V = _random_vectors(W, nv, 72)
    prm = MGParams(blocks=[(2, 2, 2, 2)], nv=[nv], tol_coarse=1e-14, maxit_coarse=400, restart_coarse=400,
                   nu_post=0)
    mg = Multigrid(W, prm, null_vectors=[V])
    Pd = _dense_P(mg.transfers[0])
    assert np.abs(Pd @ Pd.conj().T - np.eye(Pd.shape[0])).max() < 1e-12
    b = _vec(dims, 73)
    x, info = mg.solve(b, tol=1e-10)
    assert info.converged and info.outer_iterations == 1


@pytest.mark.parametrize("nu_post", [4, 1])
def test_complete_basis_cycle_with_post_smoothing_is_exact(nu_post):
    """P9 with post-smoothing: with a unitary P and an exact coarse solve the
    coarse correction already is D_r^{-1} r_e, so the MR steps on the residual
    r_e - D_r z_e must leave it unchanged (one cycle equals the dense inverse
    of D_r) and MG-GCR still converges in one outer iteration.  A smoother run
    on r_e instead of the updated residual, or before the prolongated
    correction is added, fails both."""
    dims = (4, 4, 4, 4)
    W = WilsonClover(I.make_gauge(dims, 0.3, 0, 0.5, 71), 1.0, -0.1)
    nv = 96
    V = _random_vectors(W, nv, 72)
    prm = MGParams(blocks=[(2, 2, 2, 2)], nv=[nv], tol_coarse=1e-14, maxit_coarse=400, restart_coarse=400,
                   nu_post=nu_post)
    mg = Multigrid(W, prm, null_vectors=[V])
    r = _vec(dims, 74) * W.even
    z = mg.cycle(0, r)
    sel = np.flatnonzero((np.ones(W.shape + (12,)) * W.even).ravel())   # even-site components
    cols = []
    for j in sel:                                   # dense D_r on the even sites, column by column
        e = np.zeros(r.size, dtype=np.complex128)
        e[j] = 1.0
        cols.append(W.Dr(e.reshape(r.shape)).ravel()[sel])
    ze = np.linalg.solve(np.stack(cols, axis=1), r.ravel()[sel])
    assert np.abs(z.ravel()[sel] - ze).max() < 1e-10 * np.abs(ze).max()
    assert np.abs(z.ravel()[np.setdiff1d(np.arange(r.size), sel)]).max() == 0.0
    x, info = mg.solve(_vec(dims, 73), tol=1e-10)
    assert info.converged and info.outer_iterations == 1


def test_mg_gcr_config1_matches_dense(two_grid_44):
    """P10: 2-level MG-GCR with setup on config 1 (4^4, 2^4 blocks, Nv = 8) reaches
    true residual <= 1e-10 and matches dense LU within cond * 1e-10."""
    W, _ = two_grid_44
    hist = []
    mg = Multigrid(W, MGParams(blocks=[(2, 2, 2, 2)], nv=[8], seed=1003), setup_history=hist)
    b = _vec(W.dims, 1002)
    x, info = mg.solve(b, tol=1e-10)
    assert info.converged and info.true_residual <= 1e-10
    Dd = W.as_dense(W.D)
    xr = np.linalg.solve(Dd, b.ravel())
    cond = np.linalg.cond(Dd)
    assert np.linalg.norm(x.ravel() - xr) / np.linalg.norm(xr) < cond * 1e-10
    # MG needs far fewer outer iterations than unpreconditioned EO-GCR
    _, info_eo = eo_solve(W, b, tol=1e-10)
    assert info.outer_iterations * 2 < info_eo.outer_iterations


def test_setup_vectors_orthonormal_and_rq_settles():
    """P12: setup vectors are globally orthonormal; the Rayleigh quotient of the
    first vector falls far below that of a random vector."""
    dims = (4, 4, 4, 4)
    W = WilsonClover(I.make_gauge(dims, 0.3, 0, 0.5, 81), 1.0, -0.1)
    hist = []
    V = setup_null_vectors(W, 4, 5, 0, iters=20, inner_iters=8, rq_tol=0.05, history=hist)
    G = np.array([[inner(a, b) for b in V] for a in V])
    assert np.abs(G - np.eye(4)).max() < 1e-13
    v0 = gaussian_vector(5, 0, 0, W.shape, 12)
    rq0 = norm2(W.Dp(v0)) / norm2(v0)
    assert hist[0][-1] < 0.05 * rq0


def test_inverse_iteration_finds_smallest_eigenvector():
    """With an exact inner solve, the setup's inverse iteration converges into the
    invariant subspace of D_p belonging to the smallest |eigenvalue| (dense eig,
    2^3x4).  D_p = D A^{-1} is similar to (D_p)^dag conjugated by gamma_5, so its
    eigenvalues come in complex-conjugate pairs: the subspace is 2-dimensional."""
    dims = (2, 2, 2, 4)
    W = WilsonClover(I.make_gauge(dims, 0.5, 0, 0.5, 91), 1.0, -0.3)
    lam, vecs = np.linalg.eig(W.as_dense(W.Dp))
    order = np.argsort(np.abs(lam))
    l0, l1, l2 = lam[order[:3]]
    assert abs(l1 - np.conj(l0)) < 1e-10          # the conjugate pair
    assert abs(l2) > 1.2 * abs(l0)                 # a gap to the next modulus
    Q, _ = np.linalg.qr(vecs[:, order[:2]])
    V = setup_null_vectors(W, 1, 9, 0, iters=110, inner_iters=384, rq_tol=0.0)
    v = V[0].ravel()
    assert np.linalg.norm(v - Q @ (Q.conj().T @ v)) < 1e-9  # ratio 0.79 per pass


def test_free_field_mg_solve_matches_fft():
    """P2 for MG-GCR: the 2-level solve of the free operator equals the
    momentum-space inverse."""
    from test_oracle_dirac import _free_solution
    dims = (4, 4, 4, 8)
    m0 = 0.1
    W = WilsonClover(I.unit_gauge(dims), 1.0, m0)
    mg = Multigrid(W, MGParams(blocks=[(2, 2, 2, 2)], nv=[6], seed=11, setup_iters=4))
    eta = I.gaussian_source(dims, 17)
    x, info = mg.solve(eta.reshape(W.shape + (12,)), tol=1e-12)
    assert info.converged
    ref = _free_solution(dims, m0, eta)
    assert np.abs(x.reshape(ref.shape) - ref).max() / np.abs(ref).max() < 1e-10


def _random_system(n, seed):
    rng = np.random.default_rng(seed)
    M = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2 * n)
    M += 2.0 * np.eye(n)                              # non-Hermitian, eigenvalues around 2
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return M, b


def test_bicgstab_and_cgnr_against_linalg_solve():
    from oracle.krylov import bicgstab, cgnr
    M, b = _random_system(60, 11)
    ref = np.linalg.solve(M, b)
    A = lambda v: M @ v
    x, info = bicgstab(A, b, tol_abs=1e-12 * np.linalg.norm(b), maxiter=200)
    assert info.converged and np.abs(x - ref).max() < 1e-10 * np.abs(ref).max()
    x, info = cgnr(A, lambda v: M.conj().T @ v, b, tol_abs=1e-12 * np.linalg.norm(b), maxiter=400)
    assert info.converged and np.abs(x - ref).max() < 1e-10 * np.abs(ref).max()
    # a wrong adjoint (the transpose without conjugation) breaks CGNR on this complex system
    _, bad = cgnr(A, lambda v: M.T @ v, b, tol_abs=1e-12 * np.linalg.norm(b), maxiter=400)
    assert not bad.converged


def test_comparison_solvers_on_the_reduced_dirac_system():
    """BiCGStab and CGNR (with D_r^dag = gamma_5 A_e^{-1} D_r A_e gamma_5) solve
    D_r y_e = b_r; the reconstructed solution satisfies D x = b."""
    from oracle.krylov import bicgstab, cgnr
    dims = (4, 4, 4, 4)
    W = WilsonClover(I.make_gauge(dims, 0.5, 1, 0.5, 21), 1.0, 0.1)
    b = I.gaussian_source(dims, 22).reshape(W.shape + (12,))
    br = W.b_r(b)
    A = lambda v: W.Dr(v * W.even) * W.even
    Adag = lambda v: W.gamma5(W.Minv(W.Dr(W.M(W.gamma5(v * W.even)))) * W.even)
    tol = 1e-11 * np.sqrt(norm2(br))
    for y, info in (bicgstab(A, br, tol_abs=tol, maxiter=500), cgnr(A, Adag, br, tol_abs=tol, maxiter=2000)):
        assert info.converged
        x = W.reconstruct(y, b)
        assert np.sqrt(norm2(b - W.D(x)) / norm2(b)) < 1e-10
