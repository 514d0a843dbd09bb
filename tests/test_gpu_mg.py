"""GPU parity of the multigrid pieces and the solvers, through the C ABI.

* Transfer and coarse operators by injection: the same Philox null vectors go
  to the oracle and (via mg_set_null_vectors) to the GPU; R, P and the
  coarse D_hat, D_hat_p, D_hat_r, X, X^{-1}, hop are compared (FP32 pipeline:
  relative error <= 1e-5), for 2 and 3 levels.
* Setup without injection: P^dag P = I and gamma_5 P = P gamma_5c hold.
* Solves: EO-GCR and MG-GCR reach ||eta - D psi|| / ||eta|| <= 1e-10 with D
  the oracle's FP64 operator applied to the returned psi.
* Failure paths return their status codes.
"""
import numpy as np
import pytest

from gpu_common import TOL32, lib_built, rel
from oracle.dirac import WilsonClover, norm2
from oracle.multigrid import MGParams, Multigrid
from oracle.philox import gaussian_vector
from paper_1011_2775_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _solver(dims, U, csw, m0):
    lib_built()
    from paper_1011_2775_gb300.solver import Solver
    S = Solver(dims)
    S.load_gauge(U)
    S.set_clover(csw, m0)
    return S


def _vectors(seed, level, nv, shape, ndof):
    return [gaussian_vector(seed, level, k, shape, ndof) for k in range(nv)]


def _true_residual(W, psi, eta):
    r = eta.reshape(W.shape + (12,)) - W.D(psi.reshape(W.shape + (12,)))
    return np.sqrt(norm2(r) / norm2(eta))


@pytest.fixture(scope="module")
def injected3():
    """3 levels on 8^4: blocks 2^4 (Nv = 8) then 2^4 (Nv = 6), vectors injected."""
    dims = (8, 8, 8, 8)
    U = I.make_gauge(dims, 0.3, 1, 0.5, 3001)
    W = WilsonClover(U, 1.0, -0.2)
    V0 = _vectors(77, 0, 8, W.shape, 12)
    V1 = _vectors(78, 1, 6, (4, 4, 4, 4), 16)
    prm = MGParams(blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[8, 6])
    mg = Multigrid(W, prm, null_vectors=[V0, V1])
    S = _solver(dims, U, 1.0, -0.2)
    S.set_params(levels=3, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[8, 6])
    S.set_null_vectors(0, np.ascontiguousarray(np.stack(V0)))
    S.set_null_vectors(1, np.ascontiguousarray(np.stack(V1)))
    S.setup()
    yield dims, W, mg, S
    S.close()


def test_level_info(injected3):
    dims, W, mg, S = injected3
    assert S.level_info(1) == ((4, 4, 4, 4), 16)
    assert S.level_info(2) == ((2, 2, 2, 2), 12)


@pytest.mark.parametrize("level", [0, 1])
def test_restrict_prolong_parity(injected3, level):
    from paper_1011_2775_gb300 import binding as B
    dims, W, mg, S = injected3
    T = mg.transfers[level]
    fine = mg.levels[level]
    rng = np.random.default_rng(level)
    v = rng.standard_normal(fine.shape + (fine.ndof,)) + 1j * rng.standard_normal(fine.shape + (fine.ndof,))
    vc = rng.standard_normal(T.cshape + (2 * T.nv,)) + 1j * rng.standard_normal(T.cshape + (2 * T.nv,))
    got_r = S.apply(B.MG_OP_R, np.ascontiguousarray(v), level=level, out_shape=vc.shape)
    assert rel(got_r, T.restrict(v)) <= TOL32
    got_p = S.apply(B.MG_OP_P, np.ascontiguousarray(vc), level=level, out_shape=v.shape)
    assert rel(got_p, T.prolong(vc)) <= TOL32


@pytest.mark.parametrize("level", [1, 2])
@pytest.mark.parametrize("op", ["D", "DP", "DR", "BR", "M", "MINV", "HOP"])
def test_coarse_operator_parity(injected3, level, op):
    from paper_1011_2775_gb300 import binding as B
    dims, W, mg, S = injected3
    C = mg.levels[level]
    rng = np.random.default_rng(10 + level)
    v = rng.standard_normal(C.shape + (C.ndof,)) + 1j * rng.standard_normal(C.shape + (C.ndof,))
    ref = {"D": C.D, "DP": C.Dp, "DR": lambda x: C.Dr(x * C.even), "BR": C.b_r, "M": C.M, "MINV": C.Minv,
           "HOP": C.hop}[op](v)
    got = S.apply(getattr(B, "MG_OP_" + op), np.ascontiguousarray(v), level=level)
    assert rel(got, ref) <= TOL32


@pytest.fixture(scope="module")
def injected3_odd():
    """3 levels on 12x8x8x8 whose coarsest lattice (3x2x2x2) has an odd extent,
    so it is solved without even-odd: blocks 2^4 (Nv = 8) then 2^4 (Nv = 6),
    vectors injected; coarse solves to 1e-6 so that the cycles can be compared."""
    dims = (12, 8, 8, 8)
    U = I.make_gauge(dims, 0.4, 1, 0.5, 3101)
    W = WilsonClover(U, 1.0, -0.2)
    V0 = _vectors(79, 0, 8, W.shape, 12)
    V1 = _vectors(80, 1, 6, (4, 4, 4, 6), 16)
    cp = dict(tol_coarse=1e-6, maxit_coarse=400, restart_coarse=64, nu_post=2)
    mg = Multigrid(W, MGParams(blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[8, 6], **cp), null_vectors=[V0, V1])
    S = _solver(dims, U, 1.0, -0.2)
    S.set_params(levels=3, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[8, 6], **cp)
    S.set_null_vectors(0, np.ascontiguousarray(np.stack(V0)))
    S.set_null_vectors(1, np.ascontiguousarray(np.stack(V1)))
    S.setup()
    yield dims, W, mg, S
    S.close()


@pytest.mark.parametrize("level,op", [(1, "D"), (1, "DP"), (1, "DR"), (1, "BR"), (1, "MINV"), (2, "D"), (2, "DP"),
                                      (2, "M"), (2, "MINV"), (2, "HOP")])
def test_odd_coarsest_operator_parity(injected3_odd, level, op):
    from paper_1011_2775_gb300 import binding as B
    dims, W, mg, S = injected3_odd
    assert S.level_info(2) == ((3, 2, 2, 2), 12)
    C = mg.levels[level]
    rng = np.random.default_rng(20 + level)
    v = rng.standard_normal(C.shape + (C.ndof,)) + 1j * rng.standard_normal(C.shape + (C.ndof,))
    ref = {"D": C.D, "DP": C.Dp, "DR": lambda x: C.Dr(x * C.even), "BR": C.b_r, "M": C.M, "MINV": C.Minv,
           "HOP": C.hop}[op](v)
    got = S.apply(getattr(B, "MG_OP_" + op), np.ascontiguousarray(v), level=level)
    assert rel(got, ref) <= TOL32


def test_odd_coarsest_rejects_even_odd_ops(injected3_odd):
    from paper_1011_2775_gb300 import binding as B
    dims, W, mg, S = injected3_odd
    C = mg.levels[2]
    v = np.ones(C.shape + (C.ndof,), dtype=np.complex128)
    for op in (B.MG_OP_DR, B.MG_OP_BR):
        with pytest.raises(B.MGError) as e:
            S.apply(op, v, level=2)
        assert e.value.status == B.MG_ERR_DIMS


@pytest.mark.parametrize("level", [1, 0])
def test_odd_coarsest_cycle_parity(injected3_odd, level):
    """The K-cycle of level 1 (its coarse solve: GCR on the full coarsest D)
    and of the fine level (a level-1 GCR preconditioned by that cycle) against
    the oracle's, on even-site input."""
    from paper_1011_2775_gb300 import binding as B
    dims, W, mg, S = injected3_odd
    lev = mg.levels[level]
    rng = np.random.default_rng(30 + level)
    r = rng.standard_normal(lev.shape + (lev.ndof,)) + 1j * rng.standard_normal(lev.shape + (lev.ndof,))
    ref = mg.cycle(level, r * lev.even)
    got = S.apply(B.MG_OP_CYCLE, np.ascontiguousarray(r), level=level)
    assert rel(got, ref) <= 1e-4


def test_odd_coarsest_solve_and_adaptive_refinement():
    """A 3-level solve whose coarsest lattice has an odd extent reaches 1e-10
    with the oracle's D, before and after refining both transfers."""
    from paper_1011_2775_gb300 import binding as B
    dims = (12, 8, 8, 16)
    U = I.make_gauge(dims, 1.0, 5, 0.5, 5101)
    W = WilsonClover(U, 1.0, -0.6)
    S = _solver(dims, U, 1.0, -0.6)
    S.set_params(levels=3, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[8, 8], setup_iters=6, maxit_fine=3000)
    S.setup()
    assert S.level_info(2)[0] == (3, 2, 2, 4)
    eta = I.gaussian_source(dims, 5102)
    psi, good = S.solve(eta, 1e-10, B.MG_MODE_MG)
    assert _true_residual(W, psi, eta) <= 1e-10
    S.adapt_setup(passes=1, relax=2, transfers=0)
    psi, adapted = S.solve(eta, 1e-10, B.MG_MODE_MG)
    assert _true_residual(W, psi, eta) <= 1e-10
    assert adapted.outer_iterations <= good.outer_iterations + 2
    S.close()


def test_changed_solve_params_take_effect_with_graphs():
    """Smoothing steps and the coarse tolerance changed between solves (setup
    kept) reach the captured cycle graph: the solve then iterates exactly as a
    context set up with those parameters from the start."""
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 16)
    U = I.make_gauge(dims, 1.0, 5, 0.5, 5301)
    eta = I.gaussian_source(dims, 5302)
    mg = dict(levels=2, blocks=[(4, 4, 4, 4)], nv=[12], seed=5303, maxit_fine=3000)
    S = _solver(dims, U, 1.0, -0.6)
    S.set_params(nu_post=4, tol_coarse=0.1, **mg)
    S.setup()
    _, a = S.solve(eta, 1e-10, B.MG_MODE_MG)
    _, a2 = S.solve(eta, 1e-10, B.MG_MODE_MG)            # graph replays
    assert a2.outer_iterations == a.outer_iterations
    S.set_params(nu_post=1, tol_coarse=0.5)
    _, b = S.solve(eta, 1e-10, B.MG_MODE_MG)
    F = _solver(dims, U, 1.0, -0.6)
    F.set_params(nu_post=1, tol_coarse=0.5, **mg)
    F.setup()
    _, c = F.solve(eta, 1e-10, B.MG_MODE_MG)
    assert b.outer_iterations == c.outer_iterations
    assert b.coarse_iterations[1] == c.coarse_iterations[1]
    assert b.outer_iterations != a.outer_iterations
    S.close()
    F.close()


def test_setup_P_orthonormal_and_chiral():
    """Setup without injection: R P = I on coarse vectors (P^dag P = I) and
    gamma_5 P = P gamma_5c."""
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 8)
    U = I.make_gauge(dims, 0.25, 2, 0.5, 4001)
    S = _solver(dims, U, 1.0, -0.25)
    S.set_params(levels=2, blocks=[(4, 4, 4, 4)], nv=[12], setup_iters=6)
    info = S.setup()
    assert info.vectors[0] == 12 and info.coarse_sites[0] == 16 and info.passes[0] >= 12
    rng = np.random.default_rng(0)
    cs = (2, 2, 2, 2, 24)
    vc = rng.standard_normal(cs) + 1j * rng.standard_normal(cs)
    pv = S.apply(B.MG_OP_P, vc, level=0, out_shape=(8, 8, 8, 8, 4, 3))
    assert rel(S.apply(B.MG_OP_R, pv, level=0, out_shape=cs), vc) <= TOL32
    g5c = np.concatenate([np.ones(12), -np.ones(12)])
    pg = S.apply(B.MG_OP_P, np.ascontiguousarray(vc * g5c), level=0, out_shape=pv.shape)
    g5 = np.array([1, 1, -1, -1])[:, None]
    assert rel(pg, pv * g5) <= TOL32
    # the vectors are globally orthonormal (setup keeps them orthogonal)
    V = S.get_null_vectors(0).reshape(12, -1)
    G = V.conj() @ V.T
    assert np.abs(G - np.eye(12)).max() < 1e-4
    S.close()


@pytest.mark.parametrize("mode", ["eo", "mg2", "mg3"])
def test_solve_true_residual(mode):
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 16)
    U = I.make_gauge(dims, 1.0, 5, 0.5, 5001)
    W = WilsonClover(U, 1.0, -0.6)
    S = _solver(dims, U, 1.0, -0.6)
    S.set_params(maxit_fine=5000)
    if mode == "mg2":
        S.set_params(levels=2, blocks=[(4, 4, 4, 4)], nv=[12])
        S.setup()
    elif mode == "mg3":
        S.set_params(levels=3, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[8, 8])
        S.setup()
    eta = I.gaussian_source(dims, 5002)
    psi, info = S.solve(eta, 1e-10, B.MG_MODE_EO_GCR if mode == "eo" else B.MG_MODE_MG)
    assert info.true_residual <= 1e-10
    assert _true_residual(W, psi, eta) <= 1e-10
    if mode != "eo":
        assert info.coarse_iterations[1] > 0
    S.close()


def test_config1_mg_matches_oracle_solution():
    """Config 1 (4^4, 2^4 blocks, Nv = 8): GPU and oracle MG-GCR solutions agree
    within the conditioning of the 1e-10 residual."""
    from paper_1011_2775_gb300 import binding as B
    dims = (4, 4, 4, 4)
    U = I.make_gauge(dims, 0.3, 0, 0.5, 1001)
    W = WilsonClover(U, 1.0, -0.1)
    S = _solver(dims, U, 1.0, -0.1)
    S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[8], seed=1003)
    S.setup()
    eta = I.gaussian_source(dims, 1002)
    psi, info = S.solve(eta, 1e-10, B.MG_MODE_MG)
    x, oinfo = Multigrid(W, MGParams(blocks=[(2, 2, 2, 2)], nv=[8], seed=1003)).solve(eta.reshape(W.shape + (12,)))
    assert _true_residual(W, psi, eta) <= 1e-10 and oinfo.true_residual <= 1e-10
    assert np.linalg.norm(psi.ravel() - x.ravel()) / np.linalg.norm(x) < 1e-7
    S.close()


def test_error_paths():
    from paper_1011_2775_gb300 import binding as B
    dims = (4, 4, 4, 4)
    lib_built()
    from paper_1011_2775_gb300.solver import Solver
    S = Solver(dims)
    eta = I.gaussian_source(dims, 1)
    with pytest.raises(B.MGError) as e:
        S.set_clover(1.0, 0.0)
    assert e.value.status == B.MG_ERR_STATE
    S.load_gauge(I.unit_gauge(dims))
    with pytest.raises(B.MGError) as e:
        S.set_clover(1.0, -4.0)            # A = 0: singular clover
    assert e.value.status == B.MG_ERR_SINGULAR_CLOVER
    S.set_clover(1.0, 0.1)
    with pytest.raises(B.MGError) as e:
        S.solve(eta, 1e-10, B.MG_MODE_MG)  # no setup
    assert e.value.status == B.MG_ERR_STATE
    with pytest.raises(B.MGError) as e:
        S.set_params(levels=2, blocks=[(3, 2, 2, 2)], nv=[4])
    assert e.value.status == B.MG_ERR_DIMS
    with pytest.raises(B.MGError) as e:
        S.set_params(levels=2, blocks=[(1, 1, 1, 2)], nv=[13])  # a block's chiral subspace has dim 12
    assert e.value.status == B.MG_ERR_NV
    S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[4])
    buf = np.zeros((4, 4, 4, 4, 4, 12), dtype=np.complex128)
    for lvl in (-1, 1):                    # no transfer from these levels
        for call in (B.mg_get_null_vectors, B.mg_set_null_vectors):
            with pytest.raises(B.MGError) as e:
                call(S.ctx, lvl, buf, 4)
            assert e.value.status == B.MG_ERR_ARG
    V = np.stack([gaussian_vector(3, 0, k, (4, 4, 4, 4), 12) for k in range(4)])
    V[3] = 2.0 * V[1] - 0.5 * V[0]        # locally dependent (to FP32 rounding)
    S.set_null_vectors(0, np.ascontiguousarray(V))
    with pytest.raises(B.MGError) as e:
        S.setup()
    assert e.value.status == B.MG_ERR_GS_BREAKDOWN
    bad = eta.copy()
    bad[0, 0, 0, 0, 0, 0] = np.nan
    with pytest.raises(B.MGError) as e:
        S.solve(bad, 1e-10, B.MG_MODE_EO_GCR)
    assert e.value.status == B.MG_ERR_NAN
    S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[4], maxit_fine=3)
    psi = np.zeros_like(eta)
    st, info = B.mg_solve(S.ctx, psi, eta, 1, 1e-12, B.MG_MODE_EO_GCR, allow_not_converged=True)
    assert st == B.MG_ERR_NOT_CONVERGED and info.outer_iterations <= 3 and np.isfinite(info.true_residual)
    S.close()


@pytest.fixture(scope="module")
def qcdlike():
    """QCD-like field (plaquette ~0.7): 8^4, eps = 1.0 + 5 APE steps, m0 = -0.6;
    2 levels with 2^4 blocks and Nv = 8 injected Philox vectors."""
    dims = (8, 8, 8, 8)
    U = I.make_gauge(dims, 1.0, 5, 0.5, 2001)
    W = WilsonClover(U, 1.0, -0.6)
    V0 = _vectors(91, 0, 8, W.shape, 12)
    return dims, U, W, V0


@pytest.mark.parametrize("nu", [0, 2])
def test_cycle_parity(qcdlike, nu):
    """One application of the preconditioner K (restrict, near-exact coarse
    solve, prolong, nu MR steps) matches the oracle's cycle."""
    from paper_1011_2775_gb300 import binding as B
    dims, U, W, V0 = qcdlike
    prm = dict(tol_coarse=1e-6, maxit_coarse=400, restart_coarse=64, nu_post=nu)
    mg = Multigrid(W, MGParams(blocks=[(2, 2, 2, 2)], nv=[8], **prm), null_vectors=[V0])
    S = _solver(dims, U, 1.0, -0.6)
    S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[8], **prm)
    S.set_null_vectors(0, np.ascontiguousarray(np.stack(V0)))
    S.setup()
    r = I.gaussian_source(dims, 7)
    got = S.apply(B.MG_OP_CYCLE, r, level=0)
    ref = mg.cycle(0, r.reshape(W.shape + (12,)) * W.even).reshape(r.shape)
    assert rel(got, ref) <= 1e-4
    S.close()


def test_mg_iterations_match_oracle(qcdlike):
    """With the same injected null vectors the GPU MG-GCR needs about as many
    outer iterations as the oracle's (FP32 preconditioner vs FP64)."""
    from paper_1011_2775_gb300 import binding as B
    dims, U, W, V0 = qcdlike
    mg = Multigrid(W, MGParams(blocks=[(2, 2, 2, 2)], nv=[8]), null_vectors=[V0])
    eta = I.gaussian_source(dims, 8)
    _, oinfo = mg.solve(eta.reshape(W.shape + (12,)), 1e-10)
    S = _solver(dims, U, 1.0, -0.6)
    S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[8])
    S.set_null_vectors(0, np.ascontiguousarray(np.stack(V0)))
    S.setup()
    psi, info = S.solve(eta, 1e-10, B.MG_MODE_MG)
    assert _true_residual(W, psi, eta) <= 1e-10
    assert abs(info.outer_iterations - oinfo.outer_iterations) <= max(3, 0.2 * oinfo.outer_iterations)
    S.close()


@pytest.mark.parametrize("rhs_block", [1, 3])
def test_outer_products_in_fp32_and_fp64(qcdlike, rhs_block):
    """mg_params.outer_prec: the outer FGCR's products D_r z in FP32 (the
    default) or FP64.  Both reach 1e-10 with the oracle's D (the true residuals
    are FP64 either way) in about as many outer iterations as the oracle, single
    and block solves alike."""
    from paper_1011_2775_gb300 import binding as B
    dims, U, W, V0 = qcdlike
    mg = Multigrid(W, MGParams(blocks=[(2, 2, 2, 2)], nv=[8]), null_vectors=[V0])
    eta = I.gaussian_source(dims, 9, nrhs=rhs_block)
    _, oinfo = mg.solve(eta[0].reshape(W.shape + (12,)), 1e-10)
    S = _solver(dims, U, 1.0, -0.6)
    S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[8], rhs_block=rhs_block)
    S.set_null_vectors(0, np.ascontiguousarray(np.stack(V0)))
    S.setup()
    its = {}
    for prec in (B.MG_FP32, B.MG_FP64):
        S.set_params(outer_prec=prec)
        psi, info = S.solve(eta, 1e-10, B.MG_MODE_MG)
        for q in range(rhs_block):
            assert _true_residual(W, psi[q], eta[q]) <= 1e-10, (prec, q)
        its[prec] = info.outer_iterations / rhs_block
        assert abs(its[prec] - oinfo.outer_iterations) <= max(3, 0.25 * oinfo.outer_iterations), (prec, its)
    S.close()


def test_level_timing():
    """mg_params.level_timing: CUDA-event times of every level's work in
    mg_solve_info.level_ms, nested (the level-l coarse solves run inside the
    level-(l-1) work), the same solution as an untimed solve, and zeros when off."""
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 16)
    U = I.make_gauge(dims, 1.0, 5, 0.5, 5201)
    W = WilsonClover(U, 1.0, -0.6)
    eta = I.gaussian_source(dims, 5202)
    for levels, blocks, nv in ((2, [(4, 4, 4, 4)], [12]), (3, [(2, 2, 2, 2), (2, 2, 2, 2)], [8, 8])):
        S = _solver(dims, U, 1.0, -0.6)
        S.set_params(levels=levels, blocks=blocks, nv=nv, seed=5203, maxit_fine=2000)
        S.setup()
        psi0, info0 = S.solve(eta, 1e-10, B.MG_MODE_MG)
        assert all(t == 0.0 for t in info0.level_ms)
        S.set_params(level_timing=1)
        psi1, info1 = S.solve(eta, 1e-10, B.MG_MODE_MG)
        assert _true_residual(W, psi1, eta) <= 1e-10
        assert info1.outer_iterations == info0.outer_iterations
        t = list(info1.level_ms)
        assert t[0] > 0 and 0 < t[1] <= t[0], t
        if levels == 3:
            assert 0 < t[2] <= t[1], t
        assert t[0] <= info1.solve_ms
        S.close()


def test_cycle_graph_replay_matches_direct_launches():
    """The single-rhs solve replays its 2-level cycle as a captured CUDA graph
    (mg_params.cuda_graphs = 1, the default); the same kernels launched one by
    one give the same solution and iteration count."""
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 16)
    U = I.make_gauge(dims, 1.0, 5, 0.5, 5001)
    W = WilsonClover(U, 1.0, -0.6)
    S = _solver(dims, U, 1.0, -0.6)
    S.set_params(levels=2, blocks=[(4, 4, 4, 4)], nv=[12], seed=5101)
    S.setup()
    eta = I.gaussian_source(dims, 5102)
    psi_g, info_g = S.solve(eta, 1e-10, B.MG_MODE_MG)
    psi_g2, info_g2 = S.solve(eta, 1e-10, B.MG_MODE_MG)   # graph captured by now: pure replay
    S.set_params(cuda_graphs=0)
    psi_d, info_d = S.solve(eta, 1e-10, B.MG_MODE_MG)
    assert _true_residual(W, psi_g2, eta) <= 1e-10
    assert info_g2.outer_iterations == info_d.outer_iterations
    assert np.abs(psi_g2 - psi_d).max() <= 1e-13 * np.abs(psi_d).max()
    S.close()


def test_four_level_solve():
    """Four levels (16^4 -> 8^4 -> 4^4 -> 2^4, 2^4 blocks, Nv = 8 each): the
    recursive cycle with two intermediate GCR levels reaches the tolerance with
    the oracle's D, and every coarse level iterates."""
    from paper_1011_2775_gb300 import binding as B
    dims = (16, 16, 16, 16)
    U = I.make_gauge(dims, 1.0, 5, 0.5, 5601)
    W = WilsonClover(U, 1.0, -0.5)
    S = _solver(dims, U, 1.0, -0.5)
    S.set_params(levels=4, blocks=[(2, 2, 2, 2)] * 3, nv=[8, 8, 8], seed=5602, maxit_fine=2000, setup_iters=6)
    info = S.setup()
    assert info.coarse_sites[0] == 4096 and info.coarse_sites[2] == 16
    assert S.level_info(3) == ((2, 2, 2, 2), 16)
    eta = I.gaussian_source(dims, 5603)
    psi, si = S.solve(eta, 1e-10, B.MG_MODE_MG)
    assert _true_residual(W, psi, eta) <= 1e-10
    assert si.coarse_iterations[1] > 0 and si.coarse_iterations[2] > 0 and si.coarse_iterations[3] > 0
    S.close()


def test_setup_rayleigh_quotients_with_the_oracle_dp():
    """Row a8 on the GPU, judged by the oracle ("Setup procedure": inverse
    iteration watched through the Rayleigh quotient v^dag D_p^dag D_p v / v^dag v).
    The GPU's null vectors, evaluated with the oracle's FP64 D_p: after one
    relaxation pass (GCR(8) from the same Philox start vectors) their
    quotients equal those of the oracle's own FP64 setup to FP32 accuracy;
    they fall as the number of passes grows; after ten passes they stay
    within a factor two of the oracle's ten-pass quotients (the FP32 and FP64
    iterations drift apart) and far below a random vector's."""
    from oracle.multigrid import setup_null_vectors
    dims = (8, 8, 8, 8)
    U = I.make_gauge(dims, 0.25, 5, 0.5, 4101)
    m0 = -0.3
    W = WilsonClover(U, 1.0, m0)
    nv, seed = 8, 4103

    def rq(v):
        v = v.reshape(W.shape + (12,))
        return norm2(W.Dp(v)) / norm2(v)

    rq_random = np.mean([rq(gaussian_vector(seed, 0, k, W.shape, 12)) for k in range(nv)])
    got = {}
    for iters in (1, 3, 10):   # rq_tol 0: every vector takes exactly `iters` passes
        S = _solver(dims, U, 1.0, m0)
        S.set_params(levels=2, blocks=[(4, 4, 4, 4)], nv=[nv], seed=seed, setup_iters=iters, setup_rq_tol=0.0)
        info = S.setup()
        assert info.passes[0] == nv * iters
        got[iters] = np.array([rq(v) for v in S.get_null_vectors(0)])
        S.close()
    ref1 = np.array([rq(v) for v in setup_null_vectors(W, nv, seed, 0, iters=1, inner_iters=8, rq_tol=0.0)])
    assert np.abs(got[1] - ref1).max() <= 1e-4 * ref1.max()
    assert got[10].mean() < got[3].mean() < got[1].mean() < rq_random
    ref10 = np.array([rq(v) for v in setup_null_vectors(W, nv, seed, 0, iters=10, inner_iters=8, rq_tol=0.0)])
    assert got[10].mean() < 2.0 * ref10.mean()
    assert got[10].mean() < 0.05 * rq_random
