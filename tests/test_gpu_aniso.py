"""GPU parity of the anisotropic Wilson-clover operator (mg_set_clover_aniso)
against the oracle's anisotropic reading, through the C ABI.

The reading: every hop in direction mu carries the weight w_mu, the mass term
is sum_mu w_mu + m0, and the planes that contain t take csw_t.

* D, D_p, D_r, b_r, M, M^{-1} and the hopping term: FP64 <= 1e-12, FP32 <= 1e-5.
* Unit weights with csw_t = csw give the isotropic context's results bit for bit.
* Galerkin coarse links from injected vectors against the oracle's (FP32 storage).
* An MG-GCR solve to 1e-10, its true residual taken with the oracle's D.
* mg_force (FP64 and FP32) against the oracle's link derivative.
"""
import numpy as np
import pytest

from gpu_common import TOL32, TOL64, lib_built, rel
from oracle import force as OF
from oracle.dirac import WilsonClover, dag, norm2
from oracle.multigrid import MGParams, Multigrid
from oracle.philox import gaussian_vector
from paper_1011_2775_gb300 import inputs as I

pytestmark = pytest.mark.gpu

AW = (0.45, 0.7, 1.25, 2.0)   # all different, so a transposed direction index fails

CASES = [
    # dims, eps, ape, csw_s, csw_t, m0, seed
    ((6, 4, 8, 10), 0.4, 1, 1.3, 0.6, -0.2, 8101),   # half volume 960: ragged last CTA
    ((8, 8, 8, 8), 0.25, 2, 1.0, 1.7, -0.35, 8102),
]


def _solver(dims, U, weights, csw_s, csw_t, m0):
    lib_built()
    from paper_1011_2775_gb300.solver import Solver
    S = Solver(dims)
    S.load_gauge(U)
    S.set_clover_aniso(weights, csw_s, csw_t, m0)
    return S


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "x".join(map(str, c[0])))
def aniso(request):
    dims, eps, ape, csw_s, csw_t, m0, seed = request.param
    U = I.make_gauge(dims, eps, ape, 0.5, seed)
    W = WilsonClover(U, csw_s, m0, weights=AW, csw_t=csw_t)
    S = _solver(dims, U, AW, csw_s, csw_t, m0)
    yield dims, U, W, S
    S.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("op", ["D", "DP", "DR", "BR", "M", "MINV", "HOP"])
def test_aniso_operator_parity(aniso, op, prec):
    from paper_1011_2775_gb300 import binding as B
    dims, U, W, S = aniso
    x = I.gaussian_source(dims, 8199)
    v = x.reshape(W.shape + (12,))
    ref = {"D": W.D, "DP": W.Dp, "DR": lambda y: W.Dr(y * W.even), "BR": W.b_r, "M": W.M, "MINV": W.Minv,
           "HOP": W.hop}[op](v).reshape(x.shape)
    got = S.apply(getattr(B, "MG_OP_" + op), x, prec=prec)
    assert rel(got, ref) <= (TOL64 if prec == 0 else TOL32)


def test_unit_weights_are_the_isotropic_operator_bit_for_bit():
    from paper_1011_2775_gb300 import binding as B
    dims, eps, ape, csw, _, m0, seed = CASES[0]
    U = I.make_gauge(dims, eps, ape, 0.5, seed)
    x = I.gaussian_source(dims, 8198)
    with _solver(dims, U, (1.0, 1.0, 1.0, 1.0), csw, csw, m0) as Sa:
        lib_built()
        from paper_1011_2775_gb300.solver import Solver
        with Solver(dims) as Si:
            Si.load_gauge(U)
            Si.set_clover(csw, m0)
            for op in (B.MG_OP_D, B.MG_OP_DR, B.MG_OP_MINV):
                for prec in (B.MG_FP64, B.MG_FP32):
                    assert np.array_equal(Sa.apply(op, x, prec=prec), Si.apply(op, x, prec=prec))
            lam = I.gaussian_source(dims, 8197)
            assert np.array_equal(Sa.force(lam, x, kind=B.MG_FORCE_SU3), Si.force(lam, x, kind=B.MG_FORCE_SU3))


def test_aniso_coarse_links_match_oracle():
    """Galerkin coarse operator of the anisotropic D_p from injected vectors
    (2 levels on 8^4, blocks 2^4, Nv = 8), applied to a random coarse vector."""
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 8)
    U = I.make_gauge(dims, 0.3, 1, 0.5, 8103)
    W = WilsonClover(U, 1.1, -0.25, weights=AW, csw_t=0.8)
    V0 = [gaussian_vector(81, 0, k, W.shape, 12) for k in range(8)]
    mg = Multigrid(W, MGParams(blocks=[(2, 2, 2, 2)], nv=[8]), null_vectors=[V0])
    with _solver(dims, U, AW, 1.1, 0.8, -0.25) as S:
        S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[8])
        S.set_null_vectors(0, np.ascontiguousarray(np.stack(V0)))
        S.setup()
        C = mg.levels[1]
        rng = np.random.default_rng(8104)
        v = rng.standard_normal(C.shape + (C.ndof,)) + 1j * rng.standard_normal(C.shape + (C.ndof,))
        for op in ("D", "M"):
            got = S.apply(getattr(B, "MG_OP_" + op), np.ascontiguousarray(v), level=1)
            assert rel(got, getattr(C, op)(v)) <= TOL32


@pytest.mark.parametrize("levels", [2, 3])
def test_aniso_mg_solve_true_residual(levels):
    """A t-fine lattice (spatial weights 0.3, w_t = 1, csw_t != csw_s) solved to
    1e-10 by MG-GCR; the residual is taken with the oracle's operator.  The
    rough field puts the critical mass near +0.25 for these weights (smallest
    Re lambda of D at m0 = 0 is -0.247 on 4^3x8), so m0 = 0.35 is 0.1 above it."""
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 16)
    w = (0.3, 0.3, 0.3, 1.0)
    U = I.make_gauge(dims, 1.0, 5, 0.5, 8105)
    W = WilsonClover(U, 1.0, 0.35, weights=w, csw_t=1.4)
    with _solver(dims, U, w, 1.0, 1.4, 0.35) as S:
        if levels == 2:
            S.set_params(levels=2, blocks=[(4, 4, 4, 4)], nv=[12], maxit_fine=2000)
        else:
            S.set_params(levels=3, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[8, 8], maxit_fine=2000)
        S.setup()
        eta = I.gaussian_source(dims, 8106)
        psi, info = S.solve(eta, 1e-10, B.MG_MODE_MG)
    assert info.true_residual <= 1e-10
    r = eta.reshape(W.shape + (12,)) - W.D(psi.reshape(W.shape + (12,)))
    assert np.sqrt(norm2(r) / norm2(eta)) <= 1e-10
    assert info.coarse_iterations[1] > 0


@pytest.mark.parametrize("fp32", [False, True], ids=["fp64", "fp32"])
def test_aniso_force_parity(aniso, fp32):
    from paper_1011_2775_gb300 import binding as B
    dims, U, W, S = aniso
    lam = I.gaussian_source(dims, 8107)
    psi = I.gaussian_source(dims, 8108)
    K = OF.link_derivative(W, lam.reshape(W.shape + (12,)), psi.reshape(W.shape + (12,)))
    extra = B.MG_FORCE_FP32 if fp32 else 0
    tol = TOL32 if fp32 else TOL64
    assert rel(S.force(lam, psi, kind=B.MG_FORCE_WIRTINGER | extra), dag(K)) <= tol
    assert rel(S.force(lam, psi, kind=B.MG_FORCE_SU3 | extra), OF.su3_force(U, K)) <= tol


def test_aniso_bad_weights_rejected():
    from paper_1011_2775_gb300 import binding as B
    dims = (4, 4, 4, 4)
    U = I.make_gauge(dims, 0.3, 0, 0.5, 8109)
    with _solver(dims, U, AW, 1.0, 1.0, -0.1) as S:
        for bad in ((0.0, 1, 1, 1), (1, -1.0, 1, 1), (1, 1, float("nan"), 1), (1, 1, 1, float("inf"))):
            with pytest.raises(B.MGError) as e:
                S.set_clover_aniso(bad, 1.0, 1.0, -0.1)
            assert e.value.status == B.MG_ERR_ARG
        with pytest.raises(B.MGError):
            S.set_clover_aniso(AW, 1.0, float("nan"), -0.1)
