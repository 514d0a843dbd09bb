"""GPU parity of the differentiated solve, through the C ABI.

* mg_force (hop + clover link derivative, FP64) against the oracle's
  link_derivative / su3_force: relative error <= 1e-12 on lattices that span
  several CTAs with a ragged tail; its FP32 form (MG_FORCE_FP32) <= 1e-5.
* mg_solve_dagger: ||chi - D^dag lam|| / ||chi|| <= 1e-10 with the oracle's D.
* The torch.autograd Function: grad_eta and grad_U against the oracle's
  gradients from dense solves (limited by the solve tolerance), and the su(3)
  force against central differences of L computed by GPU solves of perturbed
  gauge fields.
"""
import numpy as np
import pytest

from gpu_common import TOL32, TOL64, lib_built, rel
from oracle import force as OF
from oracle.dirac import WilsonClover, dag, norm2
from paper_1011_2775_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = [
    # dims, eps, ape, csw, m0, seed
    ((4, 4, 4, 4), 0.4, 0, 1.0, -0.1, 5101),
    ((6, 4, 8, 10), 0.5, 1, 1.3, -0.2, 5102),
    ((8, 8, 8, 8), 0.25, 2, 1.0, -0.35, 5103),
]


def _solver(dims, U, csw, m0):
    lib_built()
    from paper_1011_2775_gb300.solver import Solver
    S = Solver(dims)
    S.load_gauge(U)
    S.set_clover(csw, m0)
    return S


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])))
def test_force_parity(case):
    from paper_1011_2775_gb300 import binding as B
    dims, eps, ape, csw, m0, seed = case
    U = I.make_gauge(dims, eps, ape, 0.5, seed)
    W = WilsonClover(U, csw, m0)
    lam = I.gaussian_source(dims, seed + 1)
    psi = I.gaussian_source(dims, seed + 2)
    K = OF.link_derivative(W, lam.reshape(W.shape + (12,)), psi.reshape(W.shape + (12,)))
    with _solver(dims, U, csw, m0) as S:
        got_w = S.force(lam, psi, kind=B.MG_FORCE_WIRTINGER)
        got_f = S.force(lam, psi, kind=B.MG_FORCE_SU3)
    assert rel(got_w, dag(K)) <= TOL64
    assert rel(got_f, OF.su3_force(U, K)) <= TOL64


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])))
def test_force_parity_fp32(case):
    """The FP32 form (MG_FORCE_FP32: FP32 links, vectors and arithmetic)
    against the FP64 oracle at the FP32 kernels' tolerance."""
    from paper_1011_2775_gb300 import binding as B
    dims, eps, ape, csw, m0, seed = case
    U = I.make_gauge(dims, eps, ape, 0.5, seed)
    W = WilsonClover(U, csw, m0)
    lam = I.gaussian_source(dims, seed + 1)
    psi = I.gaussian_source(dims, seed + 2)
    K = OF.link_derivative(W, lam.reshape(W.shape + (12,)), psi.reshape(W.shape + (12,)))
    with _solver(dims, U, csw, m0) as S:
        got_w = S.force(lam, psi, kind=B.MG_FORCE_WIRTINGER | B.MG_FORCE_FP32)
        got_f = S.force(lam, psi, kind=B.MG_FORCE_SU3 | B.MG_FORCE_FP32)
        f64 = S.force(lam, psi, kind=B.MG_FORCE_SU3)
    assert rel(got_w, dag(K)) <= TOL32
    assert rel(got_f, OF.su3_force(U, K)) <= TOL32
    assert rel(got_f, f64) > 0   # a separate FP32 computation, not the FP64 one


def test_force_device_buffers_match_host():
    torch = pytest.importorskip("torch")
    dims, eps, ape, csw, m0, seed = CASES[1]
    U = I.make_gauge(dims, eps, ape, 0.5, seed)
    lam = I.gaussian_source(dims, 7)
    psi = I.gaussian_source(dims, 8)
    with _solver(dims, U, csw, m0) as S:
        host = S.force(lam, psi)
        dev = S.force(torch.from_numpy(lam).cuda(), torch.from_numpy(psi).cuda())
    assert np.array_equal(host, dev.cpu().numpy())


@pytest.mark.parametrize("mode", [0, 1], ids=["mg", "eo_gcr"])
def test_solve_dagger_residual(mode):
    dims = (8, 8, 8, 8)
    U = I.make_gauge(dims, 0.3, 1, 0.5, 5201)
    W = WilsonClover(U, 1.0, -0.1)
    chi = I.gaussian_source(dims, 5202)
    with _solver(dims, U, 1.0, -0.1) as S:
        if mode == 0:
            S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[8], seed=5203)
            S.setup()
        lam, info = S.solve_dagger(chi, 1e-10, mode)
    lv = lam.reshape(W.shape + (12,))
    r = chi.reshape(W.shape + (12,)) - W.gamma5(W.D(W.gamma5(lv)))   # D^dag = gamma_5 D gamma_5
    assert np.sqrt(norm2(r) / norm2(chi)) <= 1e-10
    # the source is left untouched by the gamma_5 rotation
    assert np.array_equal(chi, I.gaussian_source(dims, 5202))


def test_autograd_matches_oracle_gradients():
    """L = Re<chi, D^{-1} eta> on 4^4: grad_eta = D^{-dag} chi and grad_U = K^dag
    from dense solves, to the accuracy of solves at tol 1e-12."""
    torch = pytest.importorskip("torch")
    from paper_1011_2775_gb300.autograd import dirac_solve
    dims = (4, 4, 4, 4)
    U = I.make_gauge(dims, 0.4, 1, 0.5, 5301)
    csw, m0 = 1.0, -0.1
    W = WilsonClover(U, csw, m0)
    chi = I.gaussian_source(dims, 5302)
    eta = I.gaussian_source(dims, 5303)
    L0, lam, K, _ = OF.gradients(W, chi.reshape(W.shape + (12,)), eta.reshape(W.shape + (12,)))
    Ut = torch.from_numpy(U).cuda().requires_grad_(True)
    et = torch.from_numpy(eta).cuda().requires_grad_(True)
    ct = torch.from_numpy(chi).cuda()
    with _solver(dims, U, csw, m0) as S:
        S.load_gauge(Ut)
        S.set_clover(csw, m0)
        S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[8], seed=5304)
        S.setup()
        psi = dirac_solve(S, et, Ut, tol=1e-12)
        L = torch.sum(torch.conj(ct) * psi).real
        L.backward()
    assert abs(L.item() - L0) <= 1e-10 * abs(L0)
    assert rel(et.grad.cpu().numpy(), lam.reshape(eta.shape)) <= 1e-9
    assert rel(Ut.grad.cpu().numpy(), dag(K)) <= 1e-9


def test_force_matches_gpu_central_differences():
    """dL/de of L(exp(i e X) U) = 2 sum tr(X F) on 8^4, L from GPU MG solves at
    tol 1e-12 of the perturbed fields (a fresh setup each), F from the
    autograd path's lam and psi."""
    pytest.importorskip("torch")
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 8)
    U = I.make_gauge(dims, 0.3, 1, 0.5, 5401)
    csw, m0 = 1.0, -0.05
    chi = I.gaussian_source(dims, 5402)
    eta = I.gaussian_source(dims, 5403)
    rng = np.random.default_rng(5404)

    def loss(Uf):
        with _solver(dims, Uf, csw, m0) as S:
            S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[8], seed=5405)
            S.setup()
            psi, _ = S.solve(eta, 1e-12)
        return float(np.vdot(chi.ravel(), psi.ravel()).real), psi

    with _solver(dims, U, csw, m0) as S:
        S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[8], seed=5405)
        S.setup()
        psi, _ = S.solve(eta, 1e-12)
        lam, _ = S.solve_dagger(chi, 1e-12)
        F = S.force(lam, psi, kind=B.MG_FORCE_SU3)
    h = 1e-5
    for trial in range(2):
        w = rng.standard_normal(U.shape[:-2] + (8,))
        X = np.einsum("...a,aij->...ij", w, I.gell_mann() / 2.0)
        e, q = np.linalg.eigh(X)
        expm = lambda s: (q * np.exp(1j * s * e)[..., None, :]) @ dag(q)  # noqa: E731
        Lp, _ = loss(np.ascontiguousarray(expm(h) @ U))
        Lm, _ = loss(np.ascontiguousarray(expm(-h) @ U))
        fd = (Lp - Lm) / (2 * h)
        an = 2.0 * float(np.sum(X * np.swapaxes(F, -1, -2)).real)
        assert abs(fd - an) <= 1e-5 * abs(an), (trial, fd, an)
