"""Pins of the oracle's gradient of Re<chi, D^{-1} eta> (oracle/force.py).

Each check compares the oracle with something other than its own formula:
- the leaf factor lists multiply out to the clover leaves of oracle/dirac.py;
- the link derivative K against exact single-link differences of
  -Re<lam, D(U) psi> (D is real-affine in any one link when every extent is at
  least 2, so the difference is exact for any step);
- the su(3) force against central differences of L along exp(i eps X) on all
  links, with L computed by dense LU solves;
- gauge covariance of the force, and linearity of L in eta.
"""
import numpy as np
import pytest

from oracle import force as F
from oracle.dirac import WilsonClover, dag, plaquette_leaves
from paper_1011_2775_gb300 import inputs as I


def _lv(dims, seed):
    return I.gaussian_source(dims, seed).reshape(I.lattice_shape(dims) + (12,))


def _random_algebra(shape, rng):
    """Random traceless Hermitian X = sum_a w^a T_a per entry of ``shape``."""
    w = rng.standard_normal(shape + (8,))
    return np.einsum("...a,aij->...ij", w, I.gell_mann() / 2.0)


def _expm_i(X):
    e, q = np.linalg.eigh(X)
    return (q * np.exp(1j * e)[..., None, :]) @ dag(q)


@pytest.mark.parametrize("mu,nu", [(0, 1), (1, 0), (0, 3), (2, 3), (3, 1)])
def test_leaf_factors_match_plaquette_leaves(mu, nu):
    dims = (4, 2, 4, 6)
    U = I.make_gauge(dims, 0.7, 0, 0.5, 31)
    got = sum(F.leaf_value(U, f) for f in F.leaf_factors(mu, nu))
    assert np.abs(got - plaquette_leaves(U, mu, nu)).max() < 1e-13


ANISO = dict(weights=(0.45, 0.7, 1.25, 2.0), csw_t=0.6)


@pytest.mark.parametrize("aniso", [False, True], ids=["iso", "aniso"])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 2, 6)])
def test_link_derivative_exact_single_link(dims, aniso):
    """-Re<lam, (D(U + dU) - D(U)) psi> = Re tr(dU K) for a change of one link,
    for arbitrary complex dU (not only su(3) directions), every term of D; also
    for the anisotropic reading (weighted hops, csw_t on the planes with t)."""
    U = I.make_gauge(dims, 0.6, 1, 0.5, 41)
    csw, m0 = 1.3, -0.15
    kw = ANISO if aniso else {}
    W = WilsonClover(U, csw, m0, **kw)
    lam, psi = _lv(dims, 42), _lv(dims, 43)
    K = F.link_derivative(W, lam, psi)
    base = W.D(psi)
    rng = np.random.default_rng(44)
    shp = I.lattice_shape(dims)
    worst = 0.0
    for _ in range(6):
        site = tuple(int(rng.integers(0, n)) for n in shp)
        mu = int(rng.integers(0, 4))
        dU = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        U2 = U.copy()
        U2[site + (mu,)] += dU
        W2 = WilsonClover(U2, csw, m0, **kw)
        lhs = -np.vdot(lam.ravel(), (W2.D(psi) - base).ravel()).real
        rhs = np.trace(dU @ K[site + (mu,)]).real
        worst = max(worst, abs(lhs - rhs) / max(abs(lhs), 1e-300))
    assert worst < 1e-10


def test_link_derivative_free_of_clover_at_csw_zero():
    """With csw = 0 only the hop contributes: K is bilinear in the neighbours and
    vanishes on links whose two ends carry no lam / psi."""
    dims = (4, 4, 2, 4)
    U = I.make_gauge(dims, 0.5, 0, 0.5, 51)
    W = WilsonClover(U, 0.0, 0.2)
    shp = I.lattice_shape(dims)
    lam = np.zeros(shp + (12,), dtype=complex)
    psi = np.zeros(shp + (12,), dtype=complex)
    lam[0, 0, 0, 0] = 1.0 + 0.5j      # site x = 0
    psi[0, 0, 0, 1] = 0.3 - 1.0j      # site x + x_hat
    K = F.link_derivative(W, lam, psi)
    nz = np.argwhere(np.abs(K).reshape(shp + (4, 9)).sum(-1) > 0)
    # only the forward x-link of site 0 pulls psi(x + x_hat) into lam(x)
    assert [tuple(r) for r in nz] == [(0, 0, 0, 0, 0)]


def _loss(U, csw, m0, chi, eta):
    W = WilsonClover(U, csw, m0)
    psi = F.solve_dense(W, eta)
    return float(np.vdot(chi.ravel(), psi.ravel()).real)


def test_force_matches_central_differences():
    """dL/de of L(exp(i e X) U) at e = 0 equals 2 sum tr(X F) (tr T_a T_b = d_ab / 2),
    along random directions X on all links and on single links."""
    dims = (2, 4, 2, 4)
    U = I.make_gauge(dims, 0.5, 1, 0.5, 61)
    csw, m0 = 1.0, -0.1
    chi, eta = _lv(dims, 62), _lv(dims, 63)
    W = WilsonClover(U, csw, m0)
    L0, lam, K, Fm = F.gradients(W, chi, eta)
    rng = np.random.default_rng(64)
    h = 1e-5
    shp = I.lattice_shape(dims)
    for trial in range(4):
        X = _random_algebra(U.shape[:-2], rng)
        if trial >= 2:          # a single link
            mask = np.zeros(U.shape[:-2] + (1, 1))
            site = tuple(int(rng.integers(0, n)) for n in shp) + (int(rng.integers(0, 4)),)
            mask[site] = 1.0
            X = X * mask
        Lp = _loss(_expm_i(h * X) @ U, csw, m0, chi, eta)
        Lm = _loss(_expm_i(-h * X) @ U, csw, m0, chi, eta)
        fd = (Lp - Lm) / (2 * h)
        an = 2.0 * float(np.sum(X * np.swapaxes(Fm, -1, -2)).real)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * np.abs(Fm).max()), (trial, fd, an)


def test_force_is_traceless_hermitian_and_gauge_covariant():
    """Under U_mu(x) -> G(x) U_mu(x) G(x+mu)^dag, psi -> G psi, lam -> G lam the
    force transforms as F_mu(x) -> G(x) F_mu(x) G(x)^dag."""
    dims = (4, 2, 4, 4)
    U = I.make_gauge(dims, 0.6, 0, 0.5, 71)
    csw, m0 = 1.2, 0.05
    lam, psi = _lv(dims, 72), _lv(dims, 73)
    W = WilsonClover(U, csw, m0)
    Fm = F.su3_force(U, F.link_derivative(W, lam, psi))
    assert np.abs(Fm - dag(Fm)).max() < 1e-13
    assert np.abs(np.trace(Fm, axis1=-2, axis2=-1)).max() < 1e-13
    G = I.random_gauge_transform(dims, 74)
    UG = np.empty_like(U)
    for mu in range(4):
        Gp = np.roll(G, -1, axis=3 - mu)
        UG[..., mu, :, :] = G @ U[..., mu, :, :] @ dag(Gp)
    rot = lambda v: np.einsum("...ab,...sb->...sa", G, v.reshape(v.shape[:-1] + (4, 3))).reshape(v.shape)  # noqa: E731
    WG = WilsonClover(UG, csw, m0)
    FG = F.su3_force(UG, F.link_derivative(WG, rot(lam), rot(psi)))
    expect = G[..., None, :, :] @ Fm @ dag(G)[..., None, :, :]
    assert np.abs(FG - expect).max() < 1e-12 * np.abs(Fm).max()


def test_source_gradient_is_adjoint_solution():
    """L is linear in eta: L(eta + d) - L(eta) = Re<lam, d> with lam = D^{-dag} chi."""
    dims = (2, 2, 4, 4)
    U = I.make_gauge(dims, 0.5, 0, 0.5, 81)
    W = WilsonClover(U, 1.0, -0.1)
    chi, eta, d = _lv(dims, 82), _lv(dims, 83), _lv(dims, 84)
    L0, lam, _, _ = F.gradients(W, chi, eta)
    L1 = float(np.vdot(chi.ravel(), F.solve_dense(W, eta + d).ravel()).real)
    assert abs((L1 - L0) - np.vdot(lam.ravel(), d.ravel()).real) < 1e-10 * abs(L1 - L0)
    # gamma_5-hermiticity: D^{-dag} chi = gamma_5 D^{-1} gamma_5 chi
    assert np.abs(lam - W.gamma5(F.solve_dense(W, W.gamma5(chi)))).max() < 1e-10 * np.abs(lam).max()
