"""Gradient of ``L = Re <chi, D^{-1} eta>`` with respect to the source and the
gauge links, FP64, whole-lattice numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper solves ``[D(U) + m] psi = eta`` (Introduction, Eq. 1) and has no
gradient; differentiating the solve is a stated extension.  The readings:

* ``psi = D^{-1} eta`` and ``lambda = D^{-dag} chi`` (the adjoint solve; with
  ``D^dag = gamma_5 D gamma_5`` it is ``gamma_5 D^{-1} gamma_5 chi``).  For fixed
  ``chi``, ``dL = Re <chi, d(D^{-1}) eta> = -Re <lambda, dD psi>`` and
  ``dL = Re <lambda, d eta>``.
* Gradients of a real function of a complex array follow the torch
  convention ``dL/dRe z + i dL/dIm z``: the source gradient is ``lambda``.
* Link derivative.  For fixed ``lambda`` and ``psi`` the functional
  ``f(U) = -Re <lambda, D(U) psi>`` changes, under any complex variation
  ``dU`` of the links, by ``df = Re sum_{x,mu} tr(dU_mu(x) K_mu(x))``.  ``K`` is
  returned by :func:`link_derivative`; the unconstrained (Wirtinger) gradient
  in torch's convention is ``K^dag``.
* su(3) force.  ``U_mu(x) -> exp(i omega^a T_a) U_mu(x)`` with
  ``T_a = lambda_a / 2`` (Gell-Mann), ``F^a = df / d omega^a``, returned as the
  traceless Hermitian ``sum_a F^a T_a``.  With ``G = i U K``,
  ``F^a = Re tr(T_a G)`` and, by the su(3) completeness relation
  ``sum_a (T_a)_ij (T_a)_kl = (d_il d_jk - d_ij d_kl / 3) / 2``,
  ``sum_a F^a T_a = (H - tr(H)/3) / 2`` with ``H = (G + G^dag) / 2``.

The clover term is differentiated by reverse accumulation through the leaf
products of ``dirac.plaquette_leaves``, each leaf written here as a list of
(link direction, displacement, adjoint) factors; a test checks that these
lists multiply out to ``plaquette_leaves``.  Nothing here is pinned against
itself: the tests compare ``K`` with exact single-link differences of
``-Re <lambda, D(U) psi>`` (the operator is real-affine in any one link when
every extent is at least 2) and the force with central differences of ``L``.
"""
from __future__ import annotations

import numpy as np

from .dirac import GAMMA, WilsonClover, dag, plane_csw, shift, sigma


def _at(f: np.ndarray, disp) -> np.ndarray:
    """``f(x + disp)`` for a periodic field, ``disp`` a 4-vector (x, y, z, t)."""
    g = f
    for mu in range(4):
        for _ in range(abs(disp[mu])):
            g = shift(g, mu, 1 if disp[mu] > 0 else -1)
    return g


def _unit(mu: int, s: int = 1):
    d = [0, 0, 0, 0]
    d[mu] = s
    return d


def _add(*ds):
    return [sum(c) for c in zip(*ds)]


def leaf_factors(mu: int, nu: int):
    """The four leaves of ``Q_{mu nu}(x)`` as lists of ``(direction, displacement,
    adjoint)``: each factor is ``U_direction(x + displacement)``, or its adjoint,
    and a leaf is the ordered product of its factors."""
    m, n = _unit(mu), _unit(nu)
    mm, nm = _unit(mu, -1), _unit(nu, -1)
    o = [0, 0, 0, 0]
    return [
        # x -> x+mu -> x+mu+nu -> x+nu -> x
        [(mu, o, False), (nu, m, False), (mu, n, True), (nu, o, True)],
        # x -> x+nu -> x+nu-mu -> x-mu -> x
        [(nu, o, False), (mu, _add(mm, n), True), (nu, mm, True), (mu, mm, False)],
        # x -> x-mu -> x-mu-nu -> x-nu -> x
        [(mu, mm, True), (nu, _add(mm, nm), True), (mu, _add(mm, nm), False), (nu, nm, False)],
        # x -> x-nu -> x-nu+mu -> x+mu -> x
        [(nu, nm, True), (mu, nm, False), (nu, _add(nm, m), False), (mu, o, True)],
    ]


def leaf_value(U: np.ndarray, factors) -> np.ndarray:
    """Product of a leaf's factors at every site."""
    out = None
    for d, disp, adj in factors:
        f = _at(U[..., d, :, :], disp)
        f = dag(f) if adj else f
        out = f if out is None else out @ f
    return out


def link_derivative(W: WilsonClover, lam: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """``K_mu(x)`` with ``d(-Re<lam, D(U) psi>) = Re sum tr(dU_mu(x) K_mu(x))``.

    ``lam`` and ``psi`` are level vectors ``(Lt, Lz, Ly, Lx, 12)``.  Returns an
    array shaped like the gauge field, ``(Lt, Lz, Ly, Lx, 4, 3, 3)``.
    """
    U = W.U
    shp = W.shape
    lam4 = lam.reshape(shp + (4, 3))
    psi4 = psi.reshape(shp + (4, 3))
    K = np.zeros(U.shape, dtype=np.complex128)
    one = np.eye(4, dtype=np.complex128)

    # Hopping term, forward part at site x:  -1/2 (1 - gamma_mu) U_mu(x) psi(x+mu)
    #   -Re lam(x)^dag [-1/2 (1-g) dU psi(x+mu)] = 1/2 Re tr(dU M),
    #   M_ba = sum_st psi(x+mu)_{t b} (1-g)_{st} conj(lam(x)_{s a})
    # backward part at site y = x+mu:  -1/2 (1 + gamma_mu) U_mu(x)^dag psi(x)
    #   contributes 1/2 Re tr(dU_mu(x) N(x+mu)),
    #   N(y)_ab = sum_st lam(y)_{s a} conj((1+g)_{st}) conj(psi(y-mu)_{t b})
    for mu in range(4):
        nb = shift(psi4, mu, +1, W.apbc)                       # psi(x+mu) with the boundary sign
        M = np.einsum("...tb,st,...sa->...ba", nb, one - GAMMA[mu], np.conj(lam4))
        nbm = shift(psi4, mu, -1, W.apbc)                      # psi(y-mu) with the boundary sign
        N = np.einsum("...sa,st,...tb->...ab", lam4, np.conj(one + GAMMA[mu]), np.conj(nbm))
        K[..., mu, :, :] += (0.5 * W.w[mu]) * M + (0.5 * W.w[mu]) * shift(N, mu, +1)   # the direction's weight

    # Clover term: -Re lam^dag dA psi with dA = csw (i/4) sum_{mu != nu} sigma_{mu nu} x dF_{mu nu}.
    #   lam^dag (sigma x dF) psi = tr(dF S),  S_ba = sum_st sigma_st psi_{t b} conj(lam_{s a}),
    #   so df = Re tr(dF C) with C = -(i csw / 4) S.  F = (Q - Q^dag)/8 minus trace/3, hence
    #   Re tr(dF C) = Re tr(dQ Wm) with C0 = C - tr(C)/3 and Wm = (C0 - C0^dag)/8.
    #   For a leaf L_1 L_2 L_3 L_4: tr(d(L_1..L_4) Wm) = sum_k tr(dL_k R_k),
    #   R_k = L_{k+1} .. L_4 Wm L_1 .. L_{k-1}; a factor U(x+s) adds R_k(z-s) to K(z),
    #   an adjoint factor adds R_k(z-s)^dag (Re tr(dU^dag R) = Re tr(dU R^dag)).
    eye3 = np.eye(3)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            S = np.einsum("st,...tb,...sa->...ba", sigma(mu, nu), psi4, np.conj(lam4))
            C = -(0.25j * plane_csw(mu, nu, W.csw, W.csw_t)) * S
            C0 = C - (np.trace(C, axis1=-2, axis2=-1) / 3.0)[..., None, None] * eye3
            Wm = (C0 - dag(C0)) / 8.0
            for factors in leaf_factors(mu, nu):
                mats = []
                for d, disp, adj in factors:
                    f = _at(U[..., d, :, :], disp)
                    mats.append(dag(f) if adj else f)
                for k, (d, disp, adj) in enumerate(factors):
                    R = None
                    for j in range(k + 1, 4):
                        R = mats[j] if R is None else R @ mats[j]
                    R = Wm if R is None else R @ Wm
                    for j in range(0, k):
                        R = R @ mats[j]
                    back = [-c for c in disp]
                    contrib = _at(dag(R) if adj else R, back)
                    K[..., d, :, :] += contrib
    return K


def su3_force(U: np.ndarray, K: np.ndarray) -> np.ndarray:
    """``sum_a F^a T_a`` from ``K`` (see the module header)."""
    G = 1j * (U @ K)
    H = 0.5 * (G + dag(G))
    tr = np.trace(H, axis1=-2, axis2=-1)
    return 0.5 * (H - (tr / 3.0)[..., None, None] * np.eye(3))


def solve_dense(W: WilsonClover, b: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """``D^{-1} b`` (or ``D^{-dag} b``) by a dense LU solve (small lattices only)."""
    Dm = W.as_dense(W.D)
    if adjoint:
        Dm = Dm.conj().T
    return np.linalg.solve(Dm, b.ravel()).reshape(b.shape)


def gradients(W: WilsonClover, chi: np.ndarray, eta: np.ndarray, Dm: np.ndarray | None = None):
    """``(L, grad_eta, K, F)`` for ``L = Re <chi, D^{-1} eta>`` by dense solves.

    ``grad_eta = lambda``; ``K`` as in :func:`link_derivative` (the torch
    gradient of the complex links is ``K^dag``); ``F`` the su(3) force.
    """
    if Dm is None:
        Dm = W.as_dense(W.D)
    psi = np.linalg.solve(Dm, eta.ravel()).reshape(eta.shape)
    lam = np.linalg.solve(Dm.conj().T, chi.ravel()).reshape(chi.shape)
    L = float(np.vdot(chi.ravel(), psi.ravel()).real)
    K = link_derivative(W, lam, psi)
    return L, lam, K, su3_force(W.U, K)
