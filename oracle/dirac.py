"""Wilson-clover Dirac operator and its even-odd forms, FP64, whole-lattice numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows the paper's problem statement ``[D(U) + m] psi = eta`` (Introduction,
Eq. 1) and its red-black preconditioning ("Red-black preconditioning", Eq. 2
and the D_r / b_r equations after it).  The paper never writes D out; this
module takes the following readings, used identically by the CUDA path:

* Operator: ``D psi(x) = A(x) psi(x) + (H psi)(x)`` with the Wilson hopping
  term (r = 1)
  ``H psi(x) = -1/2 sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu)
                           + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)]``
  and the site-local clover matrix
  ``A(x) = (4 + m0) + csw * (i/4) sum_{mu != nu} sigma_{mu nu} F_{mu nu}(x)``.
  The bare mass ``m0`` is the paper's ``m``; "the mass term is absorbed into
  D" is the ``4 + m0`` inside ``A``.
* Gamma matrices: DeGrand-Rossi chiral basis, ``gamma_5 = gamma_1 gamma_2
  gamma_3 gamma_4 = diag(1, 1, -1, -1)``.  Chirality of a spin index is
  ``spin // 2``.  ``A`` is then block diagonal: two 6x6 Hermitian blocks.
* Clover: ``sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu]``; ``Q_{mu nu}(x)`` is
  the sum of the four counter-clockwise plaquette leaves at ``x`` in the
  (mu, nu) plane; ``F_{mu nu} = (Q - Q^dag)/8`` minus its trace/3.  The sum
  over ``mu != nu`` runs over both orders.
* Boundaries: gauge periodic; fermion periodic in x, y, z and antiperiodic in
  t, as a sign on the hop across ``t = Lt-1 -> 0`` (never folded into U).
* Even-odd: site parity ``(x+y+z+t) mod 2``, even = 0.  ``D_ee = A_e``,
  ``D_oo = A_o``, ``D_eo = H_eo``, ``D_oe = H_oe``.  Right-preconditioned
  ``D_p = D diag(A)^{-1} = 1 + H A^{-1}``; reduced
  ``D_r = 1 - H_eo A_o^{-1} H_oe A_e^{-1}`` acting on ``y_e = A_e x_e``;
  ``b_r = b_e - H_eo A_o^{-1} b_o``; ``x_e = A_e^{-1} y_e``;
  ``x_o = A_o^{-1}(b_o - H_oe x_e)``.

Vectors on a level are arrays of shape ``(Lt, Lz, Ly, Lx, ndof)``.  On the
fine level ``ndof = 12`` with ``dof = 3*spin + colour``.  Even-odd vectors are
whole-lattice arrays that are zero on the other parity.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------- gamma basis
def gamma_matrices():
    """``(gamma_1..gamma_4, gamma_5)`` in the DeGrand-Rossi chiral basis."""
    s1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    s2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    s3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    z = np.zeros((2, 2), dtype=np.complex128)
    one = np.eye(2, dtype=np.complex128)

    def off(a, b):
        return np.block([[z, a], [b, z]])

    g = np.stack([off(1j * s1, -1j * s1), off(-1j * s2, 1j * s2), off(1j * s3, -1j * s3), off(one, one)])
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


GAMMA, GAMMA5 = gamma_matrices()


def sigma(mu: int, nu: int) -> np.ndarray:
    """``sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu]``."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])


# ----------------------------------------------------------------------------- lattice helpers
def shape_of(dims):
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def site_parity(dims) -> np.ndarray:
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in shape_of(dims)], indexing="ij")
    return (x + y + z + t) % 2


def shift(f: np.ndarray, mu: int, sign: int, antiperiodic_t: bool = False) -> np.ndarray:
    """``f(x + sign * mu_hat)`` on a periodic lattice; with ``antiperiodic_t`` the
    value that crossed the t boundary picks up a factor -1."""
    g = np.roll(f, -sign, axis=3 - mu)
    if antiperiodic_t and mu == 3:
        g = g.copy()
        if sign > 0:
            g[-1] *= -1.0
        else:
            g[0] *= -1.0
    return g


def dag(m: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(m, -1, -2))


def inner(a: np.ndarray, b: np.ndarray) -> complex:
    """``<a, b> = sum conj(a) b``."""
    return complex(np.vdot(a.ravel(), b.ravel()))


def norm2(a: np.ndarray) -> float:
    return float(np.vdot(a.ravel(), a.ravel()).real)


# ----------------------------------------------------------------------------- generic level
class LatticeLevel:
    """An operator ``D = M + H`` on one lattice: ``M`` site-local, ``H`` a
    nearest-neighbour hop split into 8 directional terms ``d`` (``d < 4``:
    pulls from ``x + mu_hat``, ``mu = d``; ``d >= 4``: from ``x - mu_hat``,
    ``mu = d - 4``).  Subclasses give ``hop_dir``, ``M`` and ``Minv``."""

    ndof: int

    def __init__(self, dims):
        self.dims = tuple(int(d) for d in dims)
        self.shape = shape_of(self.dims)
        par = site_parity(self.dims)
        self.even = (par == 0)[..., None]
        self.odd = (par == 1)[..., None]
        self.eo_ok = all(d % 2 == 0 for d in self.dims)

    # chirality (gamma_5 eigenvalue) of each dof: first half +1, second half -1
    def chirality_sign(self) -> np.ndarray:
        h = self.ndof // 2
        return np.concatenate([np.ones(h), -np.ones(h)])

    def gamma5(self, v):
        return v * self.chirality_sign()

    def zeros(self):
        return np.zeros(self.shape + (self.ndof,), dtype=np.complex128)

    def hop(self, v):
        out = self.hop_dir(v, 0)
        for d in range(1, 8):
            out = out + self.hop_dir(v, d)
        return out

    def D(self, v):
        return self.M(v) + self.hop(v)

    def Dp(self, v):
        """Right-preconditioned full operator ``D diag(M)^{-1} = 1 + H M^{-1}``."""
        return v + self.hop(self.Minv(v))

    def Dr(self, y):
        """``D_r = 1 - H_eo M_o^{-1} H_oe M_e^{-1}`` on an even-supported ``y``."""
        ye = y * self.even
        s = self.Minv(ye)
        t = self.Minv(self.odd * self.hop(s))
        return ye - self.even * self.hop(t)

    def b_r(self, b):
        """``b_r = b_e - H_eo M_o^{-1} b_o``."""
        return self.even * b - self.even * self.hop(self.Minv(self.odd * b))

    def reconstruct(self, y, b):
        """``x_e = M_e^{-1} y_e``, ``x_o = M_o^{-1}(b_o - H_oe x_e)``."""
        xe = self.Minv(self.even * y)
        xo = self.Minv(self.odd * (b - self.hop(xe)))
        return xe + xo

    def as_dense(self, op) -> np.ndarray:
        """Dense matrix of a linear map on this level (small lattices only)."""
        n = int(np.prod(self.shape)) * self.ndof
        cols = []
        for j in range(n):
            e = np.zeros(n, dtype=np.complex128)
            e[j] = 1.0
            cols.append(op(e.reshape(self.shape + (self.ndof,))).ravel())
        return np.stack(cols, axis=1)


# ----------------------------------------------------------------------------- clover
def plaquette_leaves(U: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """``Q_{mu nu}(x)``: sum of the four counter-clockwise leaves in the (mu, nu)
    plane that touch ``x`` (periodic gauge field)."""
    um, un = U[..., mu, :, :], U[..., nu, :, :]
    sh = lambda f, m, s: shift(f, m, s)  # noqa: E731  periodic
    # leaf 1: x -> x+mu -> x+mu+nu -> x+nu -> x
    q = um @ sh(un, mu, +1) @ dag(sh(um, nu, +1)) @ dag(un)
    # leaf 2: x -> x+nu -> x+nu-mu -> x-mu -> x
    q = q + un @ dag(sh(sh(um, mu, -1), nu, +1)) @ dag(sh(un, mu, -1)) @ sh(um, mu, -1)
    # leaf 3: x -> x-mu -> x-mu-nu -> x-nu -> x
    q = q + dag(sh(um, mu, -1)) @ dag(sh(sh(un, mu, -1), nu, -1)) @ sh(sh(um, mu, -1), nu, -1) @ sh(un, nu, -1)
    # leaf 4: x -> x-nu -> x-nu+mu -> x+mu -> x
    q = q + dag(sh(un, nu, -1)) @ sh(um, nu, -1) @ sh(sh(un, nu, -1), mu, +1) @ dag(um)
    return q


def field_strength(U: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """``F_{mu nu} = (Q - Q^dag)/8`` made traceless (anti-Hermitian)."""
    q = plaquette_leaves(U, mu, nu)
    f = (q - dag(q)) / 8.0
    tr = np.trace(f, axis1=-2, axis2=-1) / 3.0
    return f - tr[..., None, None] * np.eye(3)


def plane_csw(mu: int, nu: int, csw: float, csw_t: float) -> float:
    """Clover coefficient of the (mu, nu) plane: ``csw_t`` when it contains t
    (direction 3), ``csw`` for the spatial planes."""
    return csw_t if 3 in (mu, nu) else csw


def clover_matrix(U: np.ndarray, csw: float, m0: float, weights=(1.0, 1.0, 1.0, 1.0), csw_t=None) -> np.ndarray:
    """``A(x)`` as a 12x12 matrix per site, index ``3*spin + colour``.

    Isotropic: ``A = (4 + m0) + csw (i/4) sum_{mu != nu} sigma_{mu nu} F_{mu nu}``.
    Anisotropic reading (the paper's lattices are anisotropic but it writes no
    operator down): the mass term becomes ``sum_mu w_mu + m0`` with the hopping
    weights ``w_mu`` of the directions, and the planes containing t take
    ``csw_t`` instead of ``csw``; both reduce to the isotropic form at
    ``w = 1``, ``csw_t = csw``."""
    csw_t = csw if csw_t is None else csw_t
    shp = U.shape[:4]
    A = np.zeros(shp + (4, 3, 4, 3), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            F = field_strength(U, mu, nu)
            A += (plane_csw(mu, nu, csw, csw_t) * 0.25j) * np.einsum("st,...ab->...satb", sigma(mu, nu), F)
    A = A.reshape(shp + (12, 12))
    A += (sum(weights) + m0) * np.eye(12)
    return A


# ----------------------------------------------------------------------------- fine level
class WilsonClover(LatticeLevel):
    """The fine Wilson-clover operator for gauge field ``U`` (library layout
    ``(Lt, Lz, Ly, Lx, 4, 3, 3)``), clover coefficient ``csw`` and bare mass ``m0``.

    ``weights`` (hopping weight per direction x, y, z, t) and ``csw_t`` (clover
    coefficient of the planes containing t) give the anisotropic reading of
    ``clover_matrix``: every hop in direction mu carries ``w_mu``; the defaults
    are the isotropic operator."""

    ndof = 12

    def __init__(self, U: np.ndarray, csw: float, m0: float, antiperiodic_t: bool = True, weights=None,
                 csw_t=None):
        lt, lz, ly, lx = U.shape[:4]
        super().__init__((lx, ly, lz, lt))
        self.U = U
        self.csw = float(csw)
        self.csw_t = float(csw) if csw_t is None else float(csw_t)
        self.w = (1.0, 1.0, 1.0, 1.0) if weights is None else tuple(float(v) for v in weights)
        self.m0 = float(m0)
        self.apbc = antiperiodic_t
        self.A = clover_matrix(U, csw, m0, self.w, self.csw_t)
        self.Ainv = np.linalg.inv(self.A)
        one = np.eye(4, dtype=np.complex128)
        self.proj_minus = [one - GAMMA[mu] for mu in range(4)]
        self.proj_plus = [one + GAMMA[mu] for mu in range(4)]
        self.Ub = [shift(U[..., mu, :, :], mu, -1) for mu in range(4)]  # U_mu(x - mu)

    def hop_dir(self, v, d):
        psi = v.reshape(self.shape + (4, 3))
        mu = d % 4
        if d < 4:
            nb = shift(psi, mu, +1, self.apbc)
            c = np.einsum("...ab,...sb->...sa", self.U[..., mu, :, :], nb)
            out = (-0.5 * self.w[mu]) * np.einsum("st,...ta->...sa", self.proj_minus[mu], c)
        else:
            nb = shift(psi, mu, -1, self.apbc)
            c = np.einsum("...ba,...sb->...sa", np.conj(self.Ub[mu]), nb)
            out = (-0.5 * self.w[mu]) * np.einsum("st,...ta->...sa", self.proj_plus[mu], c)
        return out.reshape(self.shape + (12,))

    def M(self, v):
        return np.einsum("...ij,...j->...i", self.A, v)

    def Minv(self, v):
        return np.einsum("...ij,...j->...i", self.Ainv, v)


def spinor_to_level(psi: np.ndarray) -> np.ndarray:
    """``(..., 4, 3)`` library spinor -> ``(..., 12)`` level vector (same memory order)."""
    return psi.reshape(psi.shape[:-2] + (12,))


def level_to_spinor(v: np.ndarray) -> np.ndarray:
    return v.reshape(v.shape[:-1] + (4, 3))
