"""Pins of the oracle's Dirac operator against what the physics fixes.

Each test checks the oracle against something other than itself: a closed
form (free field in momentum space, constant abelian field strength), an
invariance (gamma_5-hermiticity, gauge covariance), or a library routine on a
dense assembly (LU solve, eigendecomposition).
"""
import numpy as np
import pytest

from oracle.dirac import WilsonClover, inner, norm2
from paper_1011_2775_gb300 import inputs as I

# Independently typed DeGrand-Rossi table (rows of gamma_1..gamma_4).
G1 = np.array([[0, 0, 0, 1j], [0, 0, 1j, 0], [0, -1j, 0, 0], [-1j, 0, 0, 0]])
G2 = np.array([[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]], dtype=complex)
G3 = np.array([[0, 0, 1j, 0], [0, 0, 0, -1j], [-1j, 0, 0, 0], [0, 1j, 0, 0]])
G4 = np.array([[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]], dtype=complex)
GT = [G1, G2, G3, G4]


def _vec(dims, seed):
    return I.gaussian_source(dims, seed).reshape(I.lattice_shape(dims) + (12,))


def test_gamma_algebra_and_basis():
    from oracle.dirac import GAMMA, GAMMA5
    for mu in range(4):
        assert np.allclose(GAMMA[mu], GT[mu])
        assert np.allclose(GAMMA[mu], GAMMA[mu].conj().T)
        for nu in range(4):
            ac = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
            assert np.allclose(ac, 2 * np.eye(4) * (mu == nu))
    assert np.allclose(GAMMA5, np.diag([1, 1, -1, -1]))


@pytest.mark.parametrize("m0,csw", [(0.1, 0.0), (-0.2, 1.0)])
def test_free_field_plane_wave(m0, csw):
    """P1: at U = 1, D e^{ipx} u = [m0 + sum(1-cos p) + i sum gamma sin p] e^{ipx} u,
    with antiperiodic t momenta 2 pi (n + 1/2) / Lt."""
    dims = (4, 6, 2, 8)
    lx, ly, lz, lt = dims
    W = WilsonClover(I.unit_gauge(dims), csw, m0)
    rng = np.random.default_rng(0)
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in (lt, lz, ly, lx)], indexing="ij")
    for n in [(0, 0, 0, 0), (1, 2, 1, 3), (3, 5, 1, 6)]:
        p = [2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz, 2 * np.pi * (n[3] + 0.5) / lt]
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        psi = phase[..., None, None] * u
        Dk = (m0 + sum(1 - np.cos(q) for q in p)) * np.eye(4) + 1j * sum(GT[m] * np.sin(p[m]) for m in range(4))
        expect = phase[..., None, None] * (Dk @ u)
        got = W.D(psi.reshape(W.shape + (12,))).reshape(expect.shape)
        assert np.abs(got - expect).max() < 1e-13


def _free_solution(dims, m0, eta):
    lx, ly, lz, lt = dims
    shp = I.lattice_shape(dims)
    t = np.arange(lt)[:, None, None, None, None, None]
    twist = np.exp(-1j * np.pi * t / lt)
    et = np.fft.fftn(eta * twist, axes=(0, 1, 2, 3))
    pt, pz, py, px = np.meshgrid(2 * np.pi * np.fft.fftfreq(lt) + np.pi / lt, 2 * np.pi * np.fft.fftfreq(lz),
                                 2 * np.pi * np.fft.fftfreq(ly), 2 * np.pi * np.fft.fftfreq(lx), indexing="ij")
    p = [px, py, pz, pt]
    M = m0 + sum(1 - np.cos(q) for q in p)
    s2 = sum(np.sin(q) ** 2 for q in p)
    num = M[..., None, None] * np.eye(4) - 1j * sum(np.sin(p[m])[..., None, None] * GT[m] for m in range(4))
    Dinv = num / (M ** 2 + s2)[..., None, None]
    st = np.einsum("...st,...tc->...sc", Dinv, et)
    return np.fft.ifftn(st, axes=(0, 1, 2, 3)) / twist


def test_free_field_eo_solve_matches_fft():
    """P2: the even-odd GCR solve of the free operator equals the momentum-space inverse."""
    from oracle.multigrid import eo_solve
    dims = (4, 4, 4, 8)
    m0 = 0.1
    W = WilsonClover(I.unit_gauge(dims), 1.0, m0)
    eta = I.gaussian_source(dims, 7)
    x, info = eo_solve(W, eta.reshape(W.shape + (12,)), tol=1e-12)
    assert info.converged
    ref = _free_solution(dims, m0, eta)
    assert np.abs(x.reshape(ref.shape) - ref).max() / np.abs(ref).max() < 1e-10


def test_gamma5_hermiticity():
    """P3: <phi, D psi> = <g5 D g5 phi, psi> for a random smeared field with clover."""
    dims = (4, 4, 4, 4)
    W = WilsonClover(I.make_gauge(dims, 0.3, 1, 0.5, 11), 1.3, -0.2)
    phi, psi = _vec(dims, 1), _vec(dims, 2)
    lhs = inner(phi, W.D(psi))
    rhs = inner(W.gamma5(W.D(W.gamma5(phi))), psi)
    assert abs(lhs - rhs) / abs(lhs) < 1e-14
    # and the hopping term alone is not Hermitian (the test can fail)
    assert abs(inner(phi, W.D(psi)) - inner(W.D(phi), psi)) / abs(lhs) > 1e-3


def test_gauge_covariance():
    """P4: D[U^G](G psi) = G D[U] psi, U^G_mu(x) = G(x) U_mu(x) G(x+mu)^dag, clover included."""
    dims = (4, 4, 2, 6)
    U = I.make_gauge(dims, 0.5, 0, 0.5, 21)
    G = I.random_gauge_transform(dims, 22)
    UG = np.empty_like(U)
    for mu in range(4):
        Gp = np.roll(G, -1, axis=3 - mu)
        UG[..., mu, :, :] = G @ U[..., mu, :, :] @ np.conj(np.swapaxes(Gp, -1, -2))
    W, WG = WilsonClover(U, 1.0, -0.3), WilsonClover(UG, 1.0, -0.3)
    psi = I.gaussian_source(dims, 23)
    Gpsi = np.einsum("...ab,...sb->...sa", G, psi)
    lhs = WG.D(Gpsi.reshape(W.shape + (12,))).reshape(psi.shape)
    rhs = np.einsum("...ab,...sb->...sa", G, W.D(psi.reshape(W.shape + (12,))).reshape(psi.shape))
    assert np.abs(lhs - rhs).max() < 1e-13
    # the link transform matters: the untransformed operator on G psi differs
    assert np.abs(W.D(Gpsi.reshape(W.shape + (12,))).reshape(psi.shape) - rhs).max() > 1e-2


def test_clover_hermitian_chiral_blocks_and_unit_gauge():
    """P5: A = A^dag, block diagonal in chirality, A = 4 + m0 at U = 1."""
    dims = (4, 4, 4, 4)
    W = WilsonClover(I.make_gauge(dims, 0.4, 0, 0.5, 31), 1.0, -0.35)
    A = W.A
    assert np.abs(A - np.conj(np.swapaxes(A, -1, -2))).max() < 1e-15
    assert np.abs(A[..., :6, 6:]).max() == 0 and np.abs(A[..., 6:, :6]).max() == 0
    assert np.abs(A - (4 - 0.35) * np.eye(12)).max() > 1e-3
    W1 = WilsonClover(I.unit_gauge(dims), 1.7, -0.35)
    assert np.abs(W1.A - (4 - 0.35) * np.eye(12)).max() < 1e-15


@pytest.mark.parametrize("plane", [(0, 1), (2, 3)])
def test_clover_constant_abelian_field(plane):
    """Constant U(1) flux B in one plane (embedded as diag(e^{i th}, e^{-i th}, 1)):
    every leaf is e^{iB}, so A = (4+m0) - (csw/2) sin(B) sigma_{mu nu} x diag(1, -1, 0)
    exactly, with eigenvalues 4+m0 and 4+m0 -+ (csw/2) sin B, four of each."""
    mu, nu = plane
    dims = (4, 4, 4, 4)
    m0, csw = -0.1, 1.3
    B = 2 * np.pi / dims[mu]
    U = I.unit_gauge(dims)
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in I.lattice_shape(dims)], indexing="ij")
    th = B * (x, y, z, t)[mu]
    U[..., nu, 0, 0] = np.exp(1j * th)
    U[..., nu, 1, 1] = np.exp(-1j * th)
    W = WilsonClover(U, csw, m0)
    sig = 0.5j * (GT[mu] @ GT[nu] - GT[nu] @ GT[mu])
    expect = (4 + m0) * np.eye(12) - 0.5 * csw * np.sin(B) * np.kron(sig, np.diag([1.0, -1.0, 0.0]))
    assert np.abs(W.A - expect).max() < 1e-14
    ev = np.sort(np.linalg.eigvalsh(W.A[0, 0, 0, 0]))
    h = 0.5 * csw * np.sin(B)
    assert np.allclose(ev, np.sort([4 + m0 - h] * 4 + [4 + m0] * 4 + [4 + m0 + h] * 4), atol=1e-14)


@pytest.fixture(scope="module")
def dense44():
    dims = (4, 4, 4, 4)
    W = WilsonClover(I.make_gauge(dims, 0.3, 0, 0.5, 1001), 1.0, -0.1)
    return W, W.as_dense(W.D)


def test_eo_reduced_solve_matches_dense_lu(dense44):
    """P6: reduced solve + reconstruction equals a dense LU solve of D (4^4, 3072 dof)."""
    W, Dd = dense44
    b = _vec(W.dims, 1002)
    x_ref = np.linalg.solve(Dd, b.ravel()).reshape(b.shape)
    # D_r y_e = b_r holds for y_e = A_e x_e of the exact solution
    y = W.M(x_ref * W.even)
    assert np.sqrt(norm2(W.Dr(y) - W.b_r(b)) / norm2(b)) < 1e-13
    assert np.abs(W.reconstruct(y, b) - x_ref).max() / np.abs(x_ref).max() < 1e-13
    from oracle.multigrid import eo_solve
    x, info = eo_solve(W, b, tol=1e-12)
    assert info.converged
    assert np.abs(x - x_ref).max() / np.abs(x_ref).max() < 1e-9


def test_dp_is_d_times_inverse_clover(dense44):
    """D_p = D diag(A)^{-1}: dense D times the dense site-inverse."""
    W, Dd = dense44
    v = _vec(W.dims, 5)
    ref = (Dd @ W.Minv(v).ravel()).reshape(v.shape)
    assert np.abs(W.Dp(v) - ref).max() < 1e-12


def test_dp_dr_share_even_eigenvectors():
    """The paper's remark that D_p and D_r share eigenvectors on even sites:
    D_p u = lam u implies D_r u_e = (1 - (lam - 1)^2) u_e."""
    dims = (2, 2, 2, 4)
    W = WilsonClover(I.make_gauge(dims, 0.5, 0, 0.5, 41), 1.0, -0.2)
    Dp = W.as_dense(W.Dp)
    lam, vecs = np.linalg.eig(Dp)
    for j in np.argsort(np.abs(lam))[:6]:
        u = vecs[:, j].reshape(W.shape + (12,))
        ue = u * W.even
        mu = 1 - (lam[j] - 1) ** 2
        assert np.sqrt(norm2(W.Dr(ue) - mu * ue) / norm2(ue)) < 1e-10


def test_dr_adjoint_through_gamma5_and_clover():
    """The operator CGNR needs: D_r^dag = gamma_5 A_e^{-1} D_r A_e gamma_5
    (the Schur complement is gamma_5-hermitian, the clover blocks Hermitian and
    commuting with gamma_5), checked against the dense conjugate transpose of
    D_r restricted to the even sites."""
    dims = (2, 2, 2, 4)
    W = WilsonClover(I.make_gauge(dims, 0.6, 0, 0.5, 43), 1.3, -0.25)
    ev = np.broadcast_to(W.even, W.shape + (12,)).astype(bool).ravel()
    Dr = W.as_dense(lambda v: W.Dr(v * W.even) * W.even)[np.ix_(ev, ev)]
    u = _vec(W.dims, 7) * W.even
    got = W.gamma5(W.Minv(W.Dr(W.M(W.gamma5(u)))) * W.even)
    ref = Dr.conj().T @ u.ravel()[ev]
    assert np.abs(got.ravel()[ev] - ref).max() < 1e-12 * np.abs(ref).max()
    # and D_r itself is not normal here, so the check has teeth
    assert np.abs(Dr @ Dr.conj().T - Dr.conj().T @ Dr).max() > 1e-3


# ----------------------------------------------------------------------------- anisotropic reading
AW = (0.45, 0.7, 1.25, 2.0)   # hopping weights x, y, z, t (all different: a transposed index fails)


def test_anisotropic_free_field_plane_wave():
    """The anisotropic reading at U = 1: D e^{ipx} u = [m0 + sum_mu w_mu (1 - cos p_mu)
    + i sum_mu w_mu gamma_mu sin p_mu] e^{ipx} u (the clover term vanishes)."""
    dims = (4, 6, 2, 8)
    lx, ly, lz, lt = dims
    m0 = -0.15
    W = WilsonClover(I.unit_gauge(dims), 1.1, m0, weights=AW, csw_t=0.6)
    rng = np.random.default_rng(5)
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in (lt, lz, ly, lx)], indexing="ij")
    for n in [(0, 0, 0, 0), (1, 2, 1, 3), (3, 5, 1, 6)]:
        p = [2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz, 2 * np.pi * (n[3] + 0.5) / lt]
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        psi = phase[..., None, None] * u
        Dk = (m0 + sum(AW[m] * (1 - np.cos(p[m])) for m in range(4))) * np.eye(4) + \
            1j * sum(AW[m] * GT[m] * np.sin(p[m]) for m in range(4))
        expect = phase[..., None, None] * (Dk @ u)
        got = W.D(psi.reshape(W.shape + (12,))).reshape(expect.shape)
        assert np.abs(got - expect).max() < 1e-13


def test_anisotropic_reading_reduces_to_isotropic():
    """Unit weights and csw_t = csw give exactly the isotropic operator."""
    dims = (4, 4, 4, 4)
    U = I.make_gauge(dims, 0.4, 1, 0.5, 51)
    W = WilsonClover(U, 1.3, -0.2)
    Wa = WilsonClover(U, 1.3, -0.2, weights=(1.0, 1.0, 1.0, 1.0), csw_t=1.3)
    psi = _vec(dims, 52)
    assert np.array_equal(W.A, Wa.A)
    assert np.array_equal(W.D(psi), Wa.D(psi))
    # and a non-trivial anisotropy changes it
    Wb = WilsonClover(U, 1.3, -0.2, weights=AW, csw_t=0.7)
    assert np.abs(Wb.D(psi) - W.D(psi)).max() > 1e-2


def test_anisotropic_gamma5_hermiticity_and_covariance():
    """gamma_5-hermiticity and gauge covariance hold for the anisotropic reading."""
    dims = (4, 4, 2, 6)
    U = I.make_gauge(dims, 0.5, 0, 0.5, 53)
    W = WilsonClover(U, 1.2, -0.3, weights=AW, csw_t=0.8)
    phi, psi = _vec(dims, 54), _vec(dims, 55)
    lhs = inner(phi, W.D(psi))
    assert abs(lhs - inner(W.gamma5(W.D(W.gamma5(phi))), psi)) / abs(lhs) < 1e-14
    G = I.random_gauge_transform(dims, 56)
    UG = np.empty_like(U)
    for mu in range(4):
        Gp = np.roll(G, -1, axis=3 - mu)
        UG[..., mu, :, :] = G @ U[..., mu, :, :] @ np.conj(np.swapaxes(Gp, -1, -2))
    WG = WilsonClover(UG, 1.2, -0.3, weights=AW, csw_t=0.8)
    p4 = psi.reshape(psi.shape[:-1] + (4, 3))
    Gpsi = np.einsum("...ab,...sb->...sa", G, p4)
    lhs = WG.D(Gpsi.reshape(W.shape + (12,))).reshape(p4.shape)
    rhs = np.einsum("...ab,...sb->...sa", G, W.D(psi).reshape(p4.shape))
    assert np.abs(lhs - rhs).max() < 1e-13


@pytest.mark.parametrize("plane", [(0, 1), (2, 3)])
def test_anisotropic_clover_constant_abelian_field(plane):
    """The constant-flux closed form with the plane's own coefficient and the
    weighted mass term: A = (sum w + m0) - (c/2) sin(B) sigma_{mu nu} x diag(1, -1, 0),
    c = csw for a spatial plane and csw_t for a plane containing t."""
    mu, nu = plane
    dims = (4, 4, 4, 4)
    m0, csw, csw_t = -0.1, 1.3, 0.55
    B = 2 * np.pi / dims[mu]
    U = I.unit_gauge(dims)
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in I.lattice_shape(dims)], indexing="ij")
    th = B * (x, y, z, t)[mu]
    U[..., nu, 0, 0] = np.exp(1j * th)
    U[..., nu, 1, 1] = np.exp(-1j * th)
    W = WilsonClover(U, csw, m0, weights=AW, csw_t=csw_t)
    c = csw_t if 3 in plane else csw
    sig = 0.5j * (GT[mu] @ GT[nu] - GT[nu] @ GT[mu])
    expect = (sum(AW) + m0) * np.eye(12) - 0.5 * c * np.sin(B) * np.kron(sig, np.diag([1.0, -1.0, 0.0]))
    assert np.abs(W.A - expect).max() < 1e-14


def test_uniform_weights_scale_the_isotropic_operator():
    """With every weight equal to w and csw_t = csw the reading is w times the
    isotropic operator of coefficient csw / w and mass m0 / w (the mass term
    4 w + m0 and the clover term, linear in its coefficient, both scale): this
    ties the weights of the hops, of the mass term and of the clover
    coefficient to one another on a rough field."""
    dims = (4, 4, 2, 6)
    U = I.make_gauge(dims, 0.6, 1, 0.5, 57)
    w, csw, m0 = 1.7, 1.2, -0.3
    Wa = WilsonClover(U, csw, m0, weights=(w, w, w, w), csw_t=csw)
    Wi = WilsonClover(U, csw / w, m0 / w)
    psi = _vec(dims, 58)
    ref = w * Wi.D(psi)
    assert np.abs(Wa.D(psi) - ref).max() < 1e-13 * np.abs(ref).max()
    assert np.abs(Wa.A - w * Wi.A).max() < 1e-13 * np.abs(Wa.A).max()
