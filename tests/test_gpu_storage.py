"""GPU parity of the 16-bit (FP16 / BF16) storage of prolongators and coarse
links, through the C ABI.

The kernels compute in FP32 from stored 16-bit values times an FP32 scale per
tile.  Parity is checked as the library defines it -- against the oracle
applied to the dequantised operands the GPU holds -- plus a bound on the
quantisation itself:

* P: columns extracted from the GPU (P applied to unit coarse vectors, exact
  in FP32) lie within half an ulp per component of the tile scale of the
  oracle's FP64 P (2^-12 for FP16, 2^-9 for BF16); R and P on the GPU equal the oracle's
  Transfer built on those columns (relative 1e-5).
* Y, X: mg_get_coarse_links returns the dequantised links; they lie within the
  same bound of the oracle's Galerkin links built from the extracted P, and
  the GPU's coarse D, D_p, D_r, hop equal the oracle's operator on those links
  (1e-5), on levels 1 and 2 of a 3-level hierarchy.
* One multigrid cycle equals the oracle's cycle on the dequantised hierarchy
  (1e-4, as the FP32 test), and MG-GCR reaches ||eta - D psi|| <= 1e-10.
"""
import numpy as np
import pytest

from gpu_common import TOL32, lib_built, rel
from oracle.dirac import WilsonClover, norm2
from oracle.multigrid import CoarseLevel, MGParams, Multigrid, Transfer, build_coarse
from oracle.philox import gaussian_vector
from paper_1011_2775_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# half an ulp at 1 (relative to the tile scale) of the stored format
HALF_ULP = {1: 2.0 ** -12, 2: 2.0 ** -9}


def _solver(dims, U, csw, m0):
    lib_built()
    from paper_1011_2775_gb300.solver import Solver
    S = Solver(dims)
    S.load_gauge(U)
    S.set_clover(csw, m0)
    return S


def _extract_P(S, level, fine_shape, fine_ndof, cshape, nv):
    """P of transfer `level` as the oracle's (fine_shape + (ndof, nv)) array,
    from P applied to the unit vector of every coarse dof at every coarse site
    (the blocks are disjoint, so each application yields one column per block)."""
    from paper_1011_2775_gb300 import binding as B
    h = fine_ndof // 2
    P = np.zeros(fine_shape + (fine_ndof, nv), dtype=np.complex128)
    out_shape = fine_shape + ((4, 3) if fine_ndof == 12 else (fine_ndof,))
    for s in range(2):
        for k in range(nv):
            e = np.zeros(cshape + (2 * nv,), dtype=np.complex128)
            e[..., s * nv + k] = 1.0
            col = S.apply(B.MG_OP_P, e, level=level, out_shape=out_shape).reshape(fine_shape + (fine_ndof,))
            P[..., s * h:(s + 1) * h, k] = col[..., s * h:(s + 1) * h]
    return P


def _tile_bound(ref, store):
    """Elementwise bound |stored - ref| <= sqrt(2) half_ulp * tile scale + FP32
    slack (half an ulp on each of Re and Im), with the tile scale taken as the
    largest |Re|, |Im| of the reference tile (the FP32 tile differs from it by
    FP32 rounding only)."""
    scale = np.maximum(np.abs(ref.real), np.abs(ref.imag)).max(axis=(-2, -1), keepdims=True)
    return np.sqrt(2.0) * HALF_ULP[store] * scale * (1 + 1e-4) + 2e-6 * np.abs(ref).max()


@pytest.fixture(scope="module", params=[1, 2], ids=["fp16", "bf16"])
def quantised3(request):
    """3 levels on 8^4 (2^4 blocks, Nv = 8, then 2^4 blocks, Nv = 6), injected
    null vectors, 16-bit storage of P and the coarse links."""
    store = request.param
    dims = (8, 8, 8, 8)
    U = I.make_gauge(dims, 0.3, 1, 0.5, 6001)
    W = WilsonClover(U, 1.0, -0.2)
    V0 = [gaussian_vector(61, 0, k, W.shape, 12) for k in range(8)]
    V1 = [gaussian_vector(62, 1, k, (4, 4, 4, 4), 16) for k in range(6)]
    S = _solver(dims, U, 1.0, -0.2)
    S.set_params(levels=3, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[8, 6], storage=store)
    S.set_null_vectors(0, np.ascontiguousarray(np.stack(V0)))
    S.set_null_vectors(1, np.ascontiguousarray(np.stack(V1)))
    S.setup()
    # FP64 reference hierarchy from the same vectors
    ref = Multigrid(W, MGParams(blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[8, 6]), null_vectors=[V0, V1])
    # the oracle on the GPU's dequantised operands, level by level
    P0 = _extract_P(S, 0, W.shape, 12, (4, 4, 4, 4), 8)
    T0 = Transfer(W, (2, 2, 2, 2), P0)
    Y1, X1 = S.coarse_links(1)
    L1 = CoarseLevel((4, 4, 4, 4), X1, np.moveaxis(Y1, 4, 0))
    P1 = _extract_P(S, 1, (4, 4, 4, 4), 16, (2, 2, 2, 2), 6)
    T1 = Transfer(L1, (2, 2, 2, 2), P1)
    Y2, X2 = S.coarse_links(2)
    L2 = CoarseLevel((2, 2, 2, 2), X2, np.moveaxis(Y2, 4, 0))
    yield dict(store=store, dims=dims, U=U, W=W, S=S, ref=ref, T=[T0, T1], L=[W, L1, L2],
               links=[(Y1, X1), (Y2, X2)])
    S.close()


def test_quantised_P_within_bound(quantised3):
    q = quantised3
    for l in range(2):
        Pq = q["T"][l].P
        # block Gram-Schmidt depends on the vectors only, not on the operator
        Pref = q["ref"].transfers[l].P
        # tiles: (coarse site, chirality) -> reshape to blocks
        T = q["T"][l]
        h = T.half
        for s in range(2):
            ref_t = T._split(Pref[..., s * h:(s + 1) * h, :])
            got_t = T._split(Pq[..., s * h:(s + 1) * h, :])
            # move the block-local axes (1, 3, 5, 7) and the dof/vector axes together
            ax = (0, 2, 4, 6, 1, 3, 5, 7, 8, 9)
            ref_t = np.transpose(ref_t, ax).reshape(ref_t.shape[0] * ref_t.shape[2] * ref_t.shape[4] * ref_t.shape[6],
                                                   -1, 1)
            got_t = np.transpose(got_t, ax).reshape(ref_t.shape)
            err = np.abs(got_t - ref_t)
            assert (err <= _tile_bound(ref_t, q["store"])).all()
        assert np.abs(Pq - Pref).max() > 0      # the storage really is 16-bit


@pytest.mark.parametrize("level", [0, 1])
def test_restrict_prolong_on_dequantised_P(quantised3, level):
    from paper_1011_2775_gb300 import binding as B
    q = quantised3
    T, fine = q["T"][level], q["L"][level]
    rng = np.random.default_rng(level + 5)
    v = rng.standard_normal(fine.shape + (fine.ndof,)) + 1j * rng.standard_normal(fine.shape + (fine.ndof,))
    vc = rng.standard_normal(T.cshape + (2 * T.nv,)) + 1j * rng.standard_normal(T.cshape + (2 * T.nv,))
    S = q["S"]
    assert rel(S.apply(B.MG_OP_R, np.ascontiguousarray(v), level=level, out_shape=vc.shape), T.restrict(v)) <= TOL32
    assert rel(S.apply(B.MG_OP_P, np.ascontiguousarray(vc), level=level, out_shape=v.shape), T.prolong(vc)) <= TOL32


@pytest.mark.parametrize("level", [1, 2])
def test_quantised_links_within_bound(quantised3, level):
    """The GPU's stored Y is the oracle's Galerkin Y (from the GPU's P on the
    level above) rounded to 16 bits per tile; X stays FP32."""
    q = quantised3
    Y, X = q["links"][level - 1]
    C = build_coarse(q["L"][level - 1], q["T"][level - 1])
    Yref = np.moveaxis(C.Y, 0, 4)               # (Tc, Zc, Yc, Xc, 8, nc, nc)
    assert (np.abs(Y - Yref) <= _tile_bound(Yref, q["store"])).all()
    assert rel(X, C.X) <= TOL32


@pytest.mark.parametrize("level", [1, 2])
@pytest.mark.parametrize("op", ["D", "DP", "DR", "HOP"])
def test_coarse_operator_on_dequantised_links(quantised3, level, op):
    from paper_1011_2775_gb300 import binding as B
    q = quantised3
    C = q["L"][level]
    rng = np.random.default_rng(20 + level)
    v = rng.standard_normal(C.shape + (C.ndof,)) + 1j * rng.standard_normal(C.shape + (C.ndof,))
    ref = {"D": C.D, "DP": C.Dp, "DR": lambda x: C.Dr(x * C.even), "HOP": C.hop}[op](v)
    got = q["S"].apply(getattr(B, "MG_OP_" + op), np.ascontiguousarray(v), level=level)
    assert rel(got, ref) <= TOL32


@pytest.mark.parametrize("store", [1, 2], ids=["fp16", "bf16"])
def test_cycle_parity_quantised(store):
    """One cycle with a near-exact coarsest solve equals the oracle's cycle on
    the GPU's dequantised P and links (2 levels, QCD-like 8^4 field)."""
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 8)
    U = I.make_gauge(dims, 1.0, 5, 0.5, 2001)
    W = WilsonClover(U, 1.0, -0.6)
    V0 = [gaussian_vector(91, 0, k, W.shape, 12) for k in range(8)]
    prm = dict(tol_coarse=1e-6, maxit_coarse=400, restart_coarse=64, nu_post=2)
    S = _solver(dims, U, 1.0, -0.6)
    S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[8], storage=store, **prm)
    S.set_null_vectors(0, np.ascontiguousarray(np.stack(V0)))
    S.setup()
    mg = Multigrid(W, MGParams(blocks=[(2, 2, 2, 2)], nv=[8], **prm), null_vectors=[V0])
    mg.transfers[0] = Transfer(W, (2, 2, 2, 2), _extract_P(S, 0, W.shape, 12, (4, 4, 4, 4), 8))
    Y, X = S.coarse_links(1)
    mg.levels[1] = CoarseLevel((4, 4, 4, 4), X, np.moveaxis(Y, 4, 0))
    r = I.gaussian_source(dims, 7)
    got = S.apply(B.MG_OP_CYCLE, r, level=0)
    ref = mg.cycle(0, r.reshape(W.shape + (12,)) * W.even).reshape(r.shape)
    assert rel(got, ref) <= 1e-4
    eta = I.gaussian_source(dims, 8)
    psi, info = S.solve(eta, 1e-10)
    res = eta.reshape(W.shape + (12,)) - W.D(psi.reshape(W.shape + (12,)))
    assert np.sqrt(norm2(res) / norm2(eta)) <= 1e-10
    S.close()


@pytest.mark.parametrize("store", [1, 2], ids=["fp16", "bf16"])
def test_quantised_three_level_solve(store):
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 16)
    U = I.make_gauge(dims, 1.0, 5, 0.5, 5001)
    W = WilsonClover(U, 1.0, -0.6)
    S = _solver(dims, U, 1.0, -0.6)
    S.set_params(levels=3, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[8, 8], storage=store, maxit_fine=2000)
    S.setup()
    eta = I.gaussian_source(dims, 5002)
    psi, info = S.solve(eta, 1e-10, B.MG_MODE_MG)
    res = eta.reshape(W.shape + (12,)) - W.D(psi.reshape(W.shape + (12,)))
    assert np.sqrt(norm2(res) / norm2(eta)) <= 1e-10
    assert info.coarse_iterations[2] > 0
    S.close()
