"""GPU parity of the multigrid pieces at the sizes the benchmark runs, through
the C ABI.

The benchmark hierarchy has Nv = 24 null vectors on 4^4 blocks (Nc = 48 coarse
dof per site, 256 fine sites per block) and, with three levels, Nv = 32 on the
second transfer (Nc = 64).  Several kernels size their work by Nc (GEMV rows
per warp, the pivot buffer of the coarse site inverse, the persistent
coarsest solve), so their parity is checked at exactly these Nc:

* ``nv24``: 8^4 fine lattice of the benchmark ensemble, 4^4 blocks, Nv = 24
  (coarse lattice 2^4, Nc = 48), injected null vectors, FP32 and BF16 storage.
* ``nv24_32``: 8^4, 2^4 blocks with Nv = 24 (4^4, Nc = 48), then 2^4 blocks
  with Nv = 32 (2^4, Nc = 64).
* The 16^3x32 benchmark lattice itself (the GPU's own setup, as timed): R and
  P against the oracle's block Gram-Schmidt of the GPU's null vectors, and the
  coarse operator on one vector against ``R D_p P`` with the oracle's fine
  D_p (the Galerkin definition, section "Red-black preconditioning").

Tolerances: 1e-5 relative for FP32 kernels, 1e-4 for a cycle (an FP32 Krylov
solve inside), as in the smaller parity tests; 16-bit storage is compared
against the oracle on the GPU's dequantised operands.
"""
import numpy as np
import pytest

from gpu_common import TOL32, lib_built, rel
from oracle.dirac import WilsonClover, norm2
from oracle.multigrid import CoarseLevel, MGParams, Multigrid, Transfer, block_gram_schmidt, build_coarse
from oracle.philox import gaussian_vector
from paper_1011_2775_gb300 import inputs as I

pytestmark = pytest.mark.gpu

OPS = ["D", "DP", "DR", "BR", "M", "MINV", "HOP"]


def _solver(dims, U, csw, m0):
    lib_built()
    from paper_1011_2775_gb300.solver import Solver
    S = Solver(dims)
    S.load_gauge(U)
    S.set_clover(csw, m0)
    return S


def _extract_P(S, level, fine_shape, fine_ndof, cshape, nv):
    """The GPU's (dequantised) P of transfer `level`, from P applied to unit
    coarse vectors (blocks are disjoint: one application gives one column per
    block)."""
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


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _op_ref(C, op):
    return {"D": C.D, "DP": C.Dp, "DR": lambda x: C.Dr(x * C.even), "BR": C.b_r, "M": C.M, "MINV": C.Minv,
            "HOP": C.hop}[op]


# ----------------------------------------------------------------------------- Nv = 24 on 4^4 blocks
@pytest.fixture(scope="module", params=[0, 2], ids=["fp32", "bf16"])
def nv24(request):
    store = request.param
    dims = (8, 8, 8, 8)
    U = I.make_gauge(dims, 0.25, 5, 0.5, 8101)
    m0 = -0.3
    W = WilsonClover(U, 1.0, m0)
    V0 = [gaussian_vector(8102, 0, k, W.shape, 12) for k in range(24)]
    cp = dict(tol_coarse=1e-6, maxit_coarse=400, restart_coarse=64)
    S = _solver(dims, U, 1.0, m0)
    S.set_params(levels=2, blocks=[(4, 4, 4, 4)], nv=[24], storage=store, nu_post=0, **cp)
    S.set_null_vectors(0, np.ascontiguousarray(np.stack(V0)))
    S.setup()
    ref = Multigrid(W, MGParams(blocks=[(4, 4, 4, 4)], nv=[24], nu_post=0, **cp), null_vectors=[V0])
    if store:
        # the oracle on the GPU's dequantised P and links
        ref.transfers[0] = Transfer(W, (4, 4, 4, 4), _extract_P(S, 0, W.shape, 12, (2, 2, 2, 2), 24))
        Y, X = S.coarse_links(1)
        ref.levels[1] = CoarseLevel((2, 2, 2, 2), X, np.moveaxis(Y, 4, 0))
    yield dict(store=store, dims=dims, W=W, S=S, ref=ref, V0=V0)
    S.close()


def test_nv24_level_info(nv24):
    assert nv24["S"].level_info(1) == ((2, 2, 2, 2), 48)


def test_nv24_restrict_prolong(nv24):
    from paper_1011_2775_gb300 import binding as B
    S, W, T = nv24["S"], nv24["W"], nv24["ref"].transfers[0]
    v = _rand(W.shape + (12,), 1)
    vc = _rand(T.cshape + (48,), 2)
    got_r = S.apply(B.MG_OP_R, np.ascontiguousarray(v.reshape(W.shape + (4, 3))), level=0, out_shape=vc.shape)
    assert rel(got_r, T.restrict(v)) <= TOL32
    got_p = S.apply(B.MG_OP_P, vc, level=0, out_shape=W.shape + (4, 3))
    assert rel(got_p.reshape(W.shape + (12,)), T.prolong(vc)) <= TOL32


def test_nv24_P_is_the_oracle_block_gram_schmidt(nv24):
    """FP32 storage: the GPU's P equals the oracle's block Gram-Schmidt of the
    same vectors (256 fine sites x 6 components per (block, chirality) tile)."""
    if nv24["store"]:
        pytest.skip("16-bit P is compared through its dequantised values")
    S, W = nv24["S"], nv24["W"]
    Pg = _extract_P(S, 0, W.shape, 12, (2, 2, 2, 2), 24)
    Po = block_gram_schmidt(W, (4, 4, 4, 4), nv24["V0"])
    assert rel(Pg, Po) <= TOL32


def test_nv24_coarse_links(nv24):
    """X and the eight Y_d of the GPU against the oracle's Galerkin links
    (FP32 storage) -- for 16-bit storage the fixture already holds the
    dequantised GPU links, so compare them to the oracle's links from the same P."""
    S, W, ref = nv24["S"], nv24["W"], nv24["ref"]
    Y, X = S.coarse_links(1)
    C = build_coarse(W, ref.transfers[0])
    Yref = np.moveaxis(C.Y, 0, 4)
    assert rel(X, C.X) <= TOL32
    if nv24["store"] == 0:
        assert rel(Y, Yref) <= TOL32
    else:
        scale = np.maximum(np.abs(Yref.real), np.abs(Yref.imag)).max(axis=(-2, -1), keepdims=True)
        assert (np.abs(Y - Yref) <= np.sqrt(2.0) * 2.0 ** -9 * scale * (1 + 1e-4) + 2e-6 * np.abs(Yref).max()).all()


@pytest.mark.parametrize("op", OPS)
def test_nv24_coarse_operator(nv24, op):
    from paper_1011_2775_gb300 import binding as B
    S, C = nv24["S"], nv24["ref"].levels[1]
    v = _rand(C.shape + (C.ndof,), 3)
    got = S.apply(getattr(B, "MG_OP_" + op), v, level=1)
    assert rel(got, _op_ref(C, op)(v)) <= TOL32


def test_nv24_cycle_through_persistent_coarsest_solve(nv24):
    """nu_post = 0: the cycle is the even part of P D_hat^{-1} R (r_e, 0), the
    coarsest system solved by the persistent kernel to 1e-6 at Nc = 48."""
    from paper_1011_2775_gb300 import binding as B
    S, W, mg = nv24["S"], nv24["W"], nv24["ref"]
    r = I.gaussian_source(nv24["dims"], 8103)
    got = S.apply(B.MG_OP_CYCLE, r, level=0)
    ref = mg.cycle(0, r.reshape(W.shape + (12,)) * W.even).reshape(r.shape)
    assert rel(got, ref) <= 1e-4


# ----------------------------------------------------------------------------- Nv = 24 then Nv = 32
@pytest.fixture(scope="module")
def nv24_32():
    dims = (8, 8, 8, 8)
    U = I.make_gauge(dims, 0.25, 5, 0.5, 8201)
    m0 = -0.3
    W = WilsonClover(U, 1.0, m0)
    V0 = [gaussian_vector(8202, 0, k, W.shape, 12) for k in range(24)]
    V1 = [gaussian_vector(8203, 1, k, (4, 4, 4, 4), 48) for k in range(32)]
    cp = dict(tol_coarse=1e-6, maxit_coarse=400, restart_coarse=64, nu_post=2)
    blocks = [(2, 2, 2, 2), (2, 2, 2, 2)]
    S = _solver(dims, U, 1.0, m0)
    S.set_params(levels=3, blocks=blocks, nv=[24, 32], **cp)
    S.set_null_vectors(0, np.ascontiguousarray(np.stack(V0)))
    S.set_null_vectors(1, np.ascontiguousarray(np.stack(V1)))
    S.setup()
    ref = Multigrid(W, MGParams(blocks=blocks, nv=[24, 32], **cp), null_vectors=[V0, V1])
    yield dict(dims=dims, W=W, S=S, ref=ref)
    S.close()


def test_nv24_32_level_info(nv24_32):
    S = nv24_32["S"]
    assert S.level_info(1) == ((4, 4, 4, 4), 48)
    assert S.level_info(2) == ((2, 2, 2, 2), 64)


@pytest.mark.parametrize("level", [0, 1])
def test_nv24_32_restrict_prolong(nv24_32, level):
    from paper_1011_2775_gb300 import binding as B
    S, mg = nv24_32["S"], nv24_32["ref"]
    T, fine = mg.transfers[level], mg.levels[level]
    v = _rand(fine.shape + (fine.ndof,), 10 + level)
    vc = _rand(T.cshape + (2 * T.nv,), 20 + level)
    fshape = fine.shape + ((4, 3) if fine.ndof == 12 else (fine.ndof,))
    got_r = S.apply(B.MG_OP_R, np.ascontiguousarray(v.reshape(fshape)), level=level, out_shape=vc.shape)
    assert rel(got_r, T.restrict(v)) <= TOL32
    got_p = S.apply(B.MG_OP_P, vc, level=level, out_shape=fshape)
    assert rel(got_p.reshape(v.shape), T.prolong(vc)) <= TOL32


@pytest.mark.parametrize("level", [1, 2])
def test_nv24_32_coarse_links(nv24_32, level):
    S, mg = nv24_32["S"], nv24_32["ref"]
    Y, X = S.coarse_links(level)
    C = mg.levels[level]
    assert rel(X, C.X) <= TOL32
    assert rel(Y, np.moveaxis(C.Y, 0, 4)) <= TOL32


@pytest.mark.parametrize("level", [1, 2])
@pytest.mark.parametrize("op", OPS)
def test_nv24_32_coarse_operator(nv24_32, level, op):
    from paper_1011_2775_gb300 import binding as B
    S, C = nv24_32["S"], nv24_32["ref"].levels[level]
    v = _rand(C.shape + (C.ndof,), 30 + level)
    got = S.apply(getattr(B, "MG_OP_" + op), v, level=level)
    assert rel(got, _op_ref(C, op)(v)) <= TOL32


@pytest.mark.parametrize("level", [1, 0])
def test_nv24_32_cycle(nv24_32, level):
    """Level 1: restriction to Nc = 64, the persistent coarsest solve, MR
    smoothing; level 0: the recursive cycle (a level-1 GCR preconditioned by
    the level-1 cycle)."""
    from paper_1011_2775_gb300 import binding as B
    S, mg = nv24_32["S"], nv24_32["ref"]
    lev = mg.levels[level]
    r = _rand(lev.shape + (lev.ndof,), 40 + level)
    shape = lev.shape + ((4, 3) if lev.ndof == 12 else (lev.ndof,))
    got = S.apply(B.MG_OP_CYCLE, np.ascontiguousarray(r.reshape(shape)), level=level)
    ref = mg.cycle(level, r * lev.even)
    assert rel(got.reshape(ref.shape), ref) <= 1e-4


# ----------------------------------------------------------------------------- the 16^3x32 benchmark lattice
@pytest.fixture(scope="module")
def bench_lattice():
    """The benchmark's system and hierarchy (16^3x32, eps = 0.25 + 5 APE,
    csw = 1, m0 = -0.35, 4^4 blocks, Nv = 24), set up by the GPU as timed."""
    dims = (16, 16, 16, 32)
    U = I.make_gauge(dims, 0.25, 5, 0.5, 2001)
    m0 = -0.35
    W = WilsonClover(U, 1.0, m0)
    S = _solver(dims, U, 1.0, m0)
    S.set_params(levels=2, blocks=[(4, 4, 4, 4)], nv=[24], seed=2003)
    S.setup()
    V = S.get_null_vectors(0)
    T = Transfer(W, (4, 4, 4, 4), block_gram_schmidt(W, (4, 4, 4, 4), [v for v in V]))
    yield dict(dims=dims, W=W, S=S, T=T)
    S.close()


def test_bench_lattice_transfers(bench_lattice):
    """R and P of the benchmark hierarchy against the oracle's block
    Gram-Schmidt of the GPU's own null vectors (512 blocks of 256 sites)."""
    from paper_1011_2775_gb300 import binding as B
    S, W, T = bench_lattice["S"], bench_lattice["W"], bench_lattice["T"]
    v = _rand(W.shape + (12,), 50)
    vc = _rand(T.cshape + (48,), 51)
    got_r = S.apply(B.MG_OP_R, np.ascontiguousarray(v.reshape(W.shape + (4, 3))), level=0, out_shape=vc.shape)
    assert rel(got_r, T.restrict(v)) <= TOL32
    got_p = S.apply(B.MG_OP_P, vc, level=0, out_shape=W.shape + (4, 3))
    assert rel(got_p.reshape(W.shape + (12,)), T.prolong(vc)) <= TOL32


def test_bench_lattice_galerkin_operator(bench_lattice):
    """The coarse D_hat of the benchmark hierarchy on one vector equals
    P^dag D_p P v evaluated with the oracle's fine D_p (the Galerkin
    definition), and the coarse D_hat_r its even-odd reduction."""
    from paper_1011_2775_gb300 import binding as B
    S, W, T = bench_lattice["S"], bench_lattice["W"], bench_lattice["T"]
    vc = _rand(T.cshape + (48,), 52)
    ref = T.restrict(W.Dp(T.prolong(vc)))
    got = S.apply(B.MG_OP_D, vc, level=1)
    assert rel(got, ref) <= TOL32
    # D_hat_r y_e = y_e - Y_eo X_o^{-1} Y_oe X_e^{-1} y_e, from the GPU's own
    # site-local and full operators: (D_hat X^{-1}) restricted to even sites
    # is [[1, Y_eo X_o^{-1}], [Y_oe X_e^{-1}, 1]]
    par = np.indices(T.cshape).sum(axis=0) % 2
    ev = (par == 0)[..., None]
    ye = vc * ev
    s = S.apply(B.MG_OP_MINV, np.ascontiguousarray(ye), level=1)
    u = S.apply(B.MG_OP_D, s, level=1) * ~ev                    # Y_oe X_e^{-1} y_e on odd sites
    t = S.apply(B.MG_OP_MINV, np.ascontiguousarray(u), level=1)
    w = S.apply(B.MG_OP_HOP, t, level=1) * ev                    # Y_eo X_o^{-1} (...)
    got_r = S.apply(B.MG_OP_DR, np.ascontiguousarray(ye), level=1)
    assert rel(got_r * ev, ye - w) <= TOL32


@pytest.mark.parametrize("impl", [1, 2, 3], ids=["single", "batched", "streamed"])
def test_nv24_cycle_with_each_coarsest_solver(nv24, impl):
    """The three persistent coarsest-level solvers (mg_params.coarse_impl: the
    single-system kernel, the batched kernel with one system, the kernel that
    streams the links through shared memory) each reproduce the oracle's
    cycle at Nc = 48."""
    from paper_1011_2775_gb300 import binding as B
    S, W, mg = nv24["S"], nv24["W"], nv24["ref"]
    S.set_params(coarse_impl=impl)
    try:
        r = I.gaussian_source(nv24["dims"], 8104)
        got = S.apply(B.MG_OP_CYCLE, r, level=0)
        ref = mg.cycle(0, r.reshape(W.shape + (12,)) * W.even).reshape(r.shape)
        assert rel(got, ref) <= 1e-4
    finally:
        S.set_params(coarse_impl=0)


@pytest.mark.parametrize("impl", [1, 3], ids=["single", "streamed"])
def test_nv24_32_cycle_with_each_coarsest_solver(nv24_32, impl):
    """Level-1 cycle of the 3-level hierarchy (coarsest Nc = 64) with each
    persistent solver."""
    from paper_1011_2775_gb300 import binding as B
    S, mg = nv24_32["S"], nv24_32["ref"]
    S.set_params(coarse_impl=impl)
    try:
        lev = mg.levels[1]
        r = _rand(lev.shape + (lev.ndof,), 45)
        got = S.apply(B.MG_OP_CYCLE, np.ascontiguousarray(r), level=1)
        ref = mg.cycle(1, r * lev.even)
        assert rel(got.reshape(ref.shape), ref) <= 1e-4
    finally:
        S.set_params(coarse_impl=0)


@pytest.mark.parametrize("store", [0, 1, 2], ids=["fp32", "fp16", "bf16"])
def test_streamed_coarsest_solver_solves_and_is_deterministic(store):
    """MG-GCR with the streamed coarsest solver reaches 1e-10 with the oracle's
    D, iterates as often as with the single-system kernel (the same GCR,
    up to rounding in the Gram-Schmidt norms), and two identical solves agree
    bit for bit (deterministic reductions)."""
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 16)
    U = I.make_gauge(dims, 1.0, 5, 0.5, 8301)
    W = WilsonClover(U, 1.0, -0.6)
    eta = I.gaussian_source(dims, 8302)
    S = _solver(dims, U, 1.0, -0.6)
    S.set_params(levels=2, blocks=[(4, 4, 4, 4)], nv=[16], seed=8303, maxit_fine=3000, storage=store, coarse_impl=3)
    S.setup()
    psi, info = S.solve(eta, 1e-10, B.MG_MODE_MG)
    psi2, info2 = S.solve(eta, 1e-10, B.MG_MODE_MG)
    r = eta.reshape(W.shape + (12,)) - W.D(psi.reshape(W.shape + (12,)))
    assert np.sqrt(norm2(r) / norm2(eta)) <= 1e-10
    assert info2.outer_iterations == info.outer_iterations
    assert np.array_equal(psi, psi2)
    S.set_params(coarse_impl=1)
    _, ref = S.solve(eta, 1e-10, B.MG_MODE_MG)
    assert abs(info.outer_iterations - ref.outer_iterations) <= 2
    S.close()
