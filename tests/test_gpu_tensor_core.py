"""GPU parity of the coarsest-level GCR on tensor cores (mg_params.coarse_impl
= 4: FP16 links, mma.sync with FP32 accumulation, the vectors split into FP16
hi + lo parts), through the C ABI.

The kernel applies exactly the operator of the stored links, so it is checked
like every 16-bit path: against the oracle applied to the GPU's dequantised P
and coarse links (one cycle with a near-exact coarsest solve, 1e-4 as the
other cycle tests), for one system and for batches of up to 16 right-hand
sides in one launch (the batched cycle of the block solve), at Nc = 16, 48
and 64.  Block solves reach 1e-10 with the oracle's D, agree with one-at-a-time
solves and repeat bit for bit.
"""
import numpy as np
import pytest

from gpu_common import lib_built, rel
from oracle.dirac import WilsonClover, norm2
from oracle.multigrid import CoarseLevel, MGParams, Multigrid, Transfer
from oracle.philox import gaussian_vector
from paper_1011_2775_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP16 = 1


def _solver(dims, U, csw, m0):
    lib_built()
    from paper_1011_2775_gb300.solver import Solver
    S = Solver(dims)
    S.load_gauge(U)
    S.set_clover(csw, m0)
    return S


def _extract_P(S, level, fine_shape, fine_ndof, cshape, nv):
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


def _dequantised(S, W, blocks, nv, cdims, mg):
    """The oracle hierarchy on the GPU's dequantised P and coarse links."""
    lev = [W]
    for l, (blk, k) in enumerate(zip(blocks, nv)):
        fine = lev[l]
        cshape = (cdims[l][3], cdims[l][2], cdims[l][1], cdims[l][0])
        mg.transfers[l] = Transfer(fine, blk, _extract_P(S, l, fine.shape, fine.ndof, cshape, k))
        Y, X = S.coarse_links(l + 1)
        mg.levels[l + 1] = CoarseLevel(cdims[l], X, np.moveaxis(Y, 4, 0))
        lev.append(mg.levels[l + 1])
    return mg


@pytest.fixture(scope="module", params=[((4, 4, 4, 4), 24, (2, 2, 2, 2)), ((2, 2, 2, 2), 8, (4, 4, 4, 4))],
                ids=["nc48", "nc16"])
def two_level(request):
    blk, nv, cd = request.param
    dims = (8, 8, 8, 8)
    U = I.make_gauge(dims, 0.25, 5, 0.5, 9101)
    m0 = -0.3
    W = WilsonClover(U, 1.0, m0)
    V0 = [gaussian_vector(9102, 0, k, W.shape, 12) for k in range(nv)]
    cp = dict(tol_coarse=1e-6, maxit_coarse=400, restart_coarse=64, nu_post=0)
    S = _solver(dims, U, 1.0, m0)
    S.set_params(levels=2, blocks=[blk], nv=[nv], storage=FP16, coarse_impl=4, **cp)
    S.set_null_vectors(0, np.ascontiguousarray(np.stack(V0)))
    S.setup()
    mg = Multigrid(W, MGParams(blocks=[blk], nv=[nv], **cp), null_vectors=[V0])
    mg = _dequantised(S, W, [blk], [nv], [cd], mg)
    yield dict(dims=dims, W=W, S=S, mg=mg)
    S.close()


def test_tensor_core_cycle_one_system(two_level):
    from paper_1011_2775_gb300 import binding as B
    S, W, mg = two_level["S"], two_level["W"], two_level["mg"]
    r = I.gaussian_source(two_level["dims"], 9103)
    got = S.apply(B.MG_OP_CYCLE, r, level=0)
    ref = mg.cycle(0, r.reshape(W.shape + (12,)) * W.even).reshape(r.shape)
    assert rel(got, ref) <= 1e-4


@pytest.mark.parametrize("nrhs", [3, 8, 12, 16])
def test_tensor_core_batched_cycle(two_level, nrhs):
    """All coarsest solves of the batch in one tensor-core launch; right-hand
    sides of different scales and a zero one."""
    from paper_1011_2775_gb300 import binding as B
    S, W, mg = two_level["S"], two_level["W"], two_level["mg"]
    r = I.gaussian_source(two_level["dims"], 9104, nrhs=nrhs)
    r[1] *= 1e-3
    r[nrhs - 1] = 0.0
    got = S.apply(B.MG_OP_CYCLE, r, level=0, nrhs=nrhs)
    for q in range(nrhs):
        if q == nrhs - 1:
            assert not got[q].any()
            continue
        ref = mg.cycle(0, r[q].reshape(W.shape + (12,)) * W.even).reshape(r[q].shape)
        assert rel(got[q], ref) <= 1e-4, q


def test_tensor_core_nc64_level_cycle():
    """Nc = 64 coarsest lattice (8^4, 2^4 blocks with Nv = 24, then 2^4 blocks
    with Nv = 32): the level-1 cycle with the tensor-core coarsest solve."""
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 8)
    U = I.make_gauge(dims, 0.25, 5, 0.5, 9201)
    m0 = -0.3
    W = WilsonClover(U, 1.0, m0)
    V0 = [gaussian_vector(9202, 0, k, W.shape, 12) for k in range(24)]
    V1 = [gaussian_vector(9203, 1, k, (4, 4, 4, 4), 48) for k in range(32)]
    blocks = [(2, 2, 2, 2), (2, 2, 2, 2)]
    cp = dict(tol_coarse=1e-6, maxit_coarse=400, restart_coarse=64, nu_post=2)
    S = _solver(dims, U, 1.0, m0)
    S.set_params(levels=3, blocks=blocks, nv=[24, 32], storage=FP16, coarse_impl=4, **cp)
    S.set_null_vectors(0, np.ascontiguousarray(np.stack(V0)))
    S.set_null_vectors(1, np.ascontiguousarray(np.stack(V1)))
    S.setup()
    mg = Multigrid(W, MGParams(blocks=blocks, nv=[24, 32], **cp), null_vectors=[V0, V1])
    mg = _dequantised(S, W, blocks, [24, 32], [(4, 4, 4, 4), (2, 2, 2, 2)], mg)
    lev = mg.levels[1]
    rng = np.random.default_rng(9204)
    r = rng.standard_normal(lev.shape + (lev.ndof,)) + 1j * rng.standard_normal(lev.shape + (lev.ndof,))
    got = S.apply(B.MG_OP_CYCLE, np.ascontiguousarray(r), level=1)
    ref = mg.cycle(1, r * lev.even)
    assert rel(got.reshape(ref.shape), ref) <= 1e-4
    S.close()


def test_tensor_core_block_solve():
    """FP16 storage, 12 right-hand sides solved in lock-step with their
    coarsest solves on tensor cores: every solution reaches 1e-10 with the
    oracle's D, agrees with one-at-a-time solves (single-system tensor-core
    coarsest solves), and a second block solve repeats the first bit for bit."""
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 16)
    U = I.make_gauge(dims, 1.0, 5, 0.5, 9301)
    W = WilsonClover(U, 1.0, -0.6)
    S = _solver(dims, U, 1.0, -0.6)
    S.set_params(levels=2, blocks=[(4, 4, 4, 4)], nv=[12], seed=9302, storage=FP16, coarse_impl=4, maxit_fine=2000)
    S.setup()
    nrhs = 12
    eta = I.gaussian_source(dims, 9303, nrhs=nrhs)
    S.set_params(rhs_block=nrhs)
    psi, info = S.solve(eta, 1e-10, B.MG_MODE_MG)
    psi2, info2 = S.solve(eta, 1e-10, B.MG_MODE_MG)
    for q in range(nrhs):
        res = eta[q].reshape(W.shape + (12,)) - W.D(psi[q].reshape(W.shape + (12,)))
        assert np.sqrt(norm2(res) / norm2(eta[q])) <= 1e-10, q
    assert np.array_equal(psi, psi2) and info2.outer_iterations == info.outer_iterations
    assert info.coarse_iterations[1] > 0
    S.set_params(rhs_block=1)
    seq, sinfo = S.solve(eta, 1e-10, B.MG_MODE_MG)
    for q in range(nrhs):
        assert np.linalg.norm((psi[q] - seq[q]).ravel()) / np.linalg.norm(seq[q].ravel()) < 1e-7, q
    assert info.outer_iterations <= 1.3 * sinfo.outer_iterations + 3
    S.close()


@pytest.mark.parametrize("store", [1, 2], ids=["fp16", "bf16"])
@pytest.mark.parametrize("nrhs", [8, 13])
def test_batched_transfers_match_single(store, nrhs):
    """The fine-level restriction and prolongation of nrhs right-hand sides in
    one launch each (one batched cycle, groups of 4 with a ragged last group)
    against the same cycle done one right-hand side at a time, and against
    the oracle's cycle on the dequantised operands, with 16-bit P (Nv = 8 on
    2^4 blocks, even sites) and a right-hand side scaled by 1e-6."""
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 8)
    U = I.make_gauge(dims, 0.25, 5, 0.5, 9401)
    m0 = -0.3
    W = WilsonClover(U, 1.0, m0)
    V0 = [gaussian_vector(9402, 0, k, W.shape, 12) for k in range(8)]
    cp = dict(tol_coarse=1e-6, maxit_coarse=400, restart_coarse=64, nu_post=0)
    S = _solver(dims, U, 1.0, m0)
    S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[8], storage=store, coarse_impl=1, **cp)
    S.set_null_vectors(0, np.ascontiguousarray(np.stack(V0)))
    S.setup()
    mg = Multigrid(W, MGParams(blocks=[(2, 2, 2, 2)], nv=[8], **cp), null_vectors=[V0])
    mg = _dequantised(S, W, [(2, 2, 2, 2)], [8], [(4, 4, 4, 4)], mg)
    r = I.gaussian_source(dims, 9403, nrhs=nrhs)
    r[2] *= 1e-6
    got = S.apply(B.MG_OP_CYCLE, r, level=0, nrhs=nrhs)
    for q in range(nrhs):
        one = S.apply(B.MG_OP_CYCLE, np.ascontiguousarray(r[q]), level=0)
        assert rel(got[q], one) <= 1e-5, q
        ref = mg.cycle(0, r[q].reshape(W.shape + (12,)) * W.even).reshape(r[q].shape)
        assert rel(got[q], ref) <= 1e-4, q
    S.close()
