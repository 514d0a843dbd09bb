"""GPU parity of the batched (multi-RHS) path, through the C ABI.

* Multi-RHS fine operators (mg_apply with nrhs > 1: every kernel launched once
  for all right-hand sides) against the oracle per right-hand side, FP64
  (<= 1e-12) and FP32 (<= 1e-5), on a lattice with a ragged last CTA.
* The batched cycle (mg_apply MG_OP_CYCLE, nrhs > 1: multi-RHS smoother, all
  coarsest-level solves in one persistent launch) against the oracle's cycle
  per right-hand side (1e-4, as the single-RHS cycle test).
* The lock-step block solve (mg_solve, rhs_block > 1): every right-hand side
  reaches ||eta - D psi|| / ||eta|| <= 1e-10 with the oracle's D, including a
  zero right-hand side, and agrees with one-at-a-time solves.
* mg_solve_batch: several lattices of uneven size solved together, their
  coarsest-level solves sharing persistent launches; every solution against
  the oracle's D of its lattice and against that context's own mg_solve.
* The multi-RHS benchmark entry point reports its byte model.
"""
import numpy as np
import pytest

from gpu_common import TOL32, TOL64, lib_built, rel
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


@pytest.fixture(scope="module")
def ragged():
    dims = (6, 4, 8, 10)
    U = I.make_gauge(dims, 0.4, 1, 0.5, 7001)
    W = WilsonClover(U, 1.3, -0.2)
    S = _solver(dims, U, 1.3, -0.2)
    yield dims, W, S
    S.close()


@pytest.mark.parametrize("nrhs", [2, 5])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("op", ["D", "DP", "DR", "BR", "M", "MINV", "HOP"])
def test_multi_rhs_fine_operators(ragged, op, prec, nrhs):
    from paper_1011_2775_gb300 import binding as B
    dims, W, S = ragged
    x = I.gaussian_source(dims, 7002, nrhs=nrhs)
    got = S.apply(getattr(B, "MG_OP_" + op), x, prec=prec, nrhs=nrhs)
    f = {"D": W.D, "DP": W.Dp, "DR": lambda v: W.Dr(v * W.even), "BR": W.b_r, "M": W.M, "MINV": W.Minv,
         "HOP": W.hop}[op]
    for q in range(nrhs):
        ref = f(x[q].reshape(W.shape + (12,))).reshape(x[q].shape)
        assert rel(got[q], ref) <= (TOL64 if prec == 0 else TOL32), q


def test_batched_cycle_matches_oracle():
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 8)
    U = I.make_gauge(dims, 1.0, 5, 0.5, 2001)
    W = WilsonClover(U, 1.0, -0.6)
    V0 = [gaussian_vector(91, 0, k, W.shape, 12) for k in range(8)]
    prm = dict(tol_coarse=1e-6, maxit_coarse=400, restart_coarse=64, nu_post=2)
    mg = Multigrid(W, MGParams(blocks=[(2, 2, 2, 2)], nv=[8], **prm), null_vectors=[V0])
    S = _solver(dims, U, 1.0, -0.6)
    S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[8], **prm)
    S.set_null_vectors(0, np.ascontiguousarray(np.stack(V0)))
    S.setup()
    nrhs = 3
    r = I.gaussian_source(dims, 7101, nrhs=nrhs)
    r[1] *= 1e-3                                  # different scales: per-problem tolerances
    got = S.apply(B.MG_OP_CYCLE, r, level=0, nrhs=nrhs)
    for q in range(nrhs):
        ref = mg.cycle(0, r[q].reshape(W.shape + (12,)) * W.even).reshape(r[q].shape)
        assert rel(got[q], ref) <= 1e-4, q
    S.close()


def test_block_solve_matches_sequential_and_oracle():
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 16)
    U = I.make_gauge(dims, 1.0, 5, 0.5, 5001)
    W = WilsonClover(U, 1.0, -0.6)
    S = _solver(dims, U, 1.0, -0.6)
    S.set_params(levels=2, blocks=[(4, 4, 4, 4)], nv=[12], seed=7201)
    S.setup()
    nrhs = 4
    eta = I.gaussian_source(dims, 7202, nrhs=nrhs)
    eta[2] = 0.0                                  # a zero right-hand side
    eta[3] = I.point_source(dims, 5, (1, 2, 3, 4))
    psi, info = S.solve(eta, 1e-10, B.MG_MODE_MG)
    for q in range(nrhs):
        if q == 2:
            assert not psi[q].any()
            continue
        res = eta[q].reshape(W.shape + (12,)) - W.D(psi[q].reshape(W.shape + (12,)))
        assert np.sqrt(norm2(res) / norm2(eta[q])) <= 1e-10, q
    assert info.true_residual <= 1e-10
    S.set_params(rhs_block=1)                     # one after another (the setup is kept)
    seq, sinfo = S.solve(eta, 1e-10, B.MG_MODE_MG)
    for q in (0, 1, 3):
        assert np.linalg.norm((psi[q] - seq[q]).ravel()) / np.linalg.norm(seq[q].ravel()) < 1e-7, q
    # lock-step does not change the per-rhs convergence much
    assert info.outer_iterations <= 1.3 * sinfo.outer_iterations + 3
    S.close()


def test_block_solve_device_buffers_and_dagger():
    torch = pytest.importorskip("torch")
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 8)
    U = I.make_gauge(dims, 0.3, 1, 0.5, 5201)
    W = WilsonClover(U, 1.0, -0.1)
    S = _solver(dims, U, 1.0, -0.1)
    S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[8], seed=5203)
    S.setup()
    chi = I.gaussian_source(dims, 7301, nrhs=3)
    lam, _ = S.solve_dagger(torch.from_numpy(chi).cuda(), 1e-10)
    lam = lam.cpu().numpy()
    for q in range(3):
        lv = lam[q].reshape(W.shape + (12,))
        r = chi[q].reshape(W.shape + (12,)) - W.gamma5(W.D(W.gamma5(lv)))
        assert np.sqrt(norm2(r) / norm2(chi[q])) <= 1e-10
    S.close()


def test_multi_rhs_benchmark_byte_model():
    from paper_1011_2775_gb300 import binding as B
    dims = (8, 8, 8, 16)
    U = I.make_gauge(dims, 0.3, 0, 0.5, 7401)
    S = _solver(dims, U, 1.0, -0.1)
    vh = 8 * 8 * 8 * 16 // 2
    for k, per in [(B.MG_KERNEL_DSLASH_CLOVER, lambda r: 216 + 48 * r), (B.MG_KERNEL_DSLASH_XPAY, lambda r: 144 + 72 * r),
                   (B.MG_KERNEL_DR, lambda r: 432 + 168 * r)]:
        for nrhs in (1, 4):
            ms, by = B.mg_benchmark_kernel_nrhs(S.ctx, k, B.MG_FP32, nrhs, 2, 5)
            assert ms > 0 and by == per(nrhs) * 4 * vh
    S.close()


def test_solve_batch_several_lattices():
    """mg_solve_batch: three lattices of uneven size (one with odd coarse extents,
    so its coarsest solves take a launch of their own) and 18 right-hand sides in
    all (two groups of up to 16); every solution reaches the tolerance with the
    oracle's D of its lattice and agrees with that context's own mg_solve."""
    from paper_1011_2775_gb300 import binding as B
    from paper_1011_2775_gb300.solver import solve_batch
    specs = [((8, 8, 8, 8), (2, 2, 2, 2), 8, 9, 0.3, -0.1, 7501),
             ((8, 8, 8, 16), (4, 4, 4, 4), 12, 5, 1.0, -0.6, 7502),
             ((6, 4, 4, 8), (2, 2, 2, 2), 8, 4, 0.4, -0.15, 7503)]
    solvers, etas, ops = [], [], []
    for dims, blk, nv, nrhs, eps, m0, seed in specs:
        ape = 5 if eps >= 1.0 else 1
        U = I.make_gauge(dims, eps, ape, 0.5, seed)
        S = _solver(dims, U, 1.0, m0)
        S.set_params(levels=2, blocks=[blk], nv=[nv], seed=seed + 1, maxit_fine=2000)
        S.setup()
        solvers.append(S)
        etas.append(I.gaussian_source(dims, seed + 2, nrhs=nrhs))
        ops.append(WilsonClover(U, 1.0, m0))
    outs, infos = solve_batch(solvers, etas, 1e-10)
    for S, eta, psi, W, info in zip(solvers, etas, outs, ops, infos):
        for q in range(eta.shape[0]):
            res = eta[q].reshape(W.shape + (12,)) - W.D(psi[q].reshape(W.shape + (12,)))
            assert np.sqrt(norm2(res) / norm2(eta[q])) <= 1e-10
        assert info.true_residual <= 1e-10 and info.coarse_iterations[1] > 0
        own, _ = S.solve(eta, 1e-10, B.MG_MODE_MG)
        for q in range(eta.shape[0]):
            assert np.linalg.norm((psi[q] - own[q]).ravel()) / np.linalg.norm(own[q].ravel()) < 1e-7
    for S in solvers:
        S.close()


def test_solve_batch_rejects_bad_input():
    from paper_1011_2775_gb300 import binding as B
    dims = (4, 4, 4, 4)
    U = I.make_gauge(dims, 0.3, 0, 0.5, 7601)
    S = _solver(dims, U, 1.0, -0.1)
    eta = I.gaussian_source(dims, 7602)
    psi = np.zeros_like(eta)
    with pytest.raises(B.MGError) as e:          # no setup
        B.mg_solve_batch([S.ctx], [psi], [eta], [1], 1e-10)
    assert e.value.status == B.MG_ERR_STATE
    S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[8])
    S.setup()
    with pytest.raises(B.MGError) as e:          # the same context twice
        B.mg_solve_batch([S.ctx, S.ctx], [psi, psi.copy()], [eta, eta], [1, 1], 1e-10)
    assert e.value.status == B.MG_ERR_ARG
    S.close()


_FORCED_DR_SCRIPT = r"""
import sys
import numpy as np
from oracle.dirac import WilsonClover
from paper_1011_2775_gb300 import binding as B
from paper_1011_2775_gb300 import inputs as I
from paper_1011_2775_gb300.solver import Solver
dims, nrhs, w = tuple(int(v) for v in sys.argv[1].split(",")), 5, (0.45, 0.7, 1.25, 2.0)
U = I.make_gauge(dims, 0.4, 1, 0.5, 7011)
W = WilsonClover(U, 1.3, -0.2, weights=w, csw_t=0.6)
x = I.gaussian_source(dims, 7012, nrhs=nrhs)
with Solver(dims) as S:
    S.load_gauge(U)
    S.set_clover_aniso(w, 1.3, 0.6, -0.2)
    got = S.apply(B.MG_OP_DR, x, prec=B.MG_FP32, nrhs=nrhs)
worst = 0.0
for q in range(nrhs):
    ref = W.Dr(x[q].reshape(W.shape + (12,)) * W.even).reshape(x[q].shape)
    worst = max(worst, float(np.abs(got[q] - ref).max() / np.abs(ref).max()))
print(worst)
sys.exit(0 if worst <= 1e-5 else 1)
"""


@pytest.mark.parametrize("config,dims", [(203204, (6, 4, 8, 10)), (203208, (6, 4, 8, 10)), (206404, (6, 4, 8, 10)),
                                         (203214, (8, 16, 4, 16)), (206414, (8, 16, 4, 16))])
def test_shared_memory_multi_rhs_dslash_parity(tmp_path, config, dims):
    """The multi-RHS D_r with its two dslash launches forced (through the tuning
    cache) onto the shared-memory kernel -- S sites x NQ rhs lanes per CTA, 5
    right-hand sides so that the lanes hold different counts, four distinct
    hopping weights -- against the oracle per rhs: natural CTA order with a
    ragged last CTA on 6x4x8x10, tiled order (two slabs of 8 time slices,
    one or two blocks per plane) on 8x16x4x16."""
    import os
    import subprocess
    import sys
    torch = pytest.importorskip("torch")
    lib_built()
    gpu = torch.cuda.get_device_name(0).replace(" ", "_")
    cache = tmp_path / "tune.txt"
    d = " ".join(map(str, dims))
    lines = "".join(f"{k} {d} 5 1 {gpu} {config} 0\n" for k in ("dslash_ch", "dslash_xpay"))
    cache.write_text(lines)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, MGCLOVER_TUNE_CACHE=str(cache),
               PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", _FORCED_DR_SCRIPT, ",".join(map(str, dims))], cwd=root, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert cache.read_text() == lines   # the forced entries were used: the tuner appended nothing
