"""Setup reuse through the C ABI: save / load of a multigrid setup and rebuilding
it for a new mass from the current null vectors.

* A setup saved by one context and loaded by another (same lattice, gauge field,
  clover and mass) gives the same parameters, the same coarse links and the
  same solution.
* Foreign or truncated files and other lattices are rejected with a status.
* mg_update_mass: the hierarchy rebuilt for a lighter mass from the old null
  vectors solves the new system to ||eta - D psi|| / ||eta|| <= 1e-10 (the
  oracle's D at the new mass) in about as many iterations as a fresh setup.
"""
import numpy as np
import pytest

from gpu_common import lib_built
from oracle.dirac import WilsonClover, norm2
from paper_1011_2775_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 8, 16)


def _solver(U, m0):
    lib_built()
    from paper_1011_2775_gb300.solver import Solver
    S = Solver(DIMS)
    S.load_gauge(U)
    S.set_clover(1.0, m0)
    return S


def _res(W, psi, eta):
    r = eta.reshape(W.shape + (12,)) - W.D(psi.reshape(W.shape + (12,)))
    return float(np.sqrt(norm2(r) / norm2(eta)))


def test_save_load_roundtrip(tmp_path):
    from paper_1011_2775_gb300 import binding as B
    U = I.make_gauge(DIMS, 1.0, 5, 0.5, 8101)
    eta = I.gaussian_source(DIMS, 8102)
    path = str(tmp_path / "setup.bin")
    A = _solver(U, -0.6)
    A.set_params(levels=2, blocks=[(4, 4, 4, 4)], nv=[12], seed=8103, setup_iters=6)
    A.setup()
    A.save_setup(path)
    psi_a, info_a = A.solve(eta, 1e-10, B.MG_MODE_MG)
    Ya, Xa = A.coarse_links(1)
    Bs = _solver(U, -0.6)
    info = Bs.load_setup(path)
    assert info.vectors[0] == 12 and info.passes[0] == 0     # no inverse iteration
    assert Bs.params.nv[0] == 12 and Bs.params.setup_iters == 6 and tuple(Bs.params.block[0]) == (4, 4, 4, 4)
    Yb, Xb = Bs.coarse_links(1)
    assert np.array_equal(Ya, Yb) and np.array_equal(Xa, Xb)
    psi_b, info_b = Bs.solve(eta, 1e-10, B.MG_MODE_MG)
    assert info_b.outer_iterations == info_a.outer_iterations
    assert np.abs(psi_a - psi_b).max() <= 1e-13 * np.abs(psi_a).max()
    A.close()
    Bs.close()


def test_load_rejects_foreign_files(tmp_path):
    from paper_1011_2775_gb300 import binding as B
    U = I.make_gauge(DIMS, 0.3, 1, 0.5, 8201)
    S = _solver(U, -0.1)
    junk = tmp_path / "junk.bin"
    junk.write_bytes(b"not a setup" * 10)
    with pytest.raises(B.MGError) as e:
        S.load_setup(str(junk))
    assert e.value.status == B.MG_ERR_ARG
    with pytest.raises(B.MGError) as e:
        S.load_setup(str(tmp_path / "missing.bin"))
    assert e.value.status == B.MG_ERR_ARG
    S.set_params(levels=2, blocks=[(2, 2, 2, 2)], nv=[8])
    S.setup()
    good = str(tmp_path / "good.bin")
    S.save_setup(good)
    data = open(good, "rb").read()
    (tmp_path / "cut.bin").write_bytes(data[: len(data) // 2])
    with pytest.raises(B.MGError) as e:
        S.load_setup(str(tmp_path / "cut.bin"))
    assert e.value.status == B.MG_ERR_ARG
    from paper_1011_2775_gb300.solver import Solver
    other = Solver((8, 8, 8, 8))
    other.load_gauge(I.make_gauge((8, 8, 8, 8), 0.3, 1, 0.5, 8202))
    other.set_clover(1.0, -0.1)
    with pytest.raises(B.MGError) as e:
        other.load_setup(good)
    assert e.value.status == B.MG_ERR_DIMS
    other.close()
    S.close()


def test_update_mass_reuses_null_vectors():
    from paper_1011_2775_gb300 import binding as B
    U = I.make_gauge(DIMS, 1.0, 5, 0.5, 8301)
    eta = I.gaussian_source(DIMS, 8302)
    S = _solver(U, -0.5)
    S.set_params(levels=2, blocks=[(4, 4, 4, 4)], nv=[12], seed=8303, maxit_fine=2000)
    S.setup()
    info = S.update_mass(-0.6)
    assert info.passes[0] == 0
    psi, si = S.solve(eta, 1e-10, B.MG_MODE_MG)
    assert _res(WilsonClover(U, 1.0, -0.6), psi, eta) <= 1e-10
    F = _solver(U, -0.6)
    F.set_params(levels=2, blocks=[(4, 4, 4, 4)], nv=[12], seed=8303, maxit_fine=2000)
    F.setup()
    _, fi = F.solve(eta, 1e-10, B.MG_MODE_MG)
    assert si.outer_iterations <= 1.5 * fi.outer_iterations + 3
    S.close()
    F.close()


def test_adaptive_setup_improves_a_weak_setup():
    """mg_adapt_setup: after a deliberately weak setup (one inverse-iteration
    pass per vector), one adaptive pass -- inverse subspace iteration of the
    null vectors with the current solver, then a rebuild -- lowers the outer
    iteration count, and the solve still reaches 1e-10 with the oracle's D."""
    from paper_1011_2775_gb300 import binding as B
    U = I.make_gauge(DIMS, 1.0, 5, 0.5, 8401)
    W = WilsonClover(U, 1.0, -0.6)
    eta = I.gaussian_source(DIMS, 8402)
    S = _solver(U, -0.6)
    S.set_params(levels=2, blocks=[(4, 4, 4, 4)], nv=[12], seed=8403, setup_iters=1, maxit_fine=4000)
    S.setup()
    _, weak = S.solve(eta, 1e-10, B.MG_MODE_MG)
    info = S.adapt_setup(passes=1, relax=3)
    assert info.vectors[0] == 12
    psi, adapted = S.solve(eta, 1e-10, B.MG_MODE_MG)
    assert _res(W, psi, eta) <= 1e-10
    assert adapted.outer_iterations < weak.outer_iterations
    S.close()


def test_adaptive_setup_three_levels():
    """On three levels the adaptive pass refines both transfers (the level-1
    vectors iterated with the level-1 cycle); the solve still reaches 1e-10 and
    needs fewer outer iterations than the weak setup it started from."""
    from paper_1011_2775_gb300 import binding as B
    U = I.make_gauge(DIMS, 1.0, 5, 0.5, 8501)
    W = WilsonClover(U, 1.0, -0.6)
    eta = I.gaussian_source(DIMS, 8502)
    S = _solver(U, -0.6)
    S.set_params(levels=3, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nv=[8, 8], seed=8503, setup_iters=1,
                 maxit_fine=4000)
    S.setup()
    _, weak = S.solve(eta, 1e-10, B.MG_MODE_MG)
    S.adapt_setup(passes=1, relax=3, transfers=0)
    psi, adapted = S.solve(eta, 1e-10, B.MG_MODE_MG)
    assert _res(W, psi, eta) <= 1e-10
    assert adapted.outer_iterations < weak.outer_iterations
    S.close()


@pytest.mark.parametrize("levels", [2, 3])
def test_adaptive_setup_keeps_a_good_setup(levels):
    """The refinement must not undo a converged setup: the inverse iteration
    keeps the low modes the coarse space already holds (replacing v by the
    error propagator's (1 - M D_p) v would remove exactly those)."""
    from paper_1011_2775_gb300 import binding as B
    U = I.make_gauge(DIMS, 1.0, 5, 0.5, 8601)
    W = WilsonClover(U, 1.0, -0.6)
    eta = I.gaussian_source(DIMS, 8602)
    S = _solver(U, -0.6)
    blocks = [(4, 4, 4, 4)] if levels == 2 else [(2, 2, 2, 2), (2, 2, 2, 2)]
    S.set_params(levels=levels, blocks=blocks, nv=[12] if levels == 2 else [8, 8], seed=8603, setup_iters=6,
                 maxit_fine=4000)
    S.setup()
    _, good = S.solve(eta, 1e-10, B.MG_MODE_MG)
    S.adapt_setup(passes=1, relax=2, transfers=0)
    psi, adapted = S.solve(eta, 1e-10, B.MG_MODE_MG)
    assert _res(W, psi, eta) <= 1e-10
    assert adapted.outer_iterations <= good.outer_iterations + 2
    S.close()
