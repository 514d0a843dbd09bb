"""GPU parity of the fine-level kernels against the FP64 oracle, through the C ABI.

D, D_p, D_r, b_r, the clover term A, A^{-1} and the hopping term, in FP64
(relative error <= 1e-12) and FP32 (<= 1e-5), on lattices that span several
CTAs with a ragged tail, plus the 16^3x32 lattice of the solve benchmark.
"""
import numpy as np
import pytest

from gpu_common import TOL32, TOL64, lib_built, rel
from oracle.dirac import WilsonClover
from paper_1011_2775_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = [
    # dims, eps, ape, csw, m0, seed
    ((4, 4, 4, 4), 0.3, 0, 1.0, -0.1, 1001),
    ((6, 4, 8, 10), 0.4, 1, 1.3, -0.2, 7),     # half volume 960: ragged last CTA
    ((8, 8, 8, 8), 0.25, 2, 1.0, -0.35, 11),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "x".join(map(str, c[0])))
def setup(request):
    lib_built()
    from paper_1011_2775_gb300.solver import Solver
    dims, eps, ape, csw, m0, seed = request.param
    U = I.make_gauge(dims, eps, ape, 0.5, seed)
    W = WilsonClover(U, csw, m0)
    S = Solver(dims)
    S.load_gauge(U)
    S.set_clover(csw, m0)
    yield dims, W, S
    S.close()


def _oracle(W, op, v):
    from paper_1011_2775_gb300 import binding as B
    f = {B.MG_OP_D: W.D, B.MG_OP_DP: W.Dp, B.MG_OP_DR: lambda x: W.Dr(x * W.even), B.MG_OP_BR: W.b_r,
         B.MG_OP_M: W.M, B.MG_OP_MINV: W.Minv, B.MG_OP_HOP: W.hop}[op]
    return f(v)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("op", ["D", "DP", "DR", "BR", "M", "MINV", "HOP"])
def test_fine_operator_parity(setup, op, prec):
    from paper_1011_2775_gb300 import binding as B
    dims, W, S = setup
    code = getattr(B, "MG_OP_" + op)
    x = I.gaussian_source(dims, 99)
    got = S.apply(code, x, prec=prec)
    ref = _oracle(W, code, x.reshape(W.shape + (12,))).reshape(x.shape)
    assert rel(got, ref) <= (TOL64 if prec == 0 else TOL32)


def test_device_buffers_match_host(setup):
    torch = pytest.importorskip("torch")
    from paper_1011_2775_gb300 import binding as B
    dims, W, S = setup
    x = I.gaussian_source(dims, 5)
    host = S.apply(B.MG_OP_DR, x)
    dev = S.apply(B.MG_OP_DR, torch.from_numpy(x).cuda())
    assert np.array_equal(host, dev.cpu().numpy())


def test_full_size_dr_parity():
    """D_r in FP64 and FP32 on the 16^3x32 benchmark lattice."""
    lib_built()
    from paper_1011_2775_gb300 import binding as B
    from paper_1011_2775_gb300.solver import Solver
    dims = (16, 16, 16, 32)
    U = I.make_gauge(dims, 0.25, 0, 0.5, 2001)
    W = WilsonClover(U, 1.0, -0.35)
    x = I.gaussian_source(dims, 2002)
    ref = W.Dr(x.reshape(W.shape + (12,)) * W.even).reshape(x.shape)
    with Solver(dims) as S:
        S.load_gauge(U)
        S.set_clover(1.0, -0.35)
        assert rel(S.apply(B.MG_OP_DR, x, prec=B.MG_FP64), ref) <= TOL64
        assert rel(S.apply(B.MG_OP_DR, x, prec=B.MG_FP32), ref) <= TOL32
