"""mg_apply_noalloc: the allocation-free fine-level operators.

For callers that cannot call cudaMalloc (their device memory belongs to
another allocator, or their loop cannot afford cudaMalloc's implicit
synchronisation).  Checked through the C ABI against mg_apply on two calls in
a row, so that the second call runs on the shared scratch array the first
one left behind.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from gpu_common import TOL32, TOL64, lib_built, rel
from paper_1011_2775_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    torch = pytest.importorskip("torch")
    lib_built()
    from paper_1011_2775_gb300.solver import Solver
    dims = (8, 8, 8, 8)
    S = Solver(dims)
    S.load_gauge(I.make_gauge(dims, 1.0, 2, 0.5, 4242))
    S.set_clover(1.0, -0.4)
    yield dims, S, torch
    S.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("op", ["DR", "D", "DP", "BR", "M", "MINV", "HOP"])
def test_noalloc_matches_mg_apply(solver, op, prec):
    from paper_1011_2775_gb300 import binding as B
    dims, S, torch = solver
    code = getattr(B, "MG_OP_" + op)
    tol = TOL64 if prec == B.MG_FP64 else TOL32
    for seed in (11, 12):  # two calls in a row
        x = I.gaussian_source(dims, seed)
        ref = S.apply(code, x, prec=prec)
        xd = torch.from_numpy(x).cuda()
        out = torch.full_like(xd, complex(7.0, -3.0))  # stale contents must not leak through
        B.mg_apply_noalloc(S.ctx, code, out, xd, prec)
        assert rel(out.cpu().numpy(), ref) <= tol


def test_noalloc_rejects_large_lattices():
    torch = pytest.importorskip("torch")
    lib_built()
    from paper_1011_2775_gb300 import binding as B
    from paper_1011_2775_gb300.solver import Solver
    dims = (16, 16, 16, 8)  # 32768 sites > 16384
    with Solver(dims) as S:
        S.load_gauge(I.unit_gauge(dims))
        S.set_clover(1.0, 0.1)
        x = torch.zeros((8, 16, 16, 16, 4, 3), dtype=torch.complex128, device="cuda")
        with pytest.raises(B.MGError) as e:
            B.mg_apply_noalloc(S.ctx, B.MG_OP_DR, torch.zeros_like(x), x, B.MG_FP64)
        assert e.value.status == B.MG_ERR_DIMS
