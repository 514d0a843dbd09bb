"""The C ABI library: builds, loads, exports every declared entry point, and
fails cleanly (status code, no crash) where no GPU is present."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mgclover.h")


@pytest.fixture(scope="session")
def libpath():
    from paper_1011_2775_gb300 import build
    return build.build()


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"MG_API\s+[\w\s\*]+?\b(mg_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["mg_create", "mg_destroy", "mg_load_gauge", "mg_set_clover", "mg_set_params", "mg_setup",
              "mg_set_null_vectors", "mg_get_null_vectors", "mg_solve", "mg_apply", "mg_strerror"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for n in _declared():
        assert hasattr(lib, n), n
    from paper_1011_2775_gb300 import binding
    assert sorted(binding.EXPORTED) == _declared()


def test_host_only_calls(libpath):
    from paper_1011_2775_gb300 import binding as B
    assert B.mg_strerror(B.MG_ERR_GS_BREAKDOWN).startswith("block Gram-Schmidt")
    p = B.mg_default_params()
    assert p.levels == 2 and p.nv[0] == 24 and list(p.block[0]) == [4, 4, 4, 4]
    assert abs(p.tol_coarse - 0.1) < 1e-15 and p.nu_post == 4
    # null arguments are rejected before any device work
    assert B.lib().mg_default_params(None) == B.MG_ERR_ARG
    assert B.lib().mg_destroy(None) == B.MG_OK


def test_create_rejects_odd_dims(libpath):
    from paper_1011_2775_gb300 import binding as B
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(4, 4, 3, 4)
    assert B.lib().mg_create(ctypes.byref(h), d, 0, None) == B.MG_ERR_DIMS
    assert "even" in B.mg_last_error()


def test_no_gpu_fails_cleanly(libpath):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1011_2775_gb300 import binding as B
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(4, 4, 4, 4)
    assert B.lib().mg_create(ctypes.byref(h), d, 0, None) == B.MG_ERR_CUDA


def _enumerators():
    """Every `NAME = value` enumerator of the header's enums (values as written),
    and the members of enums whose values are implicit (counted from the last)."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for body in re.findall(r"enum\s+\w+\s*\{(.*?)\}", src, flags=re.S):
        nxt = 0
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            m = re.match(r"(MG_\w+)\s*(?:=\s*(-?\d+))?$", item)
            assert m, item
            val = int(m.group(2)) if m.group(2) is not None else nxt
            out[m.group(1)] = val
            nxt = val + 1
    return out


def test_binding_constants_match_the_header_enums():
    from paper_1011_2775_gb300 import binding
    enums = _enumerators()
    assert len(enums) > 30
    for name, val in enums.items():
        assert hasattr(binding, name), name
        assert getattr(binding, name) == val, name
