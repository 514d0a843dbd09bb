"""Host-side pieces of bench.py that need no GPU."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1011_2775_gb300 import inputs as I  # noqa: E402


def test_big_fields_equal_the_serial_fields():
    """The generation split into blocks of time slices over spawned processes
    (uneven blocks, blocks of one slice, more processes than slices) gives
    bitwise the fields of make_gauge, keyed by their spec."""
    specs = [((4, 4, 4, 4), 0.25, 1, 0.5, 3), ((4, 2, 4, 10), 1.0, 3, 0.5, 5), ((4, 4, 4, 4), 0.25, 1, 0.5, 3),
             ((2, 4, 2, 6), 0.4, 0, 0.5, 9)]
    for nproc in (3, 4, 16):
        got = bench.big_fields(specs, nproc)
        assert len(got) == 3
        for sp in specs:
            assert np.array_equal(got[sp], I.make_gauge(*sp)), (nproc, sp)


def test_extra_field_specs_cover_the_extra_configurations():
    specs = bench.extra_field_specs()
    assert len(specs) == len(set(specs)) == len(bench.MULTI) + 2
    assert {sp[0] for sp in specs} == {d for d, _, _ in bench.MULTI} | {bench.CONFIG3_DIMS}


def test_extra_configs_run_at_one_gpu_with_pregenerated_fields(monkeypatch):
    """run_extra_configs hands run_multi and run_config3 the fields of their
    specs, at world size 1 only, and honours --no-multi / --no-config3."""
    from types import SimpleNamespace
    calls = {}
    monkeypatch.setattr(bench, "big_fields", lambda specs: {sp: sp for sp in specs})

    def multi(dev, seq, pre):
        calls["multi"] = sorted(sp[0] for sp in pre if sp[0] != bench.CONFIG3_DIMS)
        return {"ok": 1}

    def config3(dev, pre):
        calls["config3"] = sorted(sp[1] for sp in pre if sp[0] == bench.CONFIG3_DIMS)
        return {"ok": 3}

    monkeypatch.setattr(bench, "run_multi", multi)
    monkeypatch.setattr(bench, "run_config3", config3)
    args = SimpleNamespace(no_multi=False, no_config3=False, multi_sequential=False)
    r = {"extra": {}}
    bench.run_extra_configs(args, SimpleNamespace(world=1, local=0), r)
    assert r["extra"] == {"multi_lattice": {"ok": 1}, "config3_24x64": {"ok": 3}}
    assert calls["multi"] == sorted(d for d, _, _ in bench.MULTI)
    assert calls["config3"] == sorted((bench.EPS, bench.ROUGH_EPS))
    r = {"extra": {}}
    bench.run_extra_configs(args, SimpleNamespace(world=2, local=0), r)
    assert r["extra"] == {}
    calls.clear()
    r = {"extra": {}}
    bench.run_extra_configs(SimpleNamespace(no_multi=True, no_config3=False, multi_sequential=False),
                            SimpleNamespace(world=1, local=0), r)
    assert list(r["extra"]) == ["config3_24x64"] and "multi" not in calls
