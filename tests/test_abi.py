"""The C-ABI library loads, exports every entry point include/*.h
declares, validates its inputs on the host, and fails loudly (no CPU
fallback) when no CUDA device is present.  No compute call needs a GPU here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2310_13143_gb300 import binding, gridgen as gg
from paper_2310_13143_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return binding.lib()


def _declared():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:acopf_status|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTED) == declared


def test_default_options(lib):
    o = binding.default_sqp()
    assert o.mu == 1e5 and o.tol == 1e-4 and o.admm.rho == 2e4 and o.admm.eps == 1e-4
    assert o.admm.max_iter == 20000 and o.admm.spin_limit > 0
    assert lib.acopf_status_string(4) == b"device barrier timed out"


def _create(grid, **kw):
    return binding.Solver(grid, **kw)


@pytest.mark.parametrize("mutate,msg", [
    (lambda g: g.bus_type.__setitem__(slice(None), 1), "reference bus"),
    (lambda g: g.f.__setitem__(0, g.nbus + 3), "invalid end buses"),
    (lambda g: g.vmin.__setitem__(0, 1.2), "voltage limits"),
    (lambda g: g.pmin.__setitem__(0, g.pmax[0] + 1), "invalid limits"),
    (lambda g: g.gbus.__setitem__(0, -1), "invalid bus"),
])
def test_invalid_grid_is_rejected_on_host(lib, mutate, msg):
    g = gg.grid_30bus()
    g = g.__class__(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in g.__dict__.items()})
    mutate(g)
    with pytest.raises(binding.AcopfError) as ei:
        _create(g)
    assert ei.value.status == 1 and msg in str(ei.value)


def test_isolated_bus_is_rejected(lib):
    g = gg.grid_30bus()
    keep = (g.f != 0) & (g.t != 0)
    g = g.__class__(**{**g.__dict__, "f": g.f[keep], "t": g.t[keep], "r": g.r[keep], "x": g.x[keep],
                       "b": g.b[keep], "rate": g.rate[keep], "angmin": g.angmin[keep], "angmax": g.angmax[keep],
                       "tap": g.tap[keep], "shift": g.shift[keep]})
    with pytest.raises(binding.AcopfError) as ei:
        _create(g)
    assert ei.value.status == 1


def test_no_device_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(binding.AcopfError) as ei:
        _create(gg.grid_30bus())
    assert ei.value.status == 3  # ECUDA: no CPU fallback


def test_null_arguments(lib):
    h = C.c_void_p()
    assert lib.acopf_create(None, 1, None, C.byref(h)) == 1
    assert lib.acopf_destroy(None) == 1
    assert lib.sqp_solve(None, None) == 1


def test_new_entry_points_validate_arguments_on_the_host(lib):
    """The projection, graph solve, autotune, warm-start scatter and network
    calls reject bad arguments before touching a device."""
    EINVAL = 1
    assert lib.acopf_project_linear(None, 0.5, 1e-6, 10, None, None) == EINVAL
    assert lib.sqp_solve_graph(None, None, 1) == EINVAL
    assert lib.acopf_autotune(None, None, 10, None, None) == EINVAL
    assert lib.acopf_set_warm_start_device(None, None, 0, 2e4, 1, 1, 1, 1) == EINVAL
    assert lib.acopf_set_allocator(None, binding.ALLOC_FN(), binding.FREE_FN(), None) == EINVAL
    h = C.c_void_p()
    bad_dims = (C.c_int32 * 3)(16, 12, 8)  # 12 is not a multiple of 8
    assert lib.acopf_mlp_create(bad_dims, 2, 64, 0, C.byref(h)) == EINVAL
    assert lib.acopf_mlp_create(None, 2, 64, 0, C.byref(h)) == EINVAL
    ok_dims = (C.c_int32 * 3)(16, 32, 8)
    assert lib.acopf_mlp_create(ok_dims, 2, 0, 0, C.byref(h)) == EINVAL
    assert lib.acopf_gemm_bf16(None, None, None, 8, 8, 8, 1, None, None) == EINVAL
    assert lib.acopf_mlp_train_step(None, None, None, None, 1, C.c_float(1e-3), None) == EINVAL


def test_allocator_binding_wants_both_callbacks():
    """Solver.set_allocator refuses one callback without the other before
    calling into the library."""
    s = binding.Solver.__new__(binding.Solver)
    s.h = None
    with pytest.raises(ValueError):
        s.set_allocator(alloc=lambda n: 0)
    with pytest.raises(ValueError):
        s.set_allocator(free=lambda p: None)
