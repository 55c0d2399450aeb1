"""admm_iterate_static: the ADMM sweep for callers that may not allocate
device memory while they run (a pre-sized arena, a real-time loop, a thread
without the application's allocator).  It must give the same ADMM state,
residuals and step as admm_iterate, on two calls in a row, within the
tolerance the other parity tests use (1e-7 of each array's scale), and it
must allocate nothing while doing so."""
import ctypes as C

import numpy as np
import pytest

from paper_2310_13143_gb300 import binding, gridgen as gg

pytestmark = pytest.mark.gpu


class Counting:
    """torch's caching allocator behind a call counter."""

    def __init__(self, torch):
        self.torch = torch
        self.calls = 0

    def alloc(self, n):
        self.calls += 1
        return self.torch.cuda.caching_allocator_alloc(n, device=0)

    def free(self, p):
        self.calls += 1
        self.torch.cuda.caching_allocator_delete(p)


def _static(s, n, opts, rs, iters):
    return binding.lib().admm_iterate_static(s.h, n, C.byref(opts), C.c_void_p(rs.data_ptr()),
                                             C.c_void_p(iters.data_ptr()))


def _same(ref, new, k, rs, K):
    a, b = ref.get_admm_state(k), new.get_admm_state(k)
    for key in ("x", "z", "lam", "xg", "zg", "lg", "zb", "nu", "ul"):
        scale = max(1.0, np.abs(a[key]).max())
        np.testing.assert_allclose(b[key], a[key], rtol=0, atol=1e-7 * scale, err_msg=key)
    ra = ref.get_residuals(k)
    got = rs.cpu().numpy()
    np.testing.assert_allclose([got[k], got[K + k]], [ra["r_inf"], ra["s_inf"]], rtol=1e-7, atol=1e-12)
    # the handle's own residual record follows the static sweep as well
    rb = new.get_residuals(k)
    np.testing.assert_allclose([rb["r_inf"], rb["s_inf"]], [ra["r_inf"], ra["s_inf"]], rtol=1e-7, atol=1e-12)
    da, pa = ref.get_step(k)
    db, pb = new.get_step(k)
    np.testing.assert_allclose(db, da, rtol=0, atol=1e-7 * max(1.0, np.abs(da).max()))
    np.testing.assert_allclose(pb, pa, rtol=0, atol=1e-7 * max(1.0, np.abs(pa).max()))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_sweep_matches_admm_iterate(precision):
    import torch

    grids = [gg.grid_30bus(), gg.geometric_grid(118, seed=7)]
    K = len(grids)
    ref = binding.Solver(grids, precision=precision)
    new = binding.Solver(grids, precision=precision)
    for s in (ref, new):
        s.build_qp(0.3, 2e4, True)
    # the handle's later allocations go through a counter: the static sweep must make none
    cnt = Counting(torch)
    new.set_allocator(cnt.alloc, cnt.free)
    opts = binding.default_admm()
    # device output buffers, allocated by the caller (the test), not by the entry point
    rs = torch.zeros(2 * K, dtype=torch.float64, device="cuda")
    iters = torch.zeros(K, dtype=torch.int32, device="cuda")
    for call in range(2):
        ref.admm_iterate(7, opts)
        torch.cuda.synchronize()
        calls0 = cnt.calls
        free0 = torch.cuda.mem_get_info()[0]
        st = _static(new, 7, opts, rs, iters)
        torch.cuda.synchronize()
        assert st == 0, (call, st)
        assert cnt.calls == calls0, "the static sweep called the handle's allocator"
        if call > 0:  # after the first call's one-time set-up, device memory is untouched
            assert torch.cuda.mem_get_info()[0] == free0
        assert iters.cpu().tolist() == [7] * K
        for k in range(K):
            _same(ref, new, k, rs, K)
    ref.close()
    new.close()


def test_static_sweep_after_a_solved_qp_skips_the_same_instances():
    """After admm_solve_qp, instances whose residual test passed are skipped by
    admm_iterate; the static sweep starts from the same finished flags."""
    import torch

    grids = [gg.two_bus(lossless=False, rate=2.0), gg.grid_30bus()]
    K = len(grids)
    # iterations each instance's QP needs, then a budget between the two
    probe = binding.Solver(grids, precision="fp64")
    probe.admm_solve_qp(0.3, binding.default_admm(eps=1e-4, max_iter=20000))
    need = [probe.get_residuals(k)["admm_iter"] for k in range(K)]
    probe.close()
    assert abs(need[0] - need[1]) >= 4, need
    budget = (need[0] + need[1]) // 2
    ref = binding.Solver(grids, precision="fp64")
    new = binding.Solver(grids, precision="fp64")
    solve = binding.default_admm(eps=1e-4, max_iter=budget)
    for s in (ref, new):
        s.admm_solve_qp(0.3, solve)
    done = [ref.get_residuals(k)["admm_iter"] < budget for k in range(K)]
    assert sorted(done) == [False, True], (need, budget, done)
    rs = torch.zeros(2 * K, dtype=torch.float64, device="cuda")
    iters = torch.zeros(K, dtype=torch.int32, device="cuda")
    opts = binding.default_admm()
    ref.admm_iterate(5, opts)
    assert _static(new, 5, opts, rs, iters) == 0
    torch.cuda.synchronize()
    for k in range(K):
        a, b = ref.get_admm_state(k), new.get_admm_state(k)
        for key in ("x", "z", "lam", "zb", "nu"):
            np.testing.assert_allclose(b[key], a[key], rtol=0, atol=1e-7 * max(1.0, np.abs(a[key]).max()),
                                       err_msg=f"{key} instance {k}")
    ref.close()
    new.close()


def test_static_sweep_rejects_bad_arguments():
    s = binding.Solver(gg.grid_30bus())
    opts = binding.default_admm()
    # before any QP is built
    assert binding.lib().admm_iterate_static(s.h, 3, C.byref(opts), C.c_void_p(1), C.c_void_p(1)) == 5
    s.build_qp(0.3, 2e4, True)
    assert binding.lib().admm_iterate_static(s.h, 3, C.byref(opts), None, None) == 1
    assert binding.lib().admm_iterate_static(s.h, 0, C.byref(opts), C.c_void_p(1), C.c_void_p(1)) == 1
    bad = binding.default_admm(rho=-1.0)
    assert binding.lib().admm_iterate_static(s.h, 3, C.byref(bad), C.c_void_p(1), C.c_void_p(1)) == 1
    s.close()


def test_static_sweep_rejects_more_instances_than_the_fixed_array_holds():
    n = 4097  # ACOPF_STATIC_MAX_INSTANCES + 1
    s = binding.Solver([gg.two_bus()] * n)
    opts = binding.default_admm()
    assert binding.lib().admm_iterate_static(s.h, 1, C.byref(opts), C.c_void_p(1), C.c_void_p(1)) == 1
    s.close()
