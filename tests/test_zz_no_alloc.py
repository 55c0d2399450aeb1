"""admm_iterate_static: the ADMM sweep for callers that may not allocate
device memory while they run (a pre-sized arena, a real-time loop, a thread
without the application's allocator).  It must give the same ADMM state,
residuals and step as admm_iterate, on two calls in a row, within the
tolerance the other parity tests use (1e-7 of each array's scale)."""
import ctypes as C

import numpy as np
import pytest

from paper_2310_13143_gb300 import binding, gridgen as gg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_sweep_matches_admm_iterate(precision):
    import torch

    grids = [gg.grid_30bus(), gg.geometric_grid(118, seed=7)]
    K = len(grids)
    ref = binding.Solver(grids, precision=precision)
    new = binding.Solver(grids, precision=precision)
    for s in (ref, new):
        s.build_qp(0.3, 2e4, True)
    opts = binding.default_admm()
    # device output buffers, allocated by the caller (the test), not by the entry point
    rs = torch.zeros(2 * K, dtype=torch.float64, device="cuda")
    iters = torch.zeros(K, dtype=torch.int32, device="cuda")
    for call in range(2):
        ref.admm_iterate(7, opts)
        st = binding.lib().admm_iterate_static(new.h, 7, C.byref(opts), C.c_void_p(rs.data_ptr()),
                                               C.c_void_p(iters.data_ptr()))
        assert st == 0, (call, st)
        torch.cuda.synchronize()
        assert iters.cpu().tolist() == [7] * K
        for k in range(K):
            a, b = ref.get_admm_state(k), new.get_admm_state(k)
            for key in ("x", "z", "lam", "xg", "zg", "lg", "zb", "nu", "ul"):
                scale = max(1.0, np.abs(a[key]).max())
                np.testing.assert_allclose(b[key], a[key], rtol=0, atol=1e-7 * scale, err_msg=f"{key} call {call}")
            ra = ref.get_residuals(k)
            got = rs.cpu().numpy()
            np.testing.assert_allclose([got[k], got[K + k]], [ra["r_inf"], ra["s_inf"]], rtol=1e-7, atol=1e-12)
            da, pa = ref.get_step(k)
            db, pb = new.get_step(k)
            np.testing.assert_allclose(db, da, rtol=0, atol=1e-7 * max(1.0, np.abs(da).max()))
            np.testing.assert_allclose(pb, pa, rtol=0, atol=1e-7 * max(1.0, np.abs(pa).max()))
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
    s.close()
