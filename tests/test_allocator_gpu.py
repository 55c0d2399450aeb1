"""The handle's device memory served by a caller's allocator
(acopf_set_allocator), here torch's caching allocator: the state moves
intact, every later allocation and the final release go through the
callbacks, and a failing or wrong allocator leaves the handle as it was."""
import numpy as np
import pytest

from paper_2310_13143_gb300 import binding, gridgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


class Counting:
    """torch's caching allocator behind counters of live blocks."""

    def __init__(self):
        self.live = {}
        self.calls = 0

    def alloc(self, n):
        p = torch.cuda.caching_allocator_alloc(n, device=0)
        self.live[p] = n
        self.calls += 1
        return p

    def free(self, p):
        assert p in self.live, "released a block this allocator did not give"
        del self.live[p]
        torch.cuda.caching_allocator_delete(p)

    @property
    def bytes(self):
        return sum(self.live.values())


def _solve(s, opts):
    s.sqp_solve(opts)
    sol, res = s.get_solution(0), s.get_residuals(0)
    return sol, res


def _opts():
    return binding.default_sqp(tol=1e-4, max_sqp=40, admm=dict(rho=2e4, max_iter=1000, eps=1e-3, eps_dual=5e-3))


def test_state_moves_into_the_callers_allocator_and_back():
    g = gg.geometric_grid(118, seed=11)
    ref = binding.Solver(g, precision="mixed")
    want_sol, want_res = _solve(ref, _opts())
    ref.close()

    s = binding.Solver(g, precision="mixed")
    rng = np.random.default_rng(3)
    x0, _ = s.get_iterate(0)
    x1 = x0 + 1e-3 * rng.standard_normal(x0.size)
    s.set_iterate(0, x1)
    a = Counting()
    s.set_allocator(a.alloc, a.free)
    # every block of the model and state now comes from the callbacks
    L = g.nbranch
    assert a.calls >= 80 and a.bytes >= 4 * 4 * 14 * L
    got, _ = s.get_iterate(0)
    np.testing.assert_array_equal(got, x1)
    s.set_iterate(0, x0)
    sol, res = _solve(s, _opts())
    assert res["result_name"] == want_res["result_name"] == "converged"
    np.testing.assert_allclose(sol["obj"], want_sol["obj"], rtol=1e-12)
    np.testing.assert_allclose(sol["pg"], want_sol["pg"], rtol=0, atol=1e-10)
    # scratch of later calls is taken and returned through the callbacks
    before = a.calls
    live = a.bytes
    s.project_linear(rho=0.5, eps=1e-6, max_iter=200)
    assert a.calls > before and a.bytes == live
    # graph replay after the move captures the new addresses (from the flat start again)
    s.set_iterate(0, x0)
    s.sqp_solve_graph(_opts(), check_every=2)
    assert s.get_residuals(0)["result_name"] == "converged"
    np.testing.assert_allclose(s.get_solution(0)["obj"], want_sol["obj"], rtol=1e-6)
    # back to cudaMalloc: everything returned
    s.set_allocator()
    assert a.bytes == 0
    s.set_iterate(0, x0)
    sol2, _ = _solve(s, _opts())
    np.testing.assert_allclose(sol2["obj"], want_sol["obj"], rtol=1e-12)
    # and destroy releases through the allocator in force
    b = Counting()
    s.set_allocator(b.alloc, b.free)
    assert b.bytes > 0
    s.close()
    assert b.bytes == 0


def test_failing_or_wrong_allocator_leaves_the_handle_unchanged():
    g = gg.grid_30bus()
    s = binding.Solver(g, precision="fp64")
    want, _ = s.get_iterate(0)
    a = Counting()

    def no_memory(n):
        return None

    with pytest.raises(binding.AcopfError) as e:
        s.set_allocator(no_memory, a.free)
    assert e.value.status == 2  # ENOMEM

    # a block 16 bytes past an aligned one: rejected and released again
    offs = {}

    def misaligned(n):
        p = a.alloc(n + 256)
        offs[p + 16] = p
        return p + 16

    def release_misaligned(p):
        a.free(offs.pop(p))

    with pytest.raises(binding.AcopfError) as e:
        s.set_allocator(misaligned, release_misaligned)
    assert e.value.status == 1  # EINVAL
    assert a.bytes == 0 and not offs

    # host memory is not device memory
    host = np.zeros(1 << 20, dtype=np.uint8)
    given = []

    def host_block(n):
        assert n <= host.nbytes
        given.append(host.ctypes.data)
        return host.ctypes.data

    with pytest.raises(binding.AcopfError) as e:
        s.set_allocator(host_block, lambda p: given.remove(p))
    assert e.value.status == 1 and not given

    got, _ = s.get_iterate(0)
    np.testing.assert_array_equal(got, want)
    sol, res = _solve(s, binding.default_sqp())
    assert res["result_name"] == "converged"
    s.close()
