"""GPU parity of the learned warm start: the tensor-core product against an
FP64 product of the same bfloat16 operands, one training step (forward,
gradients, Adam) against the FP64 oracle (oracle/mlp.py), the device
warm-start scatter against the layout it is defined by, and the gain of a
trained network over cold starts on held-out scenarios."""
import math

import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2310_13143_gb300 import binding, gridgen as gg, warmstart as ws

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24  # unit roundoff of FP32


def _bf16(rng, shape, scale=1.0):
    a = torch.from_numpy((scale * rng.standard_normal(shape)).astype(np.float32)).to(torch.bfloat16)
    return a.cuda(), a.float().double().numpy()


@pytest.mark.parametrize("M,N,K,splits", [(128, 128, 64, 1), (256, 256, 128, 1), (200, 136, 200, 1),
                                          (128, 384, 1024, 4), (300, 40, 4000, 8), (1, 8, 8, 1), (130, 264, 520, 3)])
def test_tensor_core_gemm_matches_fp64(M, N, K, splits):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A, An = _bf16(rng, (M, K))
    B, Bn = _bf16(rng, (N, K))
    Cd = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    binding.gemm_bf16(A.data_ptr(), B.data_ptr(), Cd.data_ptr(), M, N, K, splits)
    C = Cd.cpu().double().numpy()
    ref = An @ Bn.T
    # products of bfloat16 values are exact in FP32; K FP32 additions (plus the
    # split sums) err by at most about (K + splits) u sum |a||b|
    bound = (K + splits + 2) * U32 * (np.abs(An) @ np.abs(Bn).T) + 1e-30
    assert np.all(np.isfinite(C))
    assert np.all(np.abs(C - ref) <= bound)


def _net_params(rng, dims):
    flat = gg.mlp_init(dims, seed=int(rng.integers(1 << 30)))
    # non-zero biases so that the bias paths are exercised
    params, o = [], 0
    for i in range(len(dims) - 1):
        w = flat[o:o + dims[i] * dims[i + 1]].reshape(dims[i + 1], dims[i]).astype(np.float64)
        o += dims[i] * dims[i + 1]
        b = 0.1 * rng.standard_normal(dims[i + 1])
        flat[o:o + dims[i + 1]] = b
        o += dims[i + 1]
        params.append((w, b.astype(np.float32).astype(np.float64)))
    return flat, params


def _close(gpu, ref, rel):
    scale = np.max(np.abs(ref)) + 1e-30
    return np.max(np.abs(gpu - ref)) <= rel * scale


def test_train_step_matches_oracle():
    rng = np.random.default_rng(11)
    dims = [24, 64, 48, 64, 40]
    n, rows, lr = 100, 64, 1e-3
    X = (2.0 + rng.standard_normal((n, dims[0]))).astype(np.float32)
    X[:, 3] = 0.5  # a constant column
    T = (rng.standard_normal((n, dims[-1])) * 3.0 + 1.0).astype(np.float32)
    flat, params = _net_params(rng, dims)
    net = binding.Mlp(dims, max_batch=rows)
    net.set_params(flat)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    net.fit_standardiser(Xd.data_ptr(), Td.data_ptr(), n)
    mu_x, sd_x, mu_y, sd_y = net.get_standardiser()
    omx, osx = omlp.standardiser(X.astype(np.float64))
    omy, osy = omlp.standardiser(T.astype(np.float64))
    np.testing.assert_allclose(mu_x, omx, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(sd_x, osx, rtol=1e-6)
    np.testing.assert_allclose(mu_y, omy, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(sd_y, osy, rtol=1e-6)
    assert sd_x[3] == 1.0

    idx = rng.choice(n, size=rows, replace=False).astype(np.int32)
    idxd = torch.from_numpy(idx).cuda()
    loss = torch.zeros(1, device="cuda")
    net.train_step(Xd.data_ptr(), Td.data_ptr(), idxd.data_ptr(), rows, lr, loss.data_ptr())
    net.sync()

    # oracle with the GPU's (FP32) statistics and the same bfloat16 rounding points
    A0 = (X[idx].astype(np.float64) - mu_x) / sd_x
    Tn = (T[idx].astype(np.float64) - mu_y) / sd_y
    Y, cache = omlp.forward(params, A0, q=omlp.bf16_round)
    oloss, dY = omlp.mse(Y, Tn)
    grads = omlp.backward(params, cache, dY, q=omlp.bf16_round)
    assert abs(loss.item() - oloss) <= 1e-3 * oloss

    g = net.get_grads()
    o = 0
    for l, (gw, gb) in enumerate(grads):
        nw = gw.size
        gpu_w = g[o:o + nw].reshape(gw.shape); o += nw
        gpu_b = g[o:o + gb.size]; o += gb.size
        # bfloat16 storage of the back-propagated gradients (unit roundoff
        # 2^-9) bounds the agreement; a rounding that falls differently on the
        # two sides moves one term by 2^-8 relative
        assert _close(gpu_w, gw, 2 ** -7), l
        assert _close(gpu_b, gb, 2 ** -7), l
        assert np.median(np.abs(gpu_w - gw)) <= 2 ** -9 * np.max(np.abs(gw)), l

    # Adam's first step: W - lr g / (|g| + eps) where the gradient is not tiny
    p_new = net.get_params()
    o = 0
    for l, ((w, b), (gw, gb)) in enumerate(zip(params, grads)):
        for ref_p, ref_g in ((w, gw), (b, gb)):
            cnt = ref_p.size
            got = p_new[o:o + cnt].reshape(ref_p.shape); o += cnt
            want, _, _ = omlp.adam_step(ref_p.astype(np.float32).astype(np.float64), ref_g, 0 * ref_g, 0 * ref_g,
                                        1, lr)
            big = np.abs(ref_g) > 1e-2 * np.max(np.abs(ref_g))
            np.testing.assert_allclose(got[big], want[big], atol=1e-6 + 1e-3 * lr)
            assert np.all(np.abs(got - ref_p) <= lr * (1 + 1e-3) + 1e-6)
    net.close()


def test_forward_in_chunks_matches_oracle():
    rng = np.random.default_rng(5)
    dims = [16, 32, 32, 24]
    rows = 300  # three chunks of 128, the last one ragged
    X = rng.standard_normal((rows, dims[0])).astype(np.float32)
    flat, params = _net_params(rng, dims)
    net = binding.Mlp(dims, max_batch=128)
    net.set_params(flat)
    Xd = torch.from_numpy(X).cuda()
    Td = torch.zeros((rows, dims[-1]), device="cuda")
    net.fit_standardiser(Xd.data_ptr(), Td.data_ptr(), rows)
    mu_x, sd_x, mu_y, sd_y = net.get_standardiser()
    Yd = torch.zeros((rows, dims[-1]), device="cuda")
    net.forward(Xd.data_ptr(), rows, Yd.data_ptr())
    Y, _ = omlp.forward(params, (X.astype(np.float64) - mu_x) / sd_x, q=omlp.bf16_round)
    Y = Y * sd_y + mu_y
    assert _close(Yd.cpu().double().numpy(), Y, 2 ** -7)
    net.close()


def test_warm_start_scatter_follows_its_layout():
    g = gg.grid_30bus()
    grids = gg.scenarios_cholesky(g, 3, seed=77)
    B, L, G = g.nbus, g.nbranch, g.ngen
    width = ws.output_width(g)
    ld = width + 5
    rng = np.random.default_rng(2)
    P = rng.standard_normal((3, ld)).astype(np.float32) * 0.05
    P[:, 2 * G:2 * G + B] += 1.0                     # w near 1
    P[0, 2 * G] = 2.0                                # above vmax^2: clamped
    P[:, 2 * G + 2 * B:2 * G + 2 * B + L] += 1.0     # wR near 1
    for prec in ("fp64", "mixed"):
        s = binding.Solver(grids, precision=prec)
        Pd = torch.from_numpy(P).cuda()
        s.set_warm_start_device(Pd.data_ptr(), ld, base_rho=2e4)
        torch.cuda.synchronize()
        for k in range(3):
            row = P[k].astype(np.float64)
            x, pi = s.get_iterate(k)
            want = row[:2 * G + 2 * B + 2 * L].copy()
            want[:G] = np.clip(want[:G], g.pmin, g.pmax)
            want[G:2 * G] = np.clip(want[G:2 * G], g.qmin, g.qmax)
            want[2 * G:2 * G + B] = np.clip(want[2 * G:2 * G + B], g.vmin ** 2, g.vmax ** 2)
            ref = np.flatnonzero(g.bus_type == 3)
            want[2 * G + B + ref] = 0.0
            np.testing.assert_allclose(x, want, rtol=1e-7, atol=1e-7)
            o = 2 * G + 2 * B + 2 * L
            np.testing.assert_allclose(pi, row[o:o + 4 * L], rtol=1e-7, atol=1e-7)
            o += 4 * L
            st = s.get_admm_state(k)
            tol = 1e-6 if prec == "mixed" else 1e-12
            np.testing.assert_allclose(st["lam"].ravel(), row[o:o + 8 * L], rtol=tol, atol=tol)
            np.testing.assert_allclose(st["lg"].ravel(), row[o + 8 * L:o + 8 * L + 2 * G], rtol=tol, atol=tol)
        s.close()


def test_learned_warm_start_beats_cold_start_on_held_out_scenarios():
    """Train on cold solves of 384 sampled load scenarios of a 118-bus grid,
    then solve 32 held-out scenarios from the network's prediction.  Every
    warm-started solve must converge to the same tolerance and objective as
    its cold solve, with fewer ADMM iterations on average."""
    base = gg.geometric_grid(118, seed=11)
    scen = gg.scenarios_cholesky(base, 384 + 32, seed=901)
    opts = binding.default_sqp(tol=1e-4, max_sqp=40, admm=dict(rho=2e4, max_iter=1000, eps=1e-3, eps_dual=5e-3))
    T, conv, iters, objs = ws.solve_targets(scen, opts, precision="mixed")
    assert conv.all()
    train_s, test_s = scen[:384], scen[384:]
    X = ws.loads_matrix(scen)
    dims = ws.dims_for(base, hidden=(256, 256, 256))
    net = binding.Mlp(dims, max_batch=128)
    net.set_params(gg.mlp_init(dims, seed=3))
    Xd = torch.from_numpy(X).cuda()
    Td = torch.from_numpy(T).cuda()
    net.fit_standardiser(Xd.data_ptr(), Td.data_ptr(), 384)
    losses = ws.train(net, Xd, Td, 384, steps=600, batch=128, lr=1e-3, seed=4)
    assert losses[-20:].mean() < 0.2 * losses[:5].mean()
    s = binding.Solver(test_s, precision="mixed")
    res, warm_obj, failed = ws.solve_warm_with_fallback(s, test_s, net, Xd[384:], opts)
    s.close()
    net.close()
    assert len(failed) <= 2  # the fallback is the exception
    assert all(ws.converged(r) for r in res)
    warm_iters = [r["admm_iter"] for k, r in enumerate(res) if k not in failed]
    cold_iters = iters[384:]
    np.testing.assert_allclose(warm_obj, objs[384:], rtol=1e-5)
    assert np.mean(warm_iters) < 0.8 * np.mean(cold_iters), (np.mean(warm_iters), np.mean(cold_iters))


def test_learned_penalties_on_held_out_scenarios():
    """Form (4)'s per-component penalties: after the network learns x0, pi
    and lambda, each training scenario is solved from its prediction under a
    few candidate penalty factors (branches, generators); the fastest
    converging pair becomes the target of the penalty outputs, and the
    network is fine-tuned.  On held-out scenarios the solve with the
    predicted penalties must converge like the one without them, and its
    ADMM iteration count is compared with that of x0/pi/lambda alone."""
    base = gg.geometric_grid(118, seed=11)
    scen = gg.scenarios_cholesky(base, 384 + 32, seed=901)
    opts = binding.default_sqp(tol=1e-4, max_sqp=40, admm=dict(rho=2e4, max_iter=1000, eps=1e-3, eps_dual=5e-3))
    T, conv, iters, objs = ws.solve_targets(scen, opts, precision="mixed")
    assert conv.all()
    train_s, test_s = scen[:384], scen[384:]
    X = ws.loads_matrix(scen)
    dims = ws.dims_for(base, hidden=(256, 256, 256))
    net = binding.Mlp(dims, max_batch=128)
    net.set_params(gg.mlp_init(dims, seed=3))
    Xd = torch.from_numpy(X).cuda()
    Td = torch.from_numpy(T).cuda()
    net.fit_standardiser(Xd.data_ptr(), Td.data_ptr(), 384)
    ws.train(net, Xd, Td, 384, steps=600, batch=128, lr=1e-3, seed=4)
    pick, cand = ws.rho_targets(train_s, net, Xd, T, opts)
    o0, o1, o2 = ws.rho_columns(base)
    assert np.isfinite(cand[:, 0]).mean() > 0.95  # the base penalty converges from the prediction
    Td = torch.from_numpy(T).cuda()
    net.fit_standardiser(Xd.data_ptr(), Td.data_ptr(), 384)
    ws.train(net, Xd, Td, 384, steps=300, batch=128, lr=3e-4, seed=5)
    out = {}
    for use_rho in (False, True):
        s = binding.Solver(test_s, precision="mixed")
        res, obj, failed = ws.solve_warm_with_fallback(s, test_s, net, Xd[384:], opts, use_rho=use_rho)
        s.close()
        assert all(ws.converged(r) for r in res)
        np.testing.assert_allclose(obj, objs[384:], rtol=1e-5)
        out[use_rho] = (np.mean([r["admm_iter"] for r in res]), len(failed))
    net.close()
    chosen = np.bincount(pick, minlength=len(ws.RHO_CHOICES))
    print("penalty choices", dict(zip(map(str, ws.RHO_CHOICES), chosen.tolist())),
          "ADMM iterations without / with the learned penalties", out[False], out[True])
    assert out[True][1] <= 4  # the cold fallback stays the exception
    # the learned penalties cut the ADMM iterations of the warm-started solves
    assert out[True][0] <= 0.9 * out[False][0], out
