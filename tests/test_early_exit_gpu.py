"""GPU parity of the learned early exit: features and the network's forward pass,
gradients and Adam steps against the FP64 reference in oracle/mlp.py."""
import numpy as np
import pytest

import oracle.mlp as M
import oracle.oracle as O
from paper_2308_02329_gb300 import chym, inputs
from tests.helpers import make_case, oracle_params, oracle_schedule

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    chym.lib()
    return t


def bf16_round(a):
    """Round to BF16 (nearest-even) and back, as the network's forward pass does."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("N,D,graph,prec", [(50, 3, "sk", chym.PREC_BF16X2), (33, 4, "gauss", chym.PREC_FP64),
                                            (150, 2, "sparse", chym.PREC_BF16X2), (20, 1, "sk", chym.PREC_FP32)])
def test_features_match_reference(torch, N, D, graph, prec):
    n_h, reps = 2, 5
    J, eps, h, seeds = make_case(N, D, n_h, reps, 31, graph)
    ctx = chym.Context(J, D, chym.J_REAL if graph == "gauss" else chym.J_PM1)
    prm = chym.Params(eps=eps, prec=prec)
    sch = chym.Schedule(1, 100, 400)
    ctx.run(prm, h, seeds, 30, sch)
    dt = torch.float64 if prec == chym.PREC_FP64 else torch.float32
    snap = torch.empty(n_h * reps * N * D, dtype=dt, device="cuda")
    ctx.copy_state_device(snap.data_ptr())
    Xs, _ = ctx.get_state()
    ctx.run(prm, None, None, 30, sch, n_runs=len(seeds))
    X, _ = ctx.get_state()
    F = torch.empty(n_h * reps, 24, dtype=torch.float32, device="cuda")
    ctx.features_device(snap.data_ptr(), 60 / 400, F.data_ptr())
    torch.cuda.synchronize()
    F = F.cpu().numpy().astype(np.float64)
    hr = inputs.h_per_run(h, reps)
    for r in range(len(seeds)):
        ref = M.features(J, X[r], Xs[r], hr[r], 60 / 400)
        np.testing.assert_allclose(F[r, :12], ref[:12], rtol=1e-5, atol=1e-6)   # order statistics
        if graph != "gauss":
            assert F[r, 12] == pytest.approx(ref[12], abs=1e-6)                  # integer energies
            assert F[r, 13] == pytest.approx(ref[13], abs=1e-6)
        np.testing.assert_allclose(F[r, 12:], ref[12:], rtol=1e-4, atol=1e-5)
    ctx.close()


def _net_case(rng):
    theta = rng.standard_normal(M.N_PARAMS).astype(np.float32) * 0.3
    mean = rng.standard_normal(24).astype(np.float32) * 0.2
    istd = rng.uniform(0.5, 2.0, 24).astype(np.float32)
    return theta, mean, istd


def test_forward_matches_reference(torch):
    rng = np.random.default_rng(0)
    theta, mean, istd = _net_case(rng)
    net = chym.MLP(seed=3, max_batch=512)
    net.set_params(theta, mean, istd)
    Fh = rng.standard_normal((300, 24)).astype(np.float32)
    F = torch.from_numpy(Fh).cuda()
    out = torch.empty(300, dtype=torch.float32, device="cuda")
    net.forward_device(F.data_ptr(), 300, out.data_ptr())
    torch.cuda.synchronize()
    ref, _ = M.forward(bf16_round(theta), Fh.astype(np.float64), mean.astype(np.float64),
                       istd.astype(np.float64))
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-4, atol=1e-4)
    net.close()


def test_gradient_matches_reference(torch):
    """BF16 forward, FP32 backward: per tensor within 1e-2 relative and cosine > 0.999
    against the FP64 gradient; against the FP64 gradient of the BF16-rounded weights
    within 1e-3."""
    rng = np.random.default_rng(1)
    theta, mean, istd = _net_case(rng)
    B = 200
    Fh = rng.standard_normal((B, 24)).astype(np.float32)
    yh = rng.integers(0, 2, B).astype(np.float32)
    net = chym.MLP(seed=3, max_batch=512)
    net.set_params(theta, mean, istd)
    F, y = torch.from_numpy(Fh).cuda(), torch.from_numpy(yh).cuda()
    g = torch.empty(M.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    net.grad_device(F.data_ptr(), y.data_ptr(), B, g.data_ptr(), loss.data_ptr())
    torch.cuda.synchronize()
    gg = g.cpu().numpy().astype(np.float64)
    args = (Fh.astype(np.float64), yh.astype(np.float64), mean.astype(np.float64), istd.astype(np.float64))
    ref64 = M.grad(theta.astype(np.float64), *args)
    refb = M.grad(bf16_round(theta), *args)
    assert float(loss.item()) == pytest.approx(M.loss(bf16_round(theta), *args), rel=1e-4)
    o = 0
    for k in M.ORDER:
        n = int(np.prod(M.SIZES[k]))
        a, r64, rb = gg[o:o + n], ref64[o:o + n], refb[o:o + n]
        o += n
        assert np.linalg.norm(a - r64) <= 1e-2 * np.linalg.norm(r64) + 1e-7, k
        assert a @ r64 / (np.linalg.norm(a) * np.linalg.norm(r64) + 1e-30) > 0.999, k
        assert np.linalg.norm(a - rb) <= 1e-3 * np.linalg.norm(rb) + 1e-7, k
    net.close()


def test_adam_steps_follow_reference(torch):
    rng = np.random.default_rng(2)
    theta, mean, istd = _net_case(rng)
    B, lr, steps = 128, 1e-3, 5
    Fh = rng.standard_normal((B, 24)).astype(np.float32)
    yh = (Fh[:, 0] > 0).astype(np.float32)
    net = chym.MLP(seed=3, max_batch=512)
    net.set_params(theta, mean, istd)
    F, y = torch.from_numpy(Fh).cuda(), torch.from_numpy(yh).cuda()
    for _ in range(steps):
        net.train_step_device(F.data_ptr(), y.data_ptr(), B, lr)
    torch.cuda.synchronize()
    th_gpu = net.get_params().astype(np.float64)
    th = theta.astype(np.float64)
    m, v = np.zeros_like(th), np.zeros_like(th)
    args = (Fh.astype(np.float64), yh.astype(np.float64), mean.astype(np.float64), istd.astype(np.float64))
    for t in range(1, steps + 1):
        g = M.grad(bf16_round(th), *args)
        th, m, v = M.adam_step(th, m, v, g, t, lr)
    assert np.max(np.abs(th_gpu - th)) <= 1e-4
    assert M.loss(th, *args) < M.loss(theta.astype(np.float64), *args)
    net.close()
