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


def test_learned_early_exit_gains_over_the_plain_method(torch):
    """SK +-1 N=24, D=3, 16 pumps, K=3000 steps, decision at 10 % (step 300).

    The network is trained on GPU-generated trajectories; its threshold is set for a
    10 % false-negative rate on a calibration split and judged on a held-out split
    against the full plain integration of the same seeds.  In continuous operation
    (every slot always busy, retired slots reseeded) the ground-state hits per
    integration step must beat the plain method's."""
    from paper_2308_02329_gb300 import early_exit as EE
    N, D, K, k_dec, n_h = 24, 3, 3000, 300, 16
    J = inputs.sk_pm1(N, 77)
    ctx = chym.Context(J, D)
    prm = chym.Params(eps=0.5 / ctx.lambda_max(), prec=chym.PREC_BF16X2)
    sched = chym.Schedule(1, K // 2, K)
    h = inputs.pump_grid(0.5, n_h)
    E_gs = ctx.ground_state_exact()[0]
    assert E_gs == O.ground_state_bruteforce(J)[0]
    F, y, E = EE.generate(ctx, prm, sched, h, inputs.run_seeds(1, n_h * 1024), K, k_dec, E_gs)
    Fv, yv, Ev = EE.generate(ctx, prm, sched, h, inputs.run_seeds(2, n_h * 512), K, k_dec, E_gs)
    net = chym.MLP(seed=4, max_batch=1024)
    EE.train(net, F, y, epochs=60, batch=512, lr=2e-3)
    sv = EE.logits(net, Fv).cpu().numpy()
    yvn = yv.cpu().numpy()
    perm = np.random.default_rng(0).permutation(len(sv))
    cal, tst = perm[: len(sv) // 2], perm[len(sv) // 2:]
    theta = EE.threshold_for_fn(sv[cal], yvn[cal], 0.1)
    pos = yvn[tst] > 0.5
    n_pos = int(pos.sum())
    fn = float(np.mean(sv[tst][pos] < theta))
    rho = float(np.mean(sv[tst] < theta))
    assert n_pos >= 20
    assert fn <= 0.1 + 2.0 * np.sqrt(0.1 * 0.9 / n_pos)          # binomial 95 % bound
    expected_gain = (1 - fn) / (1 - (1 - k_dec / K) * rho)
    assert expected_gain > 1.2
    R = n_h * 128
    chunks = 80
    plain = EE.continuous(ctx, prm, sched, h, R, EE.SeedStream(10), K, k_dec, E_gs, chunks)
    learned = EE.continuous(ctx, prm, sched, h, R, EE.SeedStream(10), K, k_dec, E_gs, chunks,
                            net, theta)
    # plain continuous operation reproduces the success probability of the full runs
    p_full = yvn.mean()
    p_plain = plain.hits / plain.completed
    se = np.sqrt(p_full * (1 - p_full) / len(yvn) + p_plain * (1 - p_plain) / plain.completed)
    assert abs(p_plain - p_full) <= 1.96 * se + 1e-12
    # runs the network lets through succeed more often than the plain method's
    assert learned.hits / learned.completed > p_plain
    assert learned.hits_per_mstep > 1.05 * plain.hits_per_mstep
    net.close()
    ctx.close()


def _continuous_host_reference(torch, ctx, prm, sched, h, R, ss, K, k_dec, E_gs, chunks, net, theta):
    """Continuous operation with every decision taken on the host, chunk by chunk:
    the plain statement of the retire-and-reseed rule that the device-side
    bookkeeping of early_exit.continuous_many must reproduce exactly."""
    from paper_2308_02329_gb300 import early_exit as EE
    trace = []
    ctx.run(prm, h, ss.take(R), 0, sched)
    offs = torch.zeros(R, dtype=torch.int64, device="cuda")
    snap = torch.empty(ctx.N * ctx.D * R, dtype=torch.float32, device="cuda")
    F = torch.empty(R, chym.N_FEATURES, dtype=torch.float32, device="cuda")
    E = torch.empty(R, dtype=torch.float64, device="cuda")
    next_h = 0
    for ci in range(chunks):
        ctx.run(prm, None, None, k_dec // 2, sched, n_runs=R)
        ctx.copy_state_device(snap.data_ptr())
        ctx.run(prm, None, None, k_dec - k_dec // 2, sched, n_runs=R)
        ctx.offsets_device(offs.data_ptr())
        local = ctx.info()[2] - offs.cpu().numpy()
        done = local >= K
        ctx.energy_device(E.data_ptr())
        hit = done & (np.abs(E.cpu().numpy() - E_gs) <= 1e-9 * max(1.0, abs(E_gs)))
        at_dec = np.zeros(R, dtype=bool)
        retire = np.zeros(R, dtype=bool)
        if net is not None:
            at_dec = local == k_dec
            ctx.features_device(snap.data_ptr(), k_dec / K, F.data_ptr())
            retire = at_dec & (EE.logits(net, F).cpu().numpy() < theta)
        restart = done | retire
        trace.append((ci, 0, int(at_dec.sum()), int(retire.sum()), int(done.sum()), int(hit.sum())))
        idx = np.flatnonzero(restart).astype(np.int32)
        if len(idx):
            m = len(idx)
            fresh = torch.from_numpy(ss.take(m).view(np.int64)).cuda()
            pumps = torch.from_numpy(((next_h + np.arange(m)) % len(h)).astype(np.int32)).cuda()
            next_h = (next_h + m) % len(h)
            d_idx = torch.from_numpy(idx).cuda()
            ctx.reseed_device(d_idx.data_ptr(), m, fresh.data_ptr(), prm.init_std, pumps.data_ptr())
            torch.cuda.synchronize()
    return trace, ctx.get_state()[0]


@pytest.mark.parametrize("with_net", [False, True])
def test_continuous_bookkeeping_matches_host_reference(torch, with_net):
    """The device-side retire-and-reseed bookkeeping (one host meeting per chunk) gives
    the same decisions, retirements, completions, hits and final states as the
    host-driven statement of the rule, on a case where runs finish, are retired and
    reseeded many times over."""
    from paper_2308_02329_gb300 import early_exit as EE
    N, D, K, k_dec, n_h, R, chunks = 24, 3, 400, 40, 4, 64, 30
    J = inputs.sk_pm1(N, 78)
    E_gs = O.ground_state_bruteforce(J)[0]
    h = inputs.pump_grid(0.5, n_h)
    net, theta = None, -np.inf
    a = chym.Context(J, D)
    prm = chym.Params(eps=0.5 / a.lambda_max(), prec=chym.PREC_BF16X2)
    sched = chym.Schedule(1, K // 2, K)
    if with_net:
        net = chym.MLP(seed=4, max_batch=1024)
        F, _, _ = EE.generate(a, prm, sched, h, inputs.run_seeds(5, R), K, k_dec, E_gs)
        theta = float(np.median(EE.logits(net, F).cpu().numpy()))   # retires about half
    b = chym.Context(J, D)
    ref_trace, ref_X = _continuous_host_reference(torch, a, prm, sched, h, R, EE.SeedStream(9), K, k_dec,
                                                  E_gs, chunks, net, theta)
    trace = []
    out = EE.continuous_many([b], [prm], [sched], [h], [R], [EE.SeedStream(9)], K, k_dec, [E_gs],
                             chunks, net, theta, trace=trace)
    assert trace == ref_trace
    assert out.completed == sum(t[4] for t in ref_trace) > 0
    assert out.hits == sum(t[5] for t in ref_trace)
    if with_net:
        assert 0 < out.retired == sum(t[3] for t in ref_trace)
    assert np.array_equal(b.get_state()[0], ref_X)
    if net is not None:
        net.close()
    a.close()
    b.close()


@pytest.mark.parametrize("n_runs,with_logits", [(65536, True), (5000, True), (4096, False), (3, True), (1, False)])
def test_exit_scan_matches_its_definition(torch, n_runs, with_logits):
    """chym_exit_scan_device against the decision rule written out in numpy: runs reseeded
    at assorted steps (so their local steps differ), energies on and off the reference,
    logits on both sides of the threshold; counts and the restart order exactly."""
    N, D, K, k_dec = 8, 2, 40, 4
    J = inputs.sk_pm1(N, 3)
    ctx = chym.Context(J, D)
    prm = chym.Params(eps=0.1, prec=chym.PREC_BF16X2)
    n_h = 1
    ctx.run(prm, inputs.pump_grid(0.5, n_h), inputs.run_seeds(5, n_runs), 0, chym.Schedule(0, 0, K))
    rng = np.random.default_rng(n_runs)
    k_now = 0
    for k_next in (4, 16, 40, 44):       # reseed random subsets at a few steps
        ctx.run(prm, None, None, k_next - k_now, chym.Schedule(0, 0, K), n_runs=n_runs)
        k_now = k_next
        m = int(rng.integers(0, n_runs + 1))
        if m:
            runs = torch.from_numpy(np.sort(rng.choice(n_runs, m, replace=False)).astype(np.int32)).cuda()
            sd = torch.from_numpy(inputs.run_seeds(77 + k_now, m).view(np.int64)).cuda()
            ctx.reseed_device(runs.data_ptr(), m, sd.data_ptr(), prm.init_std)
    offs = torch.empty(n_runs, dtype=torch.int64, device="cuda")
    ctx.offsets_device(offs.data_ptr())
    local = k_now - offs.cpu().numpy()
    E_gs = -20.0
    E = np.where(rng.random(n_runs) < 0.3, E_gs, E_gs + 4.0 * rng.integers(1, 5, n_runs))
    L = rng.standard_normal(n_runs).astype(np.float32)
    theta = 0.1
    dE, dL = torch.from_numpy(E).cuda(), torch.from_numpy(L).cuda()
    counts = torch.zeros(5, dtype=torch.int64, device="cuda")
    order = torch.empty(n_runs, dtype=torch.int32, device="cuda")
    ctx.exit_scan_device(dE.data_ptr(), E_gs, dL.data_ptr() if with_logits else 0, theta, K, k_dec,
                         counts.data_ptr(), order.data_ptr())
    done = local >= K
    at_dec = (local == k_dec) & with_logits
    retire = at_dec & (L < theta)
    hit = done & (np.abs(E - E_gs) <= 1e-9 * abs(E_gs))
    restart = done | retire
    want = [int(at_dec.sum()), int(retire.sum()), int(done.sum()), int(hit.sum()), int(restart.sum())]
    assert counts.cpu().tolist() == want
    ref = np.concatenate([np.flatnonzero(restart), np.flatnonzero(~restart)])
    assert np.array_equal(order.cpu().numpy(), ref)
    ctx.close()
