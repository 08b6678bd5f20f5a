"""GPU parity of the CUDA path against the FP64 CPU oracle, through the C ABI.

Tolerances (written here, derived from the arithmetic):
  * FP64 mode: state and per-step right-hand side within 1e-10 relative;
  * FP32 mode: state within 1e-4 relative over short horizons;
  * relative errors of states are taken per (run, component) (tests.helpers.rel_err),
    so the components that annealing drives towards zero meet the same tolerance;
  * Ising spins and energies: bit-exact (integers), compared where the
    surviving component is not within rounding of zero.
"""
import numpy as np
import pytest

import oracle.oracle as O
from oracle.stats import figures_of_merit, energy_histogram
from paper_2308_02329_gb300 import chym, inputs
from tests.helpers import make_case, oracle_params, oracle_schedule, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chym.lib()


_rel_err = rel_err


def _run_both(N, D, n_h, reps, steps, prec, graph="sk", sched_kind=1, seed=7, kappa=0.1,
              sigma=1e-3):
    J, eps, h, seeds = make_case(N, D, n_h, reps, seed, graph)
    kind = chym.J_REAL if graph == "gauss" else chym.J_PM1
    ctx = chym.Context(J, D, kind)
    prm = chym.Params(eps=eps, prec=prec, kappa=kappa, sigma=sigma)
    sch = chym.Schedule(sched_kind, steps // 2 if sched_kind else 0, max(steps, 1))
    ctx.run(prm, h, seeds, steps, sch)
    X, k = ctx.get_state()
    assert k == steps
    Xo = O.run(J, D, inputs.h_per_run(h, reps), seeds, oracle_params(prm), oracle_schedule(sch),
               steps)
    return ctx, J, X, Xo


FP64_CASES = [
    # N, D, n_h, reps, steps, graph
    (1, 1, 1, 3, 20, "sk"),
    (3, 2, 2, 3, 30, "sk"),
    (20, 3, 8, 4, 60, "sk"),         # 3000-step workload's shape, short horizon
    (37, 8, 3, 7, 25, "sparse"),     # ragged N, two Philox blocks per spin
    (100, 4, 4, 5, 40, "mobius"),
    (100, 2, 2, 3, 40, "sk"),
    (130, 5, 2, 2, 20, "gauss"),     # J larger than the shared-memory budget
]


@pytest.mark.parametrize("N,D,n_h,reps,steps,graph", FP64_CASES)
def test_fp64_state_matches_oracle(N, D, n_h, reps, steps, graph):
    ctx, J, X, Xo = _run_both(N, D, n_h, reps, steps, chym.PREC_FP64, graph)
    assert _rel_err(X, Xo) <= 1e-10
    ctx.close()


def test_fp64_zero_steps_is_the_initial_state():
    ctx, J, X, Xo = _run_both(17, 3, 2, 5, 0, chym.PREC_FP64)
    assert _rel_err(X, Xo) <= 1e-15
    ctx.close()


@pytest.mark.parametrize("D", [1, 2, 3, 4, 8])
def test_fp64_one_step_rhs(D):
    """Per-step right-hand side f(x) within 1e-10 relative, from an arbitrary state."""
    N, n_h, reps = 29, 3, 3
    J, eps, h, seeds = make_case(N, D, n_h, reps, 11)
    rng = np.random.default_rng(D)
    X0 = 0.2 * rng.standard_normal((n_h * reps, N, D))
    ctx = chym.Context(J, D)
    prm = chym.Params(eps=eps, prec=chym.PREC_FP64, sigma=0.0, kappa=0.3)
    sch = chym.Schedule(1, 5, 20)
    for k0 in (0, 12):  # before and during the annealing ramp
        ctx.set_state(X0, h, seeds, k0, chym.PREC_FP64)
        ctx.run(prm, None, None, 1, sch, n_runs=len(seeds))
        X1, k = ctx.get_state()
        assert k == k0 + 1
        f_gpu = (X1 - X0) / prm.dt
        hr = inputs.h_per_run(h, reps)
        f_or = np.stack([O.drift(J, X0[r], hr[r], oracle_params(prm), oracle_schedule(sch), k0)
                         for r in range(len(seeds))])
        assert _rel_err(f_gpu, f_or) <= 1e-10
    ctx.close()


@pytest.mark.parametrize("N,D,steps", [(20, 3, 60), (100, 4, 40), (64, 2, 50), (45, 8, 30)])
def test_fp32_state_matches_oracle(N, D, steps):
    ctx, J, X, Xo = _run_both(N, D, 4, 5, steps, chym.PREC_FP32)
    assert _rel_err(X, Xo) <= 1e-4
    ctx.close()


def _comparable(X, thresh=1e-7):
    return np.abs(X[..., 0]) > thresh


@pytest.mark.parametrize("graph,prec", [("sk", chym.PREC_FP64), ("mobius", chym.PREC_FP32),
                                        ("gauss", chym.PREC_FP64)])
def test_spins_and_energies(graph, prec):
    N, D = 60, 3
    ctx, J, X, Xo = _run_both(N, D, 4, 8, 200, prec, graph)
    E, S = ctx.energy(spins=True)
    s_gpu = chym.unpack_spins(S, N)
    # the readout of the GPU's own state is exact
    assert np.array_equal(s_gpu, O.readout(X))
    Eo = O.ising_energies(J, s_gpu)
    if graph == "gauss":
        np.testing.assert_allclose(E, Eo, rtol=1e-12, atol=1e-12)
    else:
        assert np.array_equal(E, Eo)
        # every +-1 energy obeys E = -sum J (mod 4)
        assert np.all((E + J.sum()) % 4 == 0)
    # same trajectories: spins agree wherever the component is not at rounding level
    mask = _comparable(Xo, 1e-6)
    assert np.array_equal(np.sign(X[..., 0])[mask] >= 0, np.sign(Xo[..., 0])[mask] >= 0)
    ctx.close()


def test_checkpoint_resume_is_bit_identical():
    N, D, n_h, reps, K = 40, 4, 2, 4, 120
    J, eps, h, seeds = make_case(N, D, n_h, reps, 3)
    prm = chym.Params(eps=eps, prec=chym.PREC_FP64)
    sch = chym.Schedule(1, 50, K)
    a = chym.Context(J, D)
    a.run(prm, h, seeds, K, sch)
    Xa, _ = a.get_state()
    b = chym.Context(J, D)
    b.run(prm, h, seeds, K // 3, sch)
    Xb, kb = b.get_state()
    b.set_state(Xb, h, seeds, kb, chym.PREC_FP64)   # round trip through a host checkpoint
    b.run(prm, None, None, K - K // 3, sch, n_runs=len(seeds))
    Xc, kc = b.get_state()
    assert kc == K and np.array_equal(Xa, Xc)
    a.close()
    b.close()


@pytest.mark.parametrize("N,D,prec", [(40, 4, chym.PREC_FP64), (100, 3, chym.PREC_BF16X2),
                                      (200, 2, chym.PREC_FP8), (60, 5, chym.PREC_FP32)])
def test_checkpoint_restore_continues_bit_identically(N, D, prec):
    """chym_checkpoint / chym_restore carry the whole run state (storage-precision state,
    step, pumps, and per run key, seeding step and pump index): runs that were retired and
    reseeded mid-way continue in a fresh context exactly as in the original."""
    torch = pytest.importorskip("torch")
    n_h, reps, K1, K2 = 2, 6, 30, 25
    J, eps, h, seeds = make_case(N, D, n_h, reps, 23 + N)
    prm = chym.Params(eps=eps, prec=prec)
    sch = chym.Schedule(1, 20, 80)
    a = chym.Context(J, D)
    a.run(prm, h, seeds, K1, sch)
    runs = torch.tensor([1, 4, 9], dtype=torch.int32, device="cuda")
    new_seeds = torch.from_numpy(inputs.run_seeds(991, 3).view(np.int64)).cuda()
    new_pump = torch.tensor([1, 0, 1], dtype=torch.int32, device="cuda")
    a.reseed_device(runs.data_ptr(), 3, new_seeds.data_ptr(), prm.init_std, new_pump.data_ptr())
    a.run(prm, None, None, 7, sch, n_runs=len(seeds))
    blob = a.checkpoint()
    b = chym.Context(J, D)
    b.restore(blob)
    assert b.info() == a.info()
    a.run(prm, None, None, K2, sch, n_runs=len(seeds))
    b.run(prm, None, None, K2, sch, n_runs=len(seeds))
    Xa, ka = a.get_state()
    Xb, kb = b.get_state()
    assert ka == kb == K1 + 7 + K2 and np.array_equal(Xa, Xb)
    assert np.array_equal(a.energy(), b.energy())
    # a checkpoint of another size or a damaged header is refused
    c = chym.Context(inputs.sk_pm1(N + 1, 1), D)
    with pytest.raises(chym.ChymError):
        c.restore(blob)
    with pytest.raises(chym.ChymError):
        b.restore(b"XXXXXXXX" + blob[8:])
    with pytest.raises(chym.ChymError):
        b.restore(blob[:-8])
    for ctx in (a, b, c):
        ctx.close()


def test_stats_match_oracle_figures_of_merit():
    N, D, n_h, reps = 16, 2, 4, 16
    J, eps, h, seeds = make_case(N, D, n_h, reps, 5)
    ctx = chym.Context(J, D)
    prm = chym.Params(eps=eps, prec=chym.PREC_FP64)
    ctx.run(prm, h, seeds, 1500, chym.Schedule(1, 750, 1500))
    E = ctx.energy()
    E_gs, _ = O.ground_state_bruteforce(J)
    st = ctx.stats(E_gs, n_bins=64)
    fm = figures_of_merit(E, E_gs, n_h)
    assert st["hits"].tolist() == fm["hits"].tolist()
    assert st["P_max"] == fm["P_max"]
    assert st["W_range"] == pytest.approx(fm["W_range"], abs=1e-15)
    assert st["W_scan"] == pytest.approx(fm["W_scan"], abs=1e-15)
    assert st["dE_mean"] == pytest.approx(fm["dE_mean"], rel=1e-12, abs=1e-12)
    assert st["best_E"] == E.min() and st["best_run"] == int(np.argmin(E))
    assert st["n_finite"] == len(E) and st["n_hits"] == fm["hits"].sum()
    lv, ct = energy_histogram(E)
    hist = np.zeros(64, dtype=np.int64)
    for l, c in zip(lv, ct):
        hist[min(int(round((l - E_gs) / 4)), 63)] += c
    assert st["hist"].tolist() == hist.tolist()
    ctx.close()


def test_statistical_parity_fp64_full_horizon():
    """SK +-1 N=20, D=3, 8 pumps x 32 replicas, 3000 steps (1500 + 1500 annealing):
    P_Ising(h) of the GPU and of the oracle agree within binomial 95% intervals, and the
    ground state is the brute-force one."""
    N, D, n_h, reps, K = 20, 3, 8, 32, 3000
    J, eps, h, seeds = make_case(N, D, n_h, reps, 0xC0FFEE)
    ctx = chym.Context(J, D)
    prm = chym.Params(eps=eps, prec=chym.PREC_FP64)
    sch = chym.Schedule(1, 1500, K)
    ctx.run(prm, h, seeds, K, sch)
    E = ctx.energy()
    Xo = O.run(J, D, inputs.h_per_run(h, reps), seeds, oracle_params(prm), oracle_schedule(sch), K)
    Eo = O.ising_energies(J, O.readout(Xo))
    E_gs, _ = O.ground_state_bruteforce(J)
    assert E.min() >= E_gs
    P = (E.reshape(n_h, reps) == E_gs).mean(1)
    Po = (Eo.reshape(n_h, reps) == E_gs).mean(1)
    for p, q in zip(P, Po):
        half = 1.96 * np.sqrt(max(p * (1 - p), q * (1 - q), 1.0 / reps) * 2.0 / reps)
        assert abs(p - q) <= half + 1e-12
    # FP64 on both sides: the large majority of runs end in the very same state
    assert np.mean(E == Eo) >= 0.9
    ctx.close()


def test_invalid_arguments_and_order():
    J, eps, h, seeds = make_case(10, 2, 2, 3, 1)
    ctx = chym.Context(J, 2)
    prm = chym.Params(eps=eps, prec=chym.PREC_FP64)
    with pytest.raises(chym.ChymError) as e:
        ctx.energy()
    assert e.value.status == chym.ESTATE
    with pytest.raises(chym.ChymError) as e:
        ctx.run(prm, h, seeds[:5], 10, chym.Schedule(0, 0, 1))  # 5 runs, 2 pumps
    assert e.value.status == chym.EINVAL
    with pytest.raises(chym.ChymError) as e:
        ctx.run(prm, h, seeds, 10, chym.Schedule(1, 10, 5))     # k_total <= k_anneal
    assert e.value.status == chym.EINVAL
    ctx.run(prm, h, seeds, 10, chym.Schedule(0, 0, 1))
    with pytest.raises(chym.ChymError) as e:
        ctx.run(chym.Params(eps=eps, prec=chym.PREC_FP32), None, None, 5, chym.Schedule(0, 0, 1),
                n_runs=len(seeds))
    assert e.value.status == chym.EINVAL
    bad = chym.Params(eps=eps, prec=chym.PREC_FP64, dt=-1.0)
    with pytest.raises(chym.ChymError) as e:
        ctx.run(bad, h, seeds, 10, chym.Schedule(0, 0, 1))
    assert e.value.status == chym.EINVAL
    ctx.close()


def test_lambda_max_matches_eigvalsh():
    for J in (inputs.sk_pm1(50, 2), inputs.mobius_ladder(40), inputs.gaussian(70, 3)):
        ctx = chym.Context(J, 1, chym.J_REAL)
        assert ctx.lambda_max() == pytest.approx(np.linalg.eigvalsh(J)[-1], rel=1e-10)
        ctx.close()


def test_ground_state_references_match_oracle():
    for N, seed in ((8, 1), (14, 2), (20, 0xC0FFEE)):
        J = inputs.sk_pm1(N, seed)
        ctx = chym.Context(J, 1)
        e, s = ctx.ground_state_exact()
        assert e == O.ground_state_bruteforce(J)[0]
        assert O.ising_energy(J, s) == e
        e_sa, s_sa = ctx.ground_state_search(restarts=16, sweeps=300, seed=3)
        assert e_sa >= e and O.ising_energy(J, s_sa) == e_sa
        ctx.close()
    for N in (6, 10, 20, 100):
        assert chym.ground_state_mobius(N) == O.ground_state_mobius(N, -1.0, -1.0)


# ---------------------------------------------------------------------------
# tensor-core path: J on tcgen05 in BF16, x split into BF16 hi + lo, FP32 state
# ---------------------------------------------------------------------------
BF16_CASES = [
    # N, D, n_h, reps, steps, graph
    (100, 4, 4, 7, 60, "sk"),        # 28 runs: a ragged group
    (100, 2, 2, 33, 60, "mobius"),   # 66 runs: two CTAs, second one nearly empty
    (100, 3, 3, 11, 60, "sk"),
    (20, 3, 8, 4, 80, "sk"),
    (37, 8, 3, 5, 40, "sparse"),     # two Philox blocks per spin, 4-run chunks
    (128, 5, 2, 9, 40, "sk"),        # full 128-lane tile, three groups per CTA
    (64, 6, 2, 4, 40, "sk"),
    (13, 7, 1, 5, 40, "sk"),
    (1, 1, 1, 3, 20, "sk"),
    (61, 1, 2, 70, 50, "sparse"),    # D = 1: the CIM
    (90, 4, 2, 6, 40, "gauss"),      # real J: three-term split
]


@pytest.mark.parametrize("N,D,n_h,reps,steps,graph", BF16_CASES)
def test_bf16x2_state_matches_oracle(N, D, n_h, reps, steps, graph):
    ctx, J, X, Xo = _run_both(N, D, n_h, reps, steps, chym.PREC_BF16X2, graph)
    assert np.all(np.isfinite(X))
    assert _rel_err(X, Xo) <= 1e-4
    ctx.close()


def test_bf16x2_energies_and_continuation():
    N, D, n_h, reps, K = 100, 4, 4, 16, 400
    J, eps, h, seeds = make_case(N, D, n_h, reps, 21)
    prm = chym.Params(eps=eps, prec=chym.PREC_BF16X2)
    sch = chym.Schedule(1, K // 2, K)
    a = chym.Context(J, D)
    a.run(prm, h, seeds, K, sch)
    Xa, _ = a.get_state()
    E, S = a.energy(spins=True)
    s = chym.unpack_spins(S, N)
    assert np.array_equal(s, O.readout(Xa))
    assert np.array_equal(E, O.ising_energies(J, s))
    # continuing in two launches is bit-identical on the GPU
    b = chym.Context(J, D)
    b.run(prm, h, seeds, K // 4, sch)
    b.run(prm, None, None, K - K // 4, sch, n_runs=len(seeds))
    Xb, kb = b.get_state()
    assert kb == K and np.array_equal(Xa, Xb)
    # and the FP32 SIMT form agrees with the tensor-core form on this short horizon
    c = chym.Context(J, D)
    c.run(chym.Params(eps=eps, prec=chym.PREC_FP32), h, seeds, K, sch)
    Xc, _ = c.get_state()
    assert _rel_err(Xa, Xc) <= 1e-4
    for x in (a, b, c):
        x.close()


def test_bf16x2_full_size_launch_sampled_runs():
    """The benchmark's launch shape (N=100, D=4, 4096 runs = 32 h x 128 replicas):
    sampled runs against the oracle, run by run."""
    N, D, n_h, reps, K = 100, 4, 32, 128, 150
    J, eps, h, seeds = make_case(N, D, n_h, reps, 0xC0FFEE + 1)
    ctx = chym.Context(J, D)
    prm = chym.Params(eps=eps, prec=chym.PREC_BF16X2)
    sch = chym.Schedule(1, 10000, 20000)
    ctx.run(prm, h, seeds, K, sch)
    X, _ = ctx.get_state()
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(n_h * reps, 24, replace=False))
    pick[0], pick[-1] = 0, n_h * reps - 1
    hr = inputs.h_per_run(h, reps)[pick]
    Xo = O.run(J, D, hr, seeds[pick], oracle_params(prm), oracle_schedule(sch), K)
    assert _rel_err(X[pick], Xo) <= 1e-4
    ctx.close()


def test_bf16x2_statistical_parity_long_horizon():
    """Moebius ladder N=100, D=4, 8 pumps x 32 replicas, 20000 steps (annealed over the
    second half): per-pump success probability and the mean energy above the exact
    ground state agree with the FP64 oracle within 95% intervals."""
    N, D, n_h, reps, K = 100, 4, 8, 32, 20000
    J, eps, h, seeds = make_case(N, D, n_h, reps, 5, graph="mobius")
    E_gs = O.ground_state_mobius(N, -1.0, -1.0)
    ctx = chym.Context(J, D)
    prm = chym.Params(eps=eps, prec=chym.PREC_BF16X2)
    sch = chym.Schedule(1, K // 2, K)
    ctx.run(prm, h, seeds, K, sch)
    E = ctx.energy()
    Xo = O.run(J, D, inputs.h_per_run(h, reps), seeds, oracle_params(prm), oracle_schedule(sch), K)
    Eo = O.ising_energies(J, O.readout(Xo))
    assert E.min() >= E_gs and Eo.min() >= E_gs
    P = (E.reshape(n_h, reps) == E_gs).mean(1)
    Po = (Eo.reshape(n_h, reps) == E_gs).mean(1)
    for p, q in zip(P, Po):
        half = 1.96 * np.sqrt(max(p * (1 - p), q * (1 - q), 1.0 / reps) * 2.0 / reps)
        assert abs(p - q) <= half + 1e-12
    d, do = E - E_gs, Eo - E_gs
    se = np.sqrt(d.var() / d.size + do.var() / do.size)
    assert abs(d.mean() - do.mean()) <= 1.96 * se + 1e-9
    ctx.close()


# ---------------------------------------------------------------------------
# XY readout by best-axis rounding (D = 2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,graph,prec", [(30, "sk", chym.PREC_BF16X2), (100, "mobius", chym.PREC_BF16X2),
                                          (150, "gauss", chym.PREC_BF16X2), (24, "sk", chym.PREC_FP64),
                                          (45, "sparse", chym.PREC_FP32), (257, "sk", chym.PREC_BF16X2)])
def test_readout_xy_matches_oracle(N, graph, prec):
    """XY machine (D = 2, no annealing): the best-axis energies equal the oracle's
    rounding of the same final states (exactly for +-1 couplings), the returned
    spins reach them, and they are never above the first-component readout."""
    J, eps, h, seeds = make_case(N, 2, 2, 8, 21, graph)
    kind = chym.J_REAL if graph == "gauss" else chym.J_PM1
    ctx = chym.Context(J, 2, kind)
    prm = chym.Params(eps=eps, prec=prec, kappa=1e-3)
    ctx.run(prm, h, seeds, 300, chym.Schedule(0, 0, 300))
    X, _ = ctx.get_state()
    E_plain = ctx.energy()
    E, S = ctx.readout_xy(spins=True)
    s = chym.unpack_spins(S, N)
    for r in range(len(seeds)):
        e_o, _ = O.round_xy(J, X[r].astype(np.float64))
        if kind == chym.J_PM1:
            assert E[r] == e_o
            assert O.ising_energy(J, s[r]) == E[r]
        else:
            assert abs(E[r] - e_o) <= 1e-9 * max(1.0, abs(e_o))
            assert abs(O.ising_energy(J, s[r]) - E[r]) <= 1e-9 * max(1.0, abs(E[r]))
        assert E[r] <= E_plain[r] + 1e-9 * max(1.0, abs(E_plain[r]))
    torch = pytest.importorskip("torch")
    d_E = torch.empty(len(seeds), dtype=torch.float64, device="cuda")
    ctx.readout_xy_device(d_E.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(d_E.cpu().numpy(), E)
    ctx.close()
    c3 = chym.Context(J, 3, kind)
    with pytest.raises(chym.ChymError):
        c3.readout_xy()
    c3.close()


# ---------------------------------------------------------------------------
# large-N path (N > 128): per-step tcgen05 GEMM with the update in its epilogue
# ---------------------------------------------------------------------------
K2_CASES = [
    # N, D, n_h, reps, steps, graph
    (129, 4, 2, 5, 30, "sk"),       # one spin past a full tile: 2 M tiles, ragged K
    (200, 3, 3, 7, 30, "sk"),
    (256, 2, 2, 40, 25, "sparse"),  # 80 runs: two column tiles, second one partial
    (300, 8, 1, 9, 20, "sk"),
    (150, 4, 2, 4, 20, "gauss"),    # real J: three-term split
    (170, 1, 2, 70, 30, "sk"),      # the CIM
    (140, 5, 1, 20, 20, "sk"),
    (190, 6, 1, 17, 20, "sk"),
    (133, 7, 1, 17, 20, "sparse"),
    (1000, 4, 2, 3, 15, "sk"),
    (2000, 8, 1, 3, 6, "sk"),       # the largest instances of the uneven workload
    (4096, 2, 1, 2, 4, "sk"),       # the largest N the features and tiles are sized for
]


@pytest.mark.parametrize("N,D,n_h,reps,steps,graph", K2_CASES)
def test_large_n_state_matches_oracle(N, D, n_h, reps, steps, graph):
    ctx, J, X, Xo = _run_both(N, D, n_h, reps, steps, chym.PREC_BF16X2, graph)
    assert np.all(np.isfinite(X))
    assert _rel_err(X, Xo) <= 1e-4
    ctx.close()


# FP8 mode: the lo half of the split in e4m3, J in e4m3 (exact for +-1).  x is then held
# in the product within 2^-13 |x| (8 bits of the BF16 hi, 4 of the e4m3 lo), so a step's
# coupling term eps J x is off by eps sum_q J_pq d_q with |d_q| <= 2^-13 |x_q|: about
# eps sqrt(N) 2^-13 |x| for independent roundings (eps sqrt(N) = 1/4 here), 3e-7 |x| a
# step after the factor dt.  Over at most 30 steps that stays near 1e-5, within the 1e-4
# mixed-precision bound.  Real J keeps the BF16 three-term products (FP8 mode runs as
# BF16X2 there), and so does the small-N kernel.
FP8_CASES = [
    # N, D, n_h, reps, steps, graph
    (129, 4, 2, 5, 30, "sk"),
    (200, 3, 3, 7, 30, "sk"),
    (256, 2, 2, 40, 25, "sparse"),  # two column tiles, the second partial
    (300, 8, 1, 9, 20, "sk"),
    (170, 1, 2, 70, 30, "sk"),
    (190, 6, 1, 17, 20, "sk"),
    (1000, 4, 2, 3, 15, "sk"),
    (2000, 8, 1, 3, 6, "sk"),
    (150, 4, 2, 4, 20, "gauss"),    # real J: BF16 three-term products
    (100, 4, 2, 6, 30, "sk"),       # N <= 128: the small-N kernel (BF16 hi + lo)
    (4096, 2, 1, 2, 4, "sk"),       # the largest N
]


@pytest.mark.parametrize("N,D,n_h,reps,steps,graph", FP8_CASES)
def test_fp8_state_matches_oracle(N, D, n_h, reps, steps, graph):
    ctx, J, X, Xo = _run_both(N, D, n_h, reps, steps, chym.PREC_FP8, graph)
    assert np.all(np.isfinite(X))
    assert _rel_err(X, Xo) <= 1e-4
    # the sign readout of the GPU's own state: exact integer energies for +-1 J, FP64
    # sums in another order for real J
    E, Eo = ctx.energy(), O.ising_energies(J, O.readout(X))
    if graph == "gauss":
        assert np.allclose(E, Eo, rtol=1e-12, atol=1e-12)
    else:
        assert np.array_equal(E, Eo)
    ctx.close()


def test_fp8_is_less_exact_than_bf16x2_but_close():
    """FP8 mode against BF16X2 on the same seeds: the e4m3 lo half (4 bits instead of 8)
    shows as a larger but still small state difference from the oracle."""
    e = {}
    for prec in (chym.PREC_BF16X2, chym.PREC_FP8):
        ctx, J, X, Xo = _run_both(600, 4, 2, 16, 20, prec, "sk")
        e[prec] = _rel_err(X, Xo)
        ctx.close()
    assert e[chym.PREC_BF16X2] < e[chym.PREC_FP8] <= 1e-4


def test_fp8_in_a_batch_equals_alone():
    """FP8 contexts in a batch beside BF16X2 ones: each gives the state it has alone."""
    specs = [(inputs.sk_pm1(300, 3), 4, chym.PREC_FP8), (inputs.sk_pm1(260, 4), 4, chym.PREC_BF16X2),
             (inputs.sk_pm1(96, 5), 3, chym.PREC_FP8)]

    def make():
        out = []
        for k, (J, D, prec) in enumerate(specs):
            c = chym.Context(J, D)
            prm = chym.Params(eps=0.5 / c.lambda_max(), prec=prec)
            sch = chym.Schedule(1, 20, 60)
            c.run(prm, inputs.pump_grid(0.5, 2), inputs.run_seeds(71 + k, 40), 0, sch)
            out.append((c, prm, sch))
        return out

    batched = make()
    b = chym.Batch([c for c, _, _ in batched])
    b.run([p for _, p, _ in batched], [s for _, _, s in batched], 36)
    b.status()
    b.close()
    for (c, p, s), (ca, _, _) in zip(make(), batched):
        c.run(p, None, None, 36, s)
        assert np.array_equal(c.get_state()[0], ca.get_state()[0])
        c.close()
        ca.close()


def test_large_n_continuation_and_energies():
    N, D, n_h, reps, K = 257, 4, 2, 6, 40
    J, eps, h, seeds = make_case(N, D, n_h, reps, 13)
    prm = chym.Params(eps=eps, prec=chym.PREC_BF16X2)
    sch = chym.Schedule(1, 20, K)
    a = chym.Context(J, D)
    a.run(prm, h, seeds, K, sch)
    Xa, _ = a.get_state()
    b = chym.Context(J, D)
    b.run(prm, h, seeds, 17, sch)
    b.run(prm, None, None, K - 17, sch, n_runs=len(seeds))
    Xb, _ = b.get_state()
    assert np.array_equal(Xa, Xb)
    E, S = a.energy(spins=True)
    s = chym.unpack_spins(S, N)
    assert np.array_equal(s, O.readout(Xa))
    assert np.array_equal(E, O.ising_energies(J, s))
    a.close()
    b.close()


@pytest.mark.parametrize("N,runs,steps", [(1000, 16384, 12), (800, 65536, 6)])
def test_large_n_full_size_launch_sampled_runs(N, runs, steps):
    """Launch shapes of the dense SK workloads (N=1000 with 16384 runs, N=800 with
    65536 runs, D=4): sampled runs against the oracle, run by run."""
    D, n_h = 4, 32
    reps = runs // n_h
    J, eps, h, seeds = make_case(N, D, n_h, reps, 0xC0FFEE + N)
    ctx = chym.Context(J, D)
    prm = chym.Params(eps=eps, prec=chym.PREC_BF16X2)
    sch = chym.Schedule(1, 25000, 50000)
    ctx.run(prm, h, seeds, steps, sch)
    X, _ = ctx.get_state()
    rng = np.random.default_rng(1)
    pick = np.sort(rng.choice(runs, 12, replace=False))
    pick[0], pick[-1] = 0, runs - 1
    hr = inputs.h_per_run(h, reps)[pick]
    Xo = O.run(J, D, hr, seeds[pick], oracle_params(prm), oracle_schedule(sch), steps)
    assert _rel_err(X[pick], Xo) <= 1e-4
    ctx.close()


# ---------------------------------------------------------------------------
# batched integration of many contexts
# ---------------------------------------------------------------------------
def test_batch_equals_contexts_run_alone():
    """A batch mixing dimensions, sizes and paths gives bit-identical states to each
    context integrated on its own, also when split over two batch calls."""
    cases = [  # N, D, n_h, reps, graph, prec
        (100, 2, 4, 33, "mobius", chym.PREC_BF16X2),
        (100, 3, 4, 17, "sk", chym.PREC_BF16X2),
        (60, 4, 7, 11, "sk", chym.PREC_BF16X2),
        (37, 4, 2, 9, "sparse", chym.PREC_BF16X2),
        (90, 4, 2, 6, "gauss", chym.PREC_BF16X2),
        (20, 3, 2, 5, "sk", chym.PREC_FP32),
        (200, 4, 2, 4, "sk", chym.PREC_BF16X2),
    ]
    K = 60
    solo, batched, prms, schs = [], [], [], []
    for i, (N, D, n_h, reps, graph, prec) in enumerate(cases):
        J, eps, h, seeds = make_case(N, D, n_h, reps, 40 + i, graph)
        kind = chym.J_REAL if graph == "gauss" else chym.J_PM1
        prm = chym.Params(eps=eps, prec=prec)
        sch = chym.Schedule(1, 30, K)
        a = chym.Context(J, D, kind)
        a.run(prm, h, seeds, K, sch)
        solo.append(a.get_state()[0])
        a.close()
        b = chym.Context(J, D, kind)
        b.run(prm, h, seeds, 0, sch)
        batched.append(b)
        prms.append(prm)
        schs.append(sch)
    batch = chym.Batch(batched)
    batch.run(prms, schs, 25)
    batch.run(prms, schs, K - 25)
    batch.status()
    for Xs, b in zip(solo, batched):
        Xb, kb = b.get_state()
        assert kb == K
        assert np.array_equal(Xs, Xb)
    batch.close()
    for b in batched:
        b.close()


def test_batch_many_small_instances_against_oracle():
    """Twenty uneven instances (N 50..128, D in {2,3,4,8}) in one batch; sampled runs
    of each against the oracle."""
    rng = np.random.default_rng(7)
    ctxs, prms, schs, meta = [], [], [], []
    K = 30
    for i in range(20):
        N = int(rng.integers(50, 129))
        D = int(rng.choice([2, 3, 4, 8]))
        J, eps, h, seeds = make_case(N, D, 4, 16, 100 + i)
        c = chym.Context(J, D)
        prm = chym.Params(eps=eps, prec=chym.PREC_BF16X2)
        sch = chym.Schedule(1, 15, K)
        c.run(prm, h, seeds, 0, sch)
        ctxs.append(c)
        prms.append(prm)
        schs.append(sch)
        meta.append((J, D, h, seeds))
    batch = chym.Batch(ctxs)
    batch.run(prms, schs, K)
    for c, prm, sch, (J, D, h, seeds) in zip(ctxs, prms, schs, meta):
        X, _ = c.get_state()
        pick = [0, 17, 63]
        hr = inputs.h_per_run(h, 16)[pick]
        Xo = O.run(J, D, hr, seeds[pick], oracle_params(prm), oracle_schedule(sch), K)
        assert _rel_err(X[pick], Xo) <= 1e-4
        c.close()
    batch.close()


def test_batch_tuning_keeps_states_and_results(tmp_path):
    """chym_batch_tune measures the planner's cost model on the device and restores
    every state it advanced; a tuned batch (small-N dimensions next to large-N
    contexts) still equals the contexts integrated alone, and a tuning cache hit
    sets the cached costs without measuring."""
    cases = [(100, 2, 4, 20, "mobius"), (60, 3, 4, 9, "sk"), (128, 8, 2, 8, "sk"),
             (300, 4, 4, 5, "sk"), (611, 2, 2, 7, "sk"), (200, 3, 2, 4, "gauss")]
    K = 40
    solo, ctxs, prms, schs = [], [], [], []
    for i, (N, D, n_h, reps, graph) in enumerate(cases):
        J, eps, h, seeds = make_case(N, D, n_h, reps, 70 + i, graph)
        kind = chym.J_REAL if graph == "gauss" else chym.J_PM1
        prm = chym.Params(eps=eps, prec=chym.PREC_BF16X2)
        sch = chym.Schedule(1, 20, K)
        a = chym.Context(J, D, kind)
        a.run(prm, h, seeds, K, sch)
        solo.append(a.get_state()[0])
        a.close()
        b = chym.Context(J, D, kind)
        b.run(prm, h, seeds, 5, sch)
        ctxs.append(b)
        prms.append(prm)
        schs.append(sch)
    before = [c.get_state() for c in ctxs]
    batch = chym.Batch(ctxs)
    assert not batch.tuning()["tuned"]
    cache = str(tmp_path / "tuning.json")
    t = batch.tune(prms, schs, probe_steps=12, cache_path=cache)
    assert t["tuned"] and t["k2"] > 0 and all(c > 0 for c in t["chunk"])
    for (Xb, kb), c in zip(before, ctxs):
        Xa, ka = c.get_state()
        assert ka == kb and np.array_equal(Xa, Xb)
    batch.run(prms, schs, K - 5)
    batch.status()
    for Xs, c in zip(solo, ctxs):
        assert np.array_equal(Xs, c.get_state()[0])
    # a second batch of the same composition takes the cached costs
    other = chym.Batch(ctxs)
    other.set_tuning({"chunk": [1.0] * 8, "k2": 1.0})
    t2 = other.tune(prms, schs, probe_steps=12, cache_path=cache)
    assert t2["chunk"] == t["chunk"] and t2["k2"] == t["k2"] and t2["shapes"] == t["shapes"]
    # the chosen tile shapes are valid ones (0: default) for the batch's dimensions
    for D in range(1, 9):
        rt, st, ch = (t["shapes"][k][D - 1] for k in ("rt", "stages", "ch"))
        assert rt == 0 or (rt % 32 == 0 and D * rt <= 256)
        assert st == 0 or 2 <= st <= 8
        assert ch in (0, 4, 8)
    with pytest.raises(chym.ChymError):
        other.set_tuning({"chunk": [1.0] * 7 + [0.0], "k2": 1.0})
    other.close()
    batch.close()
    for c in ctxs:
        c.close()


def test_batch_tile_shapes_leave_results_unchanged():
    """Every tile shape the autotuner may choose (large-N runs per column tile and ring
    depth, small-N epilogue chunk) computes the same arithmetic per element in the same
    order: states are bit-identical to the default shapes; invalid shapes are refused."""
    cases = [(100, 2, 4, 20, "mobius"), (60, 3, 4, 9, "sk"), (90, 4, 2, 20, "sk"), (40, 1, 2, 40, "sk"),
             (300, 4, 4, 16, "sk"), (611, 2, 2, 40, "sk"), (200, 3, 2, 40, "gauss"), (250, 1, 2, 80, "sk")]
    K = 24

    def run(shapes):
        ctxs, prms, schs = [], [], []
        for i, (N, D, n_h, reps, graph) in enumerate(cases):
            J, eps, h, seeds = make_case(N, D, n_h, reps, 170 + i, graph)
            c = chym.Context(J, D, chym.J_REAL if graph == "gauss" else chym.J_PM1)
            prm = chym.Params(eps=eps, prec=chym.PREC_BF16X2)
            sch = chym.Schedule(1, 10, K)
            c.run(prm, h, seeds, 0, sch)
            ctxs.append(c)
            prms.append(prm)
            schs.append(sch)
        b = chym.Batch(ctxs)
        if shapes:
            b.set_shapes(shapes)
            assert b.shapes() == shapes
        b.run(prms, schs, K)
        b.status()
        out = [c.get_state()[0] for c in ctxs]
        b.close()
        for c in ctxs:
            c.close()
        return out

    ref = run(None)
    for shapes in ({"rt": [32] * 8, "stages": [2] * 8, "ch": [4, 4, 4, 4, 0, 0, 0, 0]},
                   {"rt": [128, 64, 32, 32, 32, 32, 32, 32], "stages": [3] * 8, "ch": [8, 8, 8, 8, 0, 0, 0, 0]}):
        for a, b in zip(ref, run(shapes)):
            assert np.array_equal(a, b)
    c = chym.Context(inputs.sk_pm1(20, 1), 2)
    b = chym.Batch([c])
    for bad in ({"rt": [48] + [0] * 7}, {"rt": [0, 0, 0, 128, 0, 0, 0, 0]}, {"stages": [1] + [0] * 7},
                {"ch": [0] * 4 + [4] + [0] * 3}, {"ch": [6] + [0] * 7}):
        with pytest.raises(chym.ChymError):
            b.set_shapes(bad)
    b.close()
    c.close()


def test_uneven_batch_full_size_sampled():
    """The batched uneven workload at its full size: 512 SK +-1 instances with N uniform
    in [50, 2000] and D in {2, 3, 4, 8}, 64 runs each (16 pumps x 4 replicas), tuned
    and integrated as one batch for a few steps; one sampled run of every 32nd
    instance against the oracle.  eps = 0.5 / (2 sqrt(N)), the edge of the SK
    spectrum."""
    comp = inputs.uneven_instances(512, 4)
    K, n_h, reps = 6, 16, 4
    ctxs, prms, schs, meta = [], [], [], []
    for N, D, seed in comp:
        J = inputs.sk_pm1(N, seed)
        eps = 0.25 / np.sqrt(N)
        h = inputs.pump_grid(0.5, n_h)
        seeds = inputs.run_seeds(seed, n_h * reps)
        c = chym.Context(J, D)
        prm = chym.Params(eps=eps, prec=chym.PREC_BF16X2)
        sch = chym.Schedule(1, 3, K)
        c.run(prm, h, seeds, 0, sch)
        ctxs.append(c)
        prms.append(prm)
        schs.append(sch)
        meta.append((N, D, seed, h, seeds))
        del J
    assert sum(1 for N, _, _ in comp if N <= 128) >= 10
    batch = chym.Batch(ctxs)
    batch.tune(prms, schs, probe_steps=2)
    batch.run(prms, schs, K)
    batch.status()
    for i in range(0, 512, 32):
        N, D, seed, h, seeds = meta[i]
        X, k = ctxs[i].get_state()
        assert k == K
        r = (7 * i) % (n_h * reps)
        hr = inputs.h_per_run(h, reps)[[r]]
        Xo = O.run(inputs.sk_pm1(N, seed), D, hr, seeds[[r]], oracle_params(prms[i]),
                   oracle_schedule(schs[i]), K)
        assert _rel_err(X[[r]], Xo) <= 1e-4, (N, D)
    batch.close()
    for c in ctxs:
        c.close()


# ---------------------------------------------------------------------------
# retire-and-reseed: a reseeded run follows the trajectory of a fresh run
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,D,prec,tol", [(24, 3, chym.PREC_FP64, 1e-10),
                                          (100, 4, chym.PREC_BF16X2, 1e-4),
                                          (150, 2, chym.PREC_BF16X2, 1e-4),
                                          (61, 1, chym.PREC_BF16X2, 1e-4),
                                          (64, 2, chym.PREC_BF16X2, 1e-4),
                                          (40, 8, chym.PREC_FP32, 1e-4)])
def test_reseeded_runs_restart_at_local_step_zero(N, D, prec, tol):
    torch = pytest.importorskip("torch")
    n_h, reps, K1, K2 = 2, 6, 40, 30
    J, eps, h, seeds = make_case(N, D, n_h, reps, 17)
    prm = chym.Params(eps=eps, prec=prec)
    sch = chym.Schedule(1, 35, 60)  # the ramp starts inside both segments
    ctx = chym.Context(J, D)
    ctx.run(prm, h, seeds, K1, sch)
    picked = np.array([1, 3, 10], dtype=np.int32)
    fresh = inputs.run_seeds(999, len(picked))
    d_runs = torch.from_numpy(picked).cuda()
    d_seeds = torch.from_numpy(fresh.view(np.int64)).cuda()
    ctx.reseed_device(d_runs.data_ptr(), len(picked), d_seeds.data_ptr(), prm.init_std)
    ctx.run(prm, None, None, K2, sch, n_runs=len(seeds))
    X, k = ctx.get_state()
    assert k == K1 + K2
    offs = torch.zeros(len(seeds), dtype=torch.int64, device="cuda")
    ctx.offsets_device(offs.data_ptr())
    torch.cuda.synchronize()
    assert offs.cpu().numpy().tolist() == [K1 if r in picked else 0 for r in range(len(seeds))]
    hr = inputs.h_per_run(h, reps)
    rest = np.array([r for r in range(len(seeds)) if r not in picked])
    Xo_rest = O.run(J, D, hr[rest], seeds[rest], oracle_params(prm), oracle_schedule(sch), K1 + K2)
    Xo_new = O.run(J, D, hr[picked], fresh, oracle_params(prm), oracle_schedule(sch), K2)
    assert _rel_err(X[rest], Xo_rest) <= tol
    assert _rel_err(X[picked], Xo_new) <= tol
    ctx.close()


@pytest.mark.parametrize("N,D,prec", [(40, 2, chym.PREC_BF16X2), (40, 2, chym.PREC_FP64),
                                      (150, 2, chym.PREC_BF16X2)])
def test_diverged_runs_are_flagged_not_counted(N, D, prec):
    """Runs whose state holds an infinity or a NaN (a diverged run) read out as NaN energies
    in both readouts, count neither as hits nor in the energy statistics, and leave the
    other runs' results untouched."""
    J, eps, h, seeds = make_case(N, D, 2, 4, 5, "sk")
    ctx = chym.Context(J, D)
    prm = chym.Params(eps=eps, prec=prec)
    ctx.run(prm, h, seeds, 20, chym.Schedule(0, 0, 20))
    X, k = ctx.get_state()
    X[1, 3, 0] = np.inf
    X[5, 0, 1] = np.nan
    ctx.set_state(X, h, seeds, k, prec)
    E = ctx.energy()
    bad = np.zeros(len(seeds), dtype=bool)
    bad[[1, 5]] = True
    assert np.all(np.isnan(E[bad])) and np.all(np.isfinite(E[~bad]))
    s = np.where(X[:, :, 0] >= 0, 1, -1).astype(np.int8)
    assert np.array_equal(E[~bad], O.ising_energies(J, s)[~bad])
    E_gs = float(np.min(E[~bad]))
    st = ctx.stats(E_gs)
    assert int(st["n_finite"]) == int(np.sum(~bad))
    assert int(st["n_hits"]) == int(np.sum(E[~bad] == E_gs))
    assert st["dE_mean"] == pytest.approx(np.mean(E[~bad] - E_gs), rel=1e-12, abs=1e-12)
    Exy = ctx.readout_xy()
    assert np.all(np.isnan(Exy[bad])) and np.all(np.isfinite(Exy[~bad]))
    for r in np.flatnonzero(~bad):
        assert Exy[r] == O.round_xy(J, X[r])[0]
    ctx.close()


@pytest.mark.parametrize("D,prec,tol", [(2, chym.PREC_FP64, 1e-10), (1, chym.PREC_FP32, 1e-4),
                                        (2, chym.PREC_BF16X2, 1e-4), (3, chym.PREC_BF16X2, 1e-4)])
def test_packed_graphs_match_oracle(D, prec, tol):
    """Three sparse graphs packed into one context (block-diagonal J, per-spin coupling
    weights 1/lambda_max of each graph): the state equals the oracle's integration of
    J' = diag(w) J, and the segment energies equal each graph's own Ising energy of the
    same state (exact integers)."""
    from paper_2308_02329_gb300 import packing
    Js = [inputs.sparse_pm1(n, 0.2, 900 + n) for n in (23, 10, 17)]
    P = packing.build(Js, [0, 2, 1])
    lam = [float(np.linalg.eigvalsh(J)[-1]) for J in Js]
    w = packing.spin_weights(P, [1.0 / lam[i] for i in P.members])
    n_h, reps, steps = 3, 5, 60
    h = inputs.pump_grid(0.5, n_h)
    seeds = inputs.run_seeds(41, n_h * reps)
    ctx = chym.Context(P.J, D)
    ctx.set_coupling_weights(w)
    prm = chym.Params(eps=0.5, prec=prec, kappa=0.1)
    sch = chym.Schedule(1, steps // 2, steps)
    ctx.run(prm, h, seeds, steps, sch)
    X, _ = ctx.get_state()
    Xo = O.run(w[:, None] * P.J, D, inputs.h_per_run(h, reps), seeds, oracle_params(prm),
               oracle_schedule(sch), steps)
    assert _rel_err(X, Xo) <= tol
    Eseg = ctx.energy_segments(P.seg_begin)
    assert Eseg.shape == (n_h * reps, 3)
    for b, i in enumerate(P.members):
        lo, hi = P.seg_begin[b], P.seg_begin[b + 1]
        assert np.array_equal(Eseg[:, b], O.ising_energies(Js[i], O.readout(X[:, lo:hi, :])))
    assert np.array_equal(Eseg.sum(axis=1), ctx.energy())   # no coupling between the blocks
    # clearing the weights restores the plain equations
    ctx.set_coupling_weights(None)
    ctx.run(prm, h, seeds, steps, sch)
    Xp = O.run(P.J, D, inputs.h_per_run(h, reps), seeds, oracle_params(prm), oracle_schedule(sch), steps)
    assert _rel_err(ctx.get_state()[0], Xp) <= tol
    ctx.close()


def test_coupling_weights_arguments():
    ctx = chym.Context(inputs.sk_pm1(200, 3), 2)
    with pytest.raises(chym.ChymError):
        ctx.set_coupling_weights(np.full(200, np.nan))
    ctx.set_coupling_weights(np.ones(200))
    prm = chym.Params(eps=0.01, prec=chym.PREC_BF16X2)
    with pytest.raises(chym.ChymError, match="ENOTSUP"):
        ctx.run(prm, inputs.pump_grid(0.5, 2), inputs.run_seeds(1, 4), 10, chym.Schedule(0, 0, 10))
    ctx.run(prm, inputs.pump_grid(0.5, 2), inputs.run_seeds(1, 4), 0, chym.Schedule(0, 0, 10))
    for bad in ([0, 100], [0, 100, 100, 200], [1, 200], [0, 201]):
        with pytest.raises(chym.ChymError):
            ctx.energy_segments(bad)
    ctx.close()


def _sparse_graph(kind, N, seed):
    return inputs.mobius_ladder(N) if kind == "mobius" else inputs.sparse_pm1(N, 0.02, seed)


@pytest.mark.parametrize("N,D,graph,prec,tol,csr", [(200, 3, "mobius", chym.PREC_FP64, 1e-10, True),
                                                    (200, 2, "mobius", chym.PREC_FP32, 1e-4, True),
                                                    (300, 4, "er2", chym.PREC_FP32, 1e-4, True),
                                                    (260, 1, "mobius", chym.PREC_FP64, 1e-10, True),
                                                    (1024, 3, "mobius", chym.PREC_BF16X2, 1e-4, True),
                                                    (410, 2, "er2", chym.PREC_BF16X2, 1e-4, False)])
def test_sparse_graphs_match_oracle(N, D, graph, prec, tol, csr):
    """Sparse J beyond one tile (the Moebius ladder, 2 % Erdos-Renyi graphs): in FP32/FP64,
    and in BF16 mode for the very sparse large ones, the product runs over the nonzeros on
    the CUDA cores (elsewhere on the tensor cores); states match the oracle's dense
    integration, energies exactly."""
    J = _sparse_graph(graph, N, 77 + N)
    ctx = chym.Context(J, D)
    assert ctx.sparse and ctx.uses_csr(prec) == csr
    n_h, reps, steps = 3, 5, 60
    h = inputs.pump_grid(0.5, n_h)
    seeds = inputs.run_seeds(5 + N, n_h * reps)
    prm = chym.Params(eps=0.5 / ctx.lambda_max(), prec=prec)
    sch = chym.Schedule(1, steps // 2, steps)
    ctx.run(prm, h, seeds, steps, sch)
    X, k = ctx.get_state()
    assert k == steps
    Xo = O.run(J, D, inputs.h_per_run(h, reps), seeds, oracle_params(prm), oracle_schedule(sch), steps)
    assert _rel_err(X, Xo) <= tol
    E = ctx.energy()
    assert np.array_equal(E, O.ising_energies(J, O.readout(X)))
    ctx.close()


def test_sparse_graph_too_large_for_the_simt_kernel_stays_on_the_tensor_cores():
    """A very sparse J whose run state (2 N D floats) exceeds the SIMT kernel's shared
    memory (Moebius ladder N = 4096, D = 8: 256 KiB a run) keeps the BF16 hi+lo product
    on the tensor cores instead of failing on the compressed-row kernel."""
    N, D = 4096, 8
    J = inputs.mobius_ladder(N)
    ctx = chym.Context(J, D)
    assert ctx.sparse and not ctx.uses_csr(chym.PREC_BF16X2)
    n_h, reps, steps = 1, 2, 6
    h = inputs.pump_grid(0.5, n_h)
    seeds = inputs.run_seeds(41, n_h * reps)
    prm = chym.Params(eps=0.5 / ctx.lambda_max(), prec=chym.PREC_BF16X2)
    sch = chym.Schedule(1, 2, 8)
    ctx.run(prm, h, seeds, steps, sch)
    X, k = ctx.get_state()
    assert k == steps
    Xo = O.run(J, D, inputs.h_per_run(h, reps), seeds, oracle_params(prm), oracle_schedule(sch), steps)
    assert _rel_err(X, Xo) <= 1e-4
    assert np.array_equal(ctx.energy(), O.ising_energies(J, O.readout(X)))
    ctx.close()


def test_batch_with_sparse_dense_and_small_contexts_equals_them_alone():
    """A batch mixing a sparse large context (CUDA-core product), a dense large one (the
    persistent tensor-core kernel) and a small one gives each the states it has alone."""
    specs = [(inputs.mobius_ladder(1024), 3), (inputs.sk_pm1(200, 9), 2), (inputs.sk_pm1(64, 10), 4)]
    steps = 48

    def make():
        out = []
        for k, (J, D) in enumerate(specs):
            c = chym.Context(J, D)
            prm = chym.Params(eps=0.5 / c.lambda_max(), prec=chym.PREC_BF16X2)
            sch = chym.Schedule(1, 20, 60)
            c.run(prm, inputs.pump_grid(0.5, 2), inputs.run_seeds(31 + k, 12), 0, sch)
            out.append((c, prm, sch))
        return out

    batched = make()
    assert [c.uses_csr(p.prec) for c, p, _ in batched] == [True, False, False]
    b = chym.Batch([c for c, _, _ in batched])
    b.run([p for _, p, _ in batched], [s for _, _, s in batched], steps)
    b.status()
    b.close()
    alone = make()
    for (c, p, s), (ca, _, _) in zip(alone, batched):
        c.run(p, None, None, steps, s)
        assert np.array_equal(c.get_state()[0], ca.get_state()[0])
        c.close()
        ca.close()
