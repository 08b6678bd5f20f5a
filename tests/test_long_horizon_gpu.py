"""Long-horizon statistical parity of the GPU path with the FP64 oracle.

Over thousands of steps the noise-driven dynamics is chaotic: the same seeds lead
the GPU and the oracle to different final states once rounding differences have
grown, so states are no longer compared.  What must agree is the statistics the
paper reports (text before Fig. 4 and the figures of merit after Fig. 3): the
success probability P_Ising(h) of reaching the lowest energy, per pump value, and
the mean energy above it.  Each test integrates the same seeded runs on both sides
over the full schedule and checks
  * P_Ising per pump, and pooled over the pumps, within the two-sample binomial 95 %
    interval, 1.96 sqrt(2 max(p(1-p), 1/R) / R) for R runs per side;
  * the mean of E - E_ref within 1.96 two-sample standard errors,
where E_ref is the lowest energy either side reached (the exact ground state where
one is known).  Sharing the seeds correlates the two samples, which only makes the
intervals conservative.
"""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2308_02329_gb300 import chym, inputs
from tests.helpers import make_case, oracle_params, oracle_schedule

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chym.lib()


def _agree(E, Eo, n_h, reps, E_ref, real_j=False):
    E, Eo = np.asarray(E), np.asarray(Eo)
    assert np.all(np.isfinite(E)) and np.all(np.isfinite(Eo))
    tol = 1e-9 * abs(E_ref) if real_j else 0.0
    assert E.min() >= E_ref - tol and Eo.min() >= E_ref - tol
    hit, hit_o = np.abs(E - E_ref) <= tol, np.abs(Eo - E_ref) <= tol

    def close(p, q, r):
        return abs(p - q) <= 1.96 * np.sqrt(max(p * (1 - p), q * (1 - q), 1.0 / r) * 2.0 / r) + 1e-12

    for p, q in zip(hit.reshape(n_h, reps).mean(1), hit_o.reshape(n_h, reps).mean(1)):
        assert close(p, q, reps)
    assert close(hit.mean(), hit_o.mean(), hit.size)
    d, do = E - E_ref, Eo - E_ref
    se = np.sqrt(d.var() / d.size + do.var() / do.size)
    assert abs(d.mean() - do.mean()) <= 1.96 * se + 1e-9 * max(1.0, abs(E_ref))
    return hit.mean(), hit_o.mean(), d.mean(), do.mean()


@pytest.mark.parametrize("D", [3, 4])
def test_sk100_bf16_full_schedule(D):
    """SK +-1 N = 100 (the benchmark's instance and constants), BF16 hi+lo on the
    small-N tensor-core kernel, 8 pumps x 32 replicas, the full 20000 steps with
    dimensional annealing over the second half."""
    N, n_h, reps, K = 100, 8, 32, 20000
    J, eps, h, seeds = make_case(N, D, n_h, reps, 0xC0FFEE + 1)
    ctx = chym.Context(J, D)
    prm = chym.Params(eps=eps, prec=chym.PREC_BF16X2)
    sch = chym.Schedule(1, K // 2, K)
    ctx.run(prm, h, seeds, K, sch)
    E = ctx.energy()
    ctx.close()
    Xo = O.run(J, D, inputs.h_per_run(h, reps), seeds, oracle_params(prm), oracle_schedule(sch), K)
    Eo = O.ising_energies(J, O.readout(Xo))
    print(f"sk100 D={D}:", _agree(E, Eo, n_h, reps, min(E.min(), Eo.min())))


@pytest.mark.parametrize("N,D,graph,prec", [(256, 3, "sk", chym.PREC_BF16X2), (200, 4, "gauss", chym.PREC_BF16X2),
                                             (256, 3, "sk", chym.PREC_FP8)])
def test_large_n_path_long_horizon(N, D, graph, prec):
    """The persistent large-N tensor-core kernel (N > 128) over 6000 steps, annealed
    over the second half: SK +-1 (hi+lo products, BF16 and FP8 lo) and Gaussian J (three
    products, energies in FP64), 4 pumps x 32 replicas."""
    n_h, reps, K = 4, 32, 6000
    J, eps, h, seeds = make_case(N, D, n_h, reps, 0x1A26E + N, graph)
    real = graph == "gauss"
    ctx = chym.Context(J, D, chym.J_REAL if real else chym.J_PM1)
    prm = chym.Params(eps=eps, prec=prec)
    sch = chym.Schedule(1, K // 2, K)
    ctx.run(prm, h, seeds, K, sch)
    E = ctx.energy()
    ctx.close()
    Xo = O.run(J, D, inputs.h_per_run(h, reps), seeds, oracle_params(prm), oracle_schedule(sch), K)
    Eo = O.ising_energies(J, O.readout(Xo))
    print(f"large N={N} D={D} {graph} prec={prec}:", _agree(E, Eo, n_h, reps, min(E.min(), Eo.min()), real))


@pytest.mark.parametrize("prec", [chym.PREC_BF16X2, chym.PREC_FP8])
def test_large_n_512_statistics(prec):
    """SK +-1 N = 512, D = 4 (the size class of the N = 800 and 1000 workloads, at an
    oracle cost of seconds): 4 pumps x 16 replicas over 3000 steps, annealed over the
    second half; pooled success and mean energy above the best energy reached."""
    N, D, n_h, reps, K = 512, 4, 4, 16, 3000
    J, eps, h, seeds = make_case(N, D, n_h, reps, 0x5120 + prec)
    ctx = chym.Context(J, D)
    prm = chym.Params(eps=eps, prec=prec)
    sch = chym.Schedule(1, K // 2, K)
    ctx.run(prm, h, seeds, K, sch)
    E = ctx.energy()
    ctx.close()
    Xo = O.run(J, D, inputs.h_per_run(h, reps), seeds, oracle_params(prm), oracle_schedule(sch), K)
    Eo = O.ising_energies(J, O.readout(Xo))
    print(f"N=512 prec={prec}:", _agree(E, Eo, 1, n_h * reps, min(E.min(), Eo.min())))


def test_uneven_batch_instances_full_schedule():
    """Instances of the batched uneven workload (SK +-1, 16 pumps x 4 replicas each, the
    benchmark's constants: D = 2 as the XY machine without annealing, D >= 3 annealed
    over the second half), integrated together as one batch over the full 30000 steps:
    one instance per D in {2, 3, 4, 8} among the smallest, one of them beyond one
    tensor-core tile.  Statistics are pooled per instance (4 replicas per pump are too
    few for per-pump intervals)."""
    comp = inputs.uneven_instances(512, 0xC0FFEE + 4)
    pick = {}
    for N, D, seed in sorted(comp):   # the smallest of each D; for D = 3 the smallest N > 128
        if D not in pick and (N > 128 or D != 3):
            pick[D] = (N, D, seed)
    assert sorted(pick) == [2, 3, 4, 8] and any(v[0] > 128 for v in pick.values())
    n_h, reps, K = 16, 4, 30000
    ctxs, jobs = [], []
    for N, D, seed in pick.values():
        J = inputs.sk_pm1(N, seed)
        c = chym.Context(J, D)
        kappa, skind = (1e-3, 0) if D == 2 else (0.1, 1)
        prm = chym.Params(eps=0.5 / c.lambda_max(), kappa=kappa, prec=chym.PREC_BF16X2)
        sch = chym.Schedule(skind, K // 2 if skind else 0, K)
        h = inputs.pump_grid(0.5, n_h)
        seeds = inputs.run_seeds(seed + D, n_h * reps)
        c.run(prm, h, seeds, 0, sch)
        ctxs.append(c)
        jobs.append((J, N, D, prm, sch, h, seeds))
    batch = chym.Batch(ctxs)
    batch.run([j[3] for j in jobs], [j[4] for j in jobs], K)
    batch.status()
    batch.close()
    for c, (J, N, D, prm, sch, h, seeds) in zip(ctxs, jobs):
        E = c.energy()
        c.close()
        Xo = O.run(J, D, inputs.h_per_run(h, reps), seeds, oracle_params(prm), oracle_schedule(sch), K)
        Eo = O.ising_energies(J, O.readout(Xo))
        print(f"uneven N={N} D={D}:", _agree(E, Eo, 1, n_h * reps, min(E.min(), Eo.min())))
