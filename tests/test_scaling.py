"""Scaling study of the success probability with N (Fig. 4): host aggregation and
fit on CPU, and a small study on the GPU checked against the oracle's figures."""
import math

import numpy as np
import pytest

import oracle.oracle as O
import oracle.stats as OS
from paper_2308_02329_gb300 import inputs
from paper_2308_02329_gb300 import scaling as SC


def test_fit_exponential_recovers_the_decay_rate():
    Ns = np.arange(10, 110, 10)
    P = np.exp(1.5 - 0.037 * Ns)
    a, c, used = SC.fit_exponential(Ns, P)
    assert used == len(Ns)
    assert abs(a - 0.037) < 1e-12 and abs(c - 1.5) < 1e-10
    P[3] = 0.0    # a size without any success is left out of the fit
    a2, _, used2 = SC.fit_exponential(Ns, P)
    assert used2 == len(Ns) - 1 and abs(a2 - 0.037) < 1e-12
    assert SC.fit_exponential([10, 20], [0.5, 0.0])[0] is None


def test_aggregate_means_and_quartiles():
    rng = np.random.default_rng(0)
    rows = []
    for N in (10, 20):
        for g in range(7):
            v = rng.random(4)
            rows.append(SC.GraphResult(N, g, -float(N), True, v[0], v[1], v[2], v[3]))
    agg = SC.aggregate(rows)
    assert sorted(agg) == [10, 20]
    for N in (10, 20):
        v = np.array([r.P_max for r in rows if r.N == N])
        q = np.percentile(v, [25, 50, 75])
        assert agg[N]["graphs"] == 7 and agg[N]["exact_gs"]
        assert math.isclose(agg[N]["P_max"]["mean"], v.mean())
        assert [agg[N]["P_max"][k] for k in ("q25", "median", "q75")] == pytest.approx(list(q))


def test_graph_set_is_seeded_and_distinct():
    a = SC.graph_set([10, 20], 3)
    assert a == SC.graph_set([10, 20], 3)
    assert len({s for _, _, s in a}) == len(a)
    J = inputs.sparse_pm1(20, 0.2, a[3][2])
    assert np.array_equal(J, J.T) and not np.any(np.diag(J))


@pytest.mark.gpu
def test_small_study_matches_oracle_figures():
    """Both machines on 3 graphs of N = 8 and 12: exact ground states agree with the
    oracle's exhaustive search, and every graph's figures of merit equal the oracle's
    figures computed from the same run energies."""
    from paper_2308_02329_gb300 import chym
    Ns, n_graphs, n_h, reps, steps = (8, 12), 3, 5, 8, 400
    for mode in ("cim", "chym_da"):
        rows = SC.run(Ns, mode, n_graphs, n_h, reps, steps)
        assert len(rows) == len(Ns) * n_graphs
        for r, (N, g, gseed) in zip(rows, SC.graph_set(Ns, n_graphs)):
            assert (r.N, r.graph) == (N, g) and r.exact
            J = inputs.sparse_pm1(N, 0.2, gseed)
            assert r.E_gs == O.ground_state_bruteforce(J)[0]
            assert 0.0 <= r.P_max <= 1.0 and 0.0 <= r.W_range <= 1.0 and r.W_scan <= r.W_range + 1e-12
            assert sum(r.hits_per_h) <= n_h * reps
            # the same graph alone, same seeds: energies -> the oracle's figures
            ctx = chym.Context(J, SC.MODES[mode]["D"])
            prm, sched = SC.params_for(mode, ctx.lambda_max(), steps)
            h = inputs.pump_grid(0.5, n_h)
            ctx.run(prm, h, inputs.run_seeds(gseed, n_h * reps), steps, sched)
            f = OS.figures_of_merit(ctx.energy(), r.E_gs, n_h)
            ctx.close()
            assert r.hits_per_h == [int(v) for v in f["hits"]]
            assert math.isclose(r.P_max, f["P_max"]) and math.isclose(r.W_range, f["W_range"])
            assert math.isclose(r.W_scan, f["W_scan"]) and math.isclose(r.dE_mean, f["dE_mean"])
    res = SC.study(Ns, n_graphs, steps, n_h=n_h, reps=reps)
    for mode in ("cim", "chym_da"):
        assert sorted(res[mode]["per_N"]) == list(Ns)
