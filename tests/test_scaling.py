"""Scaling study of the success probability with N (Fig. 4): host aggregation and
fit on CPU, and a small study on the GPU checked against the oracle's figures."""
import math

import numpy as np
import pytest

import oracle.oracle as O
import oracle.stats as OS
from paper_2308_02329_gb300 import inputs
from paper_2308_02329_gb300 import chym, packing
from paper_2308_02329_gb300 import scaling as SC
from tests.helpers import oracle_params, oracle_schedule


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


def test_packing_plan_and_blocks():
    """First-fit decreasing: every graph in exactly one bin, no bin above 128 spins, bins
    in decreasing-size order; the block-diagonal J holds each graph on its diagonal block
    and nothing else, and the per-spin weights repeat one value per block."""
    rng = np.random.default_rng(3)
    sizes = list(rng.integers(5, 101, size=60)) + [128, 1]
    bins = packing.plan(sizes)
    assert sorted(i for b in bins for i in b) == list(range(len(sizes)))
    assert all(sum(sizes[i] for i in b) <= 128 for b in bins)
    assert all([sizes[i] for i in b] == sorted((sizes[i] for i in b), reverse=True) for b in bins)
    assert len(bins) <= 2 * int(np.ceil(sum(sizes) / 128))     # first fit is within 2x of optimal
    Js = [inputs.sparse_pm1(int(n), 0.2, 100 + k) for k, n in enumerate((7, 12, 30))]
    P = packing.build(Js, [2, 0, 1])
    assert P.seg_begin.tolist() == [0, 30, 37, 49] and P.N == 49
    for b, i in enumerate(P.members):
        lo, hi = P.seg_begin[b], P.seg_begin[b + 1]
        assert np.array_equal(P.J[lo:hi, lo:hi], Js[i])
        P.J[lo:hi, lo:hi] = 0.0
    assert not np.any(P.J)
    assert packing.spin_weights(P, [1.0, 2.0, 3.0]).tolist() == [1.0] * 30 + [2.0] * 7 + [3.0] * 12


def test_host_figures_match_the_oracle():
    """The study's per-graph figures from run energies equal the oracle's definitions,
    NaN (diverged) runs included."""
    rng = np.random.default_rng(5)
    for n_h, reps in ((7, 9), (1, 30), (21, 32)):
        E = -4.0 * rng.integers(8, 12, size=n_h * reps).astype(np.float64)
        E[rng.random(E.size) < 0.05] = np.nan
        E_gs = -44.0
        f = SC.figures(E, E_gs, n_h)
        g = OS.figures_of_merit(E, E_gs, n_h)
        assert f["hits"].tolist() == [int(v) for v in g["hits"]]
        for k in ("P_max", "W_range", "W_scan", "dE_mean"):
            assert math.isclose(f[k], g[k], rel_tol=1e-12, abs_tol=1e-15), k


@pytest.mark.gpu
def test_small_study_matches_oracle_figures():
    """Both machines on 3 graphs of N = 8 and 12 each, all six packed into one context,
    FP64: every graph's figures of merit equal the oracle's figures from the oracle's
    own integration of the packed system (J' = diag(w) J with the per-graph weights), and
    the exact ground states equal the oracle's exhaustive search."""
    Ns, n_graphs, n_h, reps, steps = (8, 12), 3, 5, 8, 400
    graphs = SC.graphs_and_references(Ns, n_graphs)
    for (N, g, gseed, J, lam, E_gs, exact), (N2, g2, s2) in zip(graphs, SC.graph_set(Ns, n_graphs)):
        assert (N, g, gseed) == (N2, g2, s2) and exact
        assert E_gs == O.ground_state_bruteforce(J)[0]
        assert lam == pytest.approx(float(np.linalg.eigvalsh(J)[-1]), rel=1e-9)
    for mode in ("cim", "chym_da"):
        rows = SC.run(Ns, mode, n_graphs, n_h, reps, steps, prec=chym.PREC_FP64, graphs=graphs)
        jobs = SC.pack_contexts(graphs, mode, n_h, reps, steps, prec=chym.PREC_FP64)
        assert len(jobs) == 1 and sorted(jobs[0][3].members) == list(range(len(graphs)))
        for ctx, prm, sched, P, seeds, w in jobs:
            ctx.close()
            Jp = P.J if w is None else w[:, None] * P.J
            X = O.run(Jp, SC.MODES[mode]["D"], inputs.h_per_run(inputs.pump_grid(0.5, n_h), reps),
                      seeds, oracle_params(prm), oracle_schedule(sched), steps)
            for b, i in enumerate(P.members):
                lo, hi = P.seg_begin[b], P.seg_begin[b + 1]
                Eo = O.ising_energies(graphs[i][3], O.readout(X[:, lo:hi, :]))
                f = OS.figures_of_merit(Eo, graphs[i][5], n_h)
                r = rows[i]
                assert (r.N, r.graph, r.E_gs) == (graphs[i][0], graphs[i][1], graphs[i][5])
                assert r.hits_per_h == [int(v) for v in f["hits"]]
                assert math.isclose(r.P_max, f["P_max"]) and math.isclose(r.W_range, f["W_range"])
                assert math.isclose(r.W_scan, f["W_scan"]) and math.isclose(r.dE_mean, f["dE_mean"])
    res = SC.study(Ns, n_graphs, steps, n_h=n_h, reps=reps)
    for mode in ("cim", "chym_da"):
        assert sorted(res[mode]["per_N"]) == list(Ns)


@pytest.mark.gpu
def test_study_with_graphs_above_one_tile():
    """Graphs above 128 spins get a context each (no weights, large-N tensor-core path) and
    mixed sizes pack around them; every graph gets its figures."""
    rows = SC.run((150, 40, 90), "chym_da", 2, 3, 4, 120)
    assert [(r.N, r.graph) for r in rows] == [(N, g) for N in (150, 40, 90) for g in range(2)]
    for r in rows:
        assert np.isfinite(r.E_gs) and 0.0 <= r.P_max <= 1.0 and len(r.hits_per_h) == 3
