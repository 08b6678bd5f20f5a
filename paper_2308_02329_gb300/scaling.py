"""Scaling of the success probability with the problem size (Fig. 4 and the text
around it): the coherent Ising machine (D = 1) against the hyperspin machine with
dimensional annealing (D = 2 annealed back to 1), on random sparse +-1 graphs of
growing N.

Per graph, the figures of merit of the text after Fig. 3 come from its run
energies: the best success probability over the pump scan P_max, the pump-range
weight W and the mean energy gap dE.  Graphs of up to 128 spins in total share a
context as blocks of a block-diagonal J (`packing`), so the small graphs of the scan
fill the 128 lanes of the tensor-core tile instead of one graph per tile.  Per size N they are averaged over
the graphs (with the quartiles that Fig. 4 shades), and the decay of the mean
success probability is fitted as P_max(N) ~ exp(c - a N), the exponent a
measuring how hard the machine finds larger problems.

All integration, energies and statistics run in the CUDA library; this module
builds the seeded inputs, the ground-state references and the aggregates.
"""
import math
from dataclasses import dataclass, field

import numpy as np

from . import chym, inputs, packing

# Machine modes (readings of the text before Fig. 3 and Fig. 4): the CIM has no
# hyperspin loss (gamma = 0) and only the local saturation kappa; CHYM+DA keeps
# beta b^2 = 25 and anneals the second component away over the second half.
MODES = {
    "cim": {"D": 1, "gamma": 0.0, "kappa": 0.1, "anneal": False},
    "chym_da": {"D": 2, "gamma": 25.0, "kappa": 0.1, "anneal": True},
}


@dataclass
class GraphResult:
    N: int
    graph: int
    E_gs: float
    exact: bool
    P_max: float
    W_range: float
    W_scan: float
    dE_mean: float
    hits_per_h: list = field(default_factory=list)


def graph_set(Ns, n_graphs, density=0.2, seed=0x5CA1E):
    """The seeded sparse +-1 graphs: (N, index, seed) for every size and graph."""
    return [(int(N), g, int(seed) * 1000003 + 1009 * int(N) + g) for N in Ns for g in range(n_graphs)]


def ground_state(ctx, exact_max_n=24, restarts=16, sweeps=1000, seed=3):
    """E_GS of a context: exhaustive search up to exact_max_n spins, simulated
    annealing above (a best-known upper bound).  Returns (E, exact)."""
    if ctx.N <= exact_max_n:
        return ctx.ground_state_exact()[0], True
    return ctx.ground_state_search(restarts=restarts, sweeps=sweeps, seed=seed)[0], False


def params_for(mode, lam, steps, eps_hat=0.5, prec=chym.PREC_BF16X2):
    m = MODES[mode]
    prm = chym.Params(dt=0.01, sigma=1e-3, init_std=0.1, gamma=m["gamma"], kappa=m["kappa"],
                      eps=eps_hat / lam if lam > 0 else 0.0, prec=prec)
    sched = chym.Schedule(1, steps // 2, steps) if m["anneal"] else chym.Schedule(0, 0, steps)
    return prm, sched


def figures(E, E_gs, n_h):
    """The figures of merit (text after Fig. 3) of one graph from its run energies
    (h-major runs, as chym_stats counts them): ground-state hits per pump (E == E_GS,
    exact for the integer energies of +-1 couplings; a diverged run's NaN never
    counts), P_max, W normalised by the pumps with P > 0 (W_range) and by all scanned
    pumps (W_scan), and the mean E - E_GS over finite runs."""
    E = np.asarray(E, dtype=np.float64).reshape(n_h, -1)
    hits = np.sum(E == E_gs, axis=1).astype(np.int64)
    P = hits / E.shape[1]
    nz = int(np.count_nonzero(hits))
    fin = np.isfinite(E)
    return {"hits": hits, "P_max": float(P.max()) if n_h else 0.0,
            "W_range": float(P.sum() / nz) if nz else 0.0, "W_scan": float(P.sum() / n_h),
            "dE_mean": float(np.mean(E[fin] - E_gs)) if fin.any() else math.nan,
            "n_hits": int(hits.sum())}


def graphs_and_references(Ns, n_graphs, density=0.2, seed=0x5CA1E, exact_max_n=24):
    """Every graph of the set with lambda_max(J) and its ground-state reference:
    list of (N, index, seed, J, lambda_max, E_GS, exact)."""
    out = []
    for N, g, gseed in graph_set(Ns, n_graphs, density, seed):
        J = inputs.sparse_pm1(N, density, gseed)
        c = chym.Context(J, 1)
        lam = c.lambda_max()
        E_gs, exact = ground_state(c, exact_max_n)
        c.close()
        out.append((N, g, gseed, J, lam, E_gs, exact))
    return out


def pack_contexts(graphs, mode, n_h, reps, steps, eps_hat=0.5, prec=chym.PREC_BF16X2, stream=0,
                  pack=True):
    """Contexts of one machine mode over the graph list, several graphs per context as
    blocks of a block-diagonal J when `pack` (each with its own eps_i through the
    per-spin coupling weights 1 / lambda_max(J_i)), initialised at step 0.  Returns
    a list of (context, params, schedule, packing.Pack, seeds, weights); the params'
    eps is eps_hat, or eps_hat / lambda_max with weights None for a graph alone."""
    m = MODES[mode]
    D = m["D"]
    h = inputs.pump_grid(1.0 - eps_hat, n_h)
    groups = packing.plan([gr[0] for gr in graphs]) if pack else [[i] for i in range(len(graphs))]
    out = []
    for members in groups:
        P = packing.build([gr[3] for gr in graphs], members)
        ctx = chym.Context(P.J, D)
        lam = [graphs[i][4] for i in members]
        w = packing.spin_weights(P, [1.0 / l if l > 0 else 0.0 for l in lam])
        if len(members) > 1:
            ctx.set_coupling_weights(w)
            prm, sched = params_for(mode, 1.0, steps, eps_hat, prec)
        else:   # a graph alone (also one above 128 spins) needs no weights
            w = None
            prm, sched = params_for(mode, lam[0], steps, eps_hat, prec)
        seeds = inputs.run_seeds(graphs[members[0]][2], n_h * reps)
        ctx.run(prm, h, seeds, 0, sched, stream)
        out.append((ctx, prm, sched, P, seeds, w))
    return out


def run(Ns, mode, n_graphs, n_h, reps, steps, density=0.2, seed=0x5CA1E, eps_hat=0.5,
        exact_max_n=24, stream=0, prec=chym.PREC_BF16X2, pack=True, graphs=None):
    """Integrate every graph of every size of one machine mode in one batch (small
    graphs packed several to a context) and return the per-graph figures of merit
    (list of GraphResult, in graph-set order)."""
    graphs = graphs or graphs_and_references(Ns, n_graphs, density, seed, exact_max_n)
    jobs = pack_contexts(graphs, mode, n_h, reps, steps, eps_hat, prec, stream, pack)
    batch = chym.Batch([j[0] for j in jobs])
    try:
        batch.run([j[1] for j in jobs], [j[2] for j in jobs], steps, stream)
        batch.status()
    finally:
        batch.close()
    out = [None] * len(graphs)
    for ctx, _, _, P, _, _ in jobs:
        Eseg = ctx.energy_segments(P.seg_begin, stream)
        for b, i in enumerate(P.members):
            N, g, _, _, _, E_gs, exact = graphs[i]
            E = Eseg[:, b]
            if not exact:   # best known: the search's bound or the best run, whichever is lower
                E_gs = min(E_gs, float(np.nanmin(E)) if np.isfinite(E).any() else E_gs)
            f = figures(E, E_gs, n_h)
            out[i] = GraphResult(N, g, float(E_gs), exact, f["P_max"], f["W_range"], f["W_scan"],
                                 f["dE_mean"], [int(v) for v in f["hits"]])
        ctx.close()
    return out


def aggregate(results):
    """Per size N: the graphs' mean and quartiles (25, 50, 75 %) of P_max, W (both
    normalisations) and dE."""
    by_n = {}
    for r in results:
        by_n.setdefault(r.N, []).append(r)
    out = {}
    for N in sorted(by_n):
        rs = by_n[N]
        row = {"graphs": len(rs), "exact_gs": all(r.exact for r in rs)}
        for key in ("P_max", "W_range", "W_scan", "dE_mean"):
            v = np.array([getattr(r, key) for r in rs], dtype=np.float64)
            v = v[np.isfinite(v)]
            q = np.percentile(v, [25, 50, 75]) if v.size else [math.nan] * 3
            row[key] = {"mean": float(v.mean()) if v.size else math.nan,
                        "q25": float(q[0]), "median": float(q[1]), "q75": float(q[2])}
        out[N] = row
    return out


def fit_exponential(Ns, P):
    """Least-squares fit of ln P = c - a N over the sizes with P > 0; returns
    (a, c, points used).  a is None with fewer than two usable points."""
    Ns = np.asarray(Ns, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    ok = np.isfinite(P) & (P > 0)
    if ok.sum() < 2:
        return None, None, int(ok.sum())
    A = np.stack([np.ones(ok.sum()), -Ns[ok]], axis=1)
    coef, *_ = np.linalg.lstsq(A, np.log(P[ok]), rcond=None)
    return float(coef[1]), float(coef[0]), int(ok.sum())


def study(Ns, n_graphs, steps, modes=("cim", "chym_da"), n_h=None, reps=32, density=0.2,
          seed=0x5CA1E, stream=0):
    """Both machines on the same graphs: per mode the aggregates and the fitted decay
    rate of the mean success probability.  n_h defaults to the paper's scans (51
    pump values for the CIM, 21 for CHYM+DA)."""
    res = {}
    graphs = graphs_and_references(Ns, n_graphs, density, seed)
    for mode in modes:
        nh = n_h or (51 if MODES[mode]["D"] == 1 else 21)
        rows = run(Ns, mode, n_graphs, nh, reps, steps, density, seed, stream=stream, graphs=graphs)
        agg = aggregate(rows)
        a, c, used = fit_exponential(list(agg), [agg[N]["P_max"]["mean"] for N in agg])
        res[mode] = {"n_h": nh, "replicas": reps, "per_N": agg, "decay_a": a, "decay_c": c,
                     "fit_points": used}
    return res
