"""Shared helpers of the test suite: build the same seeded inputs for both sides."""
import numpy as np

import oracle.oracle as O
from paper_2308_02329_gb300 import inputs


def make_case(N, D, n_h, reps, seed, graph="sk", eps_hat=0.5):
    """Coupling matrix, eps, pump grid and run seeds of one synthetic case."""
    if graph == "sk":
        J = inputs.sk_pm1(N, seed)
    elif graph == "gauss":
        J = inputs.gaussian(N, seed)
    elif graph == "mobius":
        J = inputs.mobius_ladder(N)
    elif graph == "sparse":
        J = inputs.sparse_pm1(N, 0.2, seed)
    else:
        raise ValueError(graph)
    lam = float(np.linalg.eigvalsh(J)[-1]) if N > 1 else 1.0
    lam = lam if lam > 0 else 1.0
    eps = eps_hat / lam
    h = inputs.pump_grid(1.0 - eps_hat, n_h)
    seeds = inputs.run_seeds(seed, n_h * reps)
    return J, eps, h, seeds


def oracle_params(p):
    return O.Params(dt=p.dt, sigma=p.sigma, init_std=p.init_std, gamma=p.gamma, kappa=p.kappa,
                    eps=p.eps)


def oracle_schedule(s):
    return O.Schedule(kind=s.kind, k_anneal=s.k_anneal, k_total=s.k_total)


def rel_err(a, b):
    """Largest |a - b| relative to the scale of its own (run, component): for states laid
    out X[run, p, mu] the scale is max_p |b[run, :, mu]|, floored at 1e-12 of the whole
    array's scale, so that the components annealing drives towards zero are held to the
    same relative tolerance as the surviving one.  Other shapes: max |a - b| / max |b|."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    glob = max(float(np.max(np.abs(b))) if b.size else 0.0, 1e-300)
    if b.ndim == 3 and b.size:
        scale = np.maximum(np.max(np.abs(b), axis=1, keepdims=True), 1e-12 * glob)
        return float(np.max(np.abs(a - b) / scale))
    return float(np.max(np.abs(a - b))) / glob if b.size else 0.0
