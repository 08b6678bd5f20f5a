"""Figures of merit of the method (test infrastructure only).

Success probability P_Ising(h), energy histogram H_E, and the three figures of
merit of the finite-size analysis: P_Ising,max, W and Delta E (the definitions
(i)-(iii) following Fig. 3).  Runs are laid out h-major: run = ih * replicas + rep.
"""
import numpy as np


def hits_per_h(E, E_gs, n_h, real_j=False, rel_tol=1e-9):
    """Per pump value, the number of replicas whose final Ising energy equals E_GS.

    Integer couplings compare exactly; real couplings within rel_tol * |E_GS|.
    Non-finite energies (a diverged run) never count.
    """
    E = np.asarray(E, dtype=np.float64).reshape(n_h, -1)
    if real_j:
        hit = np.isfinite(E) & (np.abs(E - E_gs) <= rel_tol * abs(E_gs))
    else:
        hit = np.isfinite(E) & (E == E_gs)
    return hit.sum(axis=1).astype(np.int64)


def figures_of_merit(E, E_gs, n_h, real_j=False):
    """Return dict with P(h), P_max, W (|Delta h| and N_s normalisations) and Delta E."""
    E = np.asarray(E, dtype=np.float64)
    hits = hits_per_h(E, E_gs, n_h, real_j)
    reps = E.size // n_h
    P = hits / reps
    P_max = float(P.max()) if n_h else 0.0
    nonzero = P > 0
    W_range = float(P[nonzero].sum() / nonzero.sum()) if nonzero.any() else 0.0
    W_scan = float(P.sum() / n_h) if n_h else 0.0
    ok = np.isfinite(E)
    dE = float(np.mean(E[ok] - E_gs)) if ok.any() else float("nan")
    return {"hits": hits, "P": P, "P_max": P_max, "W_range": W_range,
            "W_scan": W_scan, "dE_mean": dE}


def energy_histogram(E):
    """H_E: distinct final Ising energies and how often each was reached."""
    E = np.asarray(E, dtype=np.float64)
    E = E[np.isfinite(E)]
    levels, counts = np.unique(E, return_counts=True)
    return levels, counts.astype(np.int64)
