"""The CHYM as the paper's discrete round-trip map (Eq. 1, Eq. 2 and the output
coupler after Eq. 2), run on the same kernels as the Euler-Maruyama equations.

One round trip of the cavity takes the PO fields A (hyperspin p, component mu) to

    A' = (1 - d) [ a K A + b K (J (x) 1_D) A - b^2 beta K^3 |A_p|^2 A ]      (a + b = 1)

with K the parametric gain of the nonlinear medium: B = K A, the FPGA feedback of
Eq. 1 with the nonlinear loss W = beta 1_N (x) I_D (its row sum over a hyperspin is
beta |B_p|^2), the coupler recombination of Eq. 2 and the output coupler.  That is
one Euler step with dt = 1 of the hyperspin equations with

    h = (1 - d) a K,   eps = (1 - d) b K,   gamma = (1 - d) b^2 beta K^3,   kappa = 0,

no annealing (alpha_mu = 1) and the step noise sigma sqrt(dt) xi = sigma xi added to
the next field.  The gain K follows the pump; the supplement that gives K(h) is not
part of the paper, so K is an input: a pump scan is a scan over K, one context per
gain value (eps and gamma are per-context constants of the kernels), and a batch
integrates all of them in one launch per dimension.
"""
from dataclasses import dataclass

import numpy as np

from . import chym, inputs


@dataclass
class Cavity:
    """Couplers of Fig. 1: a = 1 - b (CC2 transmission, b the CC1 extraction), d the
    output-coupler fraction, beta the rescaling of the nonlinear loss W."""
    a: float = 0.95
    d: float = 0.1
    beta: float = 1.0

    @property
    def b(self):
        return 1.0 - self.a

    def euler(self, K, sigma=0.0, init_std=0.1, prec=chym.PREC_BF16X2):
        """(Params, pump value h) of the Euler step that equals one round trip at gain K."""
        g = (1.0 - self.d) * K
        prm = chym.Params(dt=1.0, sigma=sigma, init_std=init_std, kappa=0.0, eps=g * self.b,
                          gamma=g * self.b * self.b * self.beta * K * K, prec=prec)
        return prm, g * self.a

    def threshold(self, lam_max):
        """Gain at which the zero field turns unstable through the top eigenmode of J
        (linear part (1 - d) K (a + b lambda)), for a + b lambda_max >= |a + b lambda_min|."""
        return 1.0 / ((1.0 - self.d) * (self.a + self.b * lam_max))


NO_ANNEALING = chym.Schedule(0, 0, 0)


def contexts(J, D, cav: Cavity, gains, replicas, seed, sigma=0.0, init_std=0.1,
             prec=chym.PREC_BF16X2, stream=0):
    """One context per gain value, each with `replicas` runs initialised from its own
    seeds (round trip 0).  Returns (contexts, params)."""
    ctxs, prms = [], []
    for i, K in enumerate(gains):
        ctx = chym.Context(J, D)
        prm, h = cav.euler(float(K), sigma, init_std, prec)
        ctx.run(prm, np.array([h]), inputs.run_seeds(seed + 7919 * i, replicas), 0, NO_ANNEALING,
                stream)
        ctxs.append(ctx)
        prms.append(prm)
    return ctxs, prms


def run(J, D, cav: Cavity, gains, replicas, round_trips, seed=1, sigma=0.0, init_std=0.1,
        prec=chym.PREC_BF16X2, stream=0):
    """Every gain value's replicas for `round_trips` round trips in one batch.  Returns
    the per-gain Ising energies of the sign readout, shape (len(gains), replicas)."""
    ctxs, prms = contexts(J, D, cav, gains, replicas, seed, sigma, init_std, prec, stream)
    try:
        batch = chym.Batch(ctxs)
        try:
            batch.run(prms, [NO_ANNEALING] * len(ctxs), round_trips, stream)
            batch.status()
        finally:
            batch.close()
        return np.stack([c.energy(stream=stream) for c in ctxs])
    finally:
        for c in ctxs:
            c.close()
