"""The discrete round-trip map of the cavity (Eq. 1, Eq. 2, output coupler).

CPU: the literal map of the oracle against the closed-form fixed point of one
hyperspin, the threshold gain from the spectrum of J, and the Euler step that the
package's reduction maps it to.  GPU: the kernels in map mode (batch of gain values)
against the literal map, FP64 and BF16 hi+lo, small-N and large-N paths.
"""
import numpy as np
import pytest

import oracle.oracle as O
import oracle.round_trip as RT
from paper_2308_02329_gb300 import chym, inputs
from paper_2308_02329_gb300 import round_trip as M
from tests.helpers import oracle_params, oracle_schedule, rel_err

CAV = M.Cavity(a=0.95, d=0.1, beta=1.3)


def test_single_hyperspin_fixed_point():
    """J = 0, one hyperspin: the map is radial, r' = g r (a - c r^2) with g = (1 - d) K and
    c = b^2 beta K^2, so the field keeps its direction and settles at
    r*^2 = (g a - 1) / (g c), stable for 1 < g a < 2."""
    a, d, beta = CAV.a, CAV.d, CAV.beta
    b = 1.0 - a
    J = np.zeros((1, 1))
    for D, ga in ((1, 1.3), (3, 1.5), (5, 1.8)):
        K = ga / ((1.0 - d) * a)
        g, c = (1.0 - d) * K, b * b * beta * K * K
        A0 = O.init_state(1, D, np.array([11 + D], dtype=np.uint64), 0.05)
        A = RT.run(J, D, a, d, beta, K, [11 + D], 3000, A0=A0)
        r2 = (g * a - 1.0) / (g * c)
        assert abs(np.sum(A[0] ** 2) / r2 - 1.0) < 1e-12
        u0, u = A0[0].ravel(), A[0].ravel()
        assert np.allclose(u / np.linalg.norm(u), u0 / np.linalg.norm(u0), atol=1e-14)
    # below the single-oscillator threshold (g a < 1) the field dies out
    K = 0.9 / ((1.0 - d) * a)
    A = RT.run(J, 3, a, d, beta, K, [5], 400, init_std=0.1)
    assert np.max(np.abs(A)) < 1e-15


@pytest.mark.parametrize("D", [1, 2, 4])
def test_threshold_gain_from_the_spectrum(D):
    """The zero field of the coupled map turns unstable at K_th = 1/((1-d)(a + b lambda_max)):
    a small field decays below it and grows above it, and the growth rate per round trip
    approaches (1 - d) K (a + b lambda_max)."""
    J = inputs.sk_pm1(16, 3)
    lam = float(np.linalg.eigvalsh(J)[-1])
    K_th = RT.threshold_gain(J, CAV.a, CAV.d)
    assert K_th == pytest.approx(CAV.threshold(lam), rel=1e-14)
    seeds = [21, 22]
    lo = RT.run(J, D, CAV.a, CAV.d, CAV.beta, 0.97 * K_th, seeds, 900, init_std=1e-8)
    hi = RT.run(J, D, CAV.a, CAV.d, CAV.beta, 1.03 * K_th, seeds, 300, init_std=1e-8)
    n0 = np.linalg.norm(O.init_state(16, D, np.array(seeds, dtype=np.uint64), 1e-8), axis=(1, 2))
    assert np.all(np.linalg.norm(lo, axis=(1, 2)) < 1e-3 * n0)
    assert np.all(np.linalg.norm(hi, axis=(1, 2)) > 1e3 * n0)
    # linear regime: the ratio of successive norms tends to the top growth factor
    a1 = RT.run(J, D, CAV.a, CAV.d, CAV.beta, 1.03 * K_th, seeds, 401, init_std=1e-15)
    a0 = RT.run(J, D, CAV.a, CAV.d, CAV.beta, 1.03 * K_th, seeds, 400, init_std=1e-15)
    rate = np.linalg.norm(a1, axis=(1, 2)) / np.linalg.norm(a0, axis=(1, 2))
    assert np.allclose(rate, 1.03, rtol=1e-3)


@pytest.mark.parametrize("sigma", [0.0, 1e-3])
def test_reduction_to_the_euler_step(sigma):
    """The package's reduction (dt = 1, h = (1-d) a K, eps = (1-d) b K,
    gamma = (1-d) b^2 beta K^3, kappa = 0, no annealing) integrated by the oracle's Euler
    stepper equals the literal map, noise included."""
    J = inputs.sk_pm1(12, 5)
    K = 1.15 * RT.threshold_gain(J, CAV.a, CAV.d)
    seeds = inputs.run_seeds(9, 3)
    for D in (1, 3):
        prm, h = CAV.euler(K, sigma=sigma, init_std=0.1, prec=chym.PREC_FP64)
        X = O.run(J, D, np.full(3, h), seeds, oracle_params(prm), oracle_schedule(M.NO_ANNEALING), 80)
        A = RT.run(J, D, CAV.a, CAV.d, CAV.beta, K, seeds, 80, init_std=0.1, sigma=sigma)
        assert np.max(np.abs(X - A)) <= 1e-12 * max(1.0, np.max(np.abs(A)))
        assert np.max(np.abs(A)) > 0.05   # above threshold: the fields did not die out


def _map_on_gpu(J, D, gains, replicas, trips, prec, sigma, seed=3):
    ctxs, prms = M.contexts(J, D, CAV, gains, replicas, seed, sigma=sigma, prec=prec)
    batch = chym.Batch(ctxs)
    batch.run(prms, [M.NO_ANNEALING] * len(ctxs), trips)
    batch.status()
    batch.close()
    out = []
    for i, (ctx, K) in enumerate(zip(ctxs, gains)):
        X, k = ctx.get_state()
        assert k == trips
        A = RT.run(J, D, CAV.a, CAV.d, CAV.beta, K, inputs.run_seeds(seed + 7919 * i, replicas),
                   trips, init_std=0.1, sigma=sigma)
        out.append((X, A, ctx.energy()))
        ctx.close()
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("N,D,prec,trips,tol", [
    (20, 3, chym.PREC_FP64, 60, 1e-10),
    (37, 8, chym.PREC_FP64, 40, 1e-10),
    (45, 2, chym.PREC_FP32, 30, 1e-4),      # SIMT FP32 path
    (100, 4, chym.PREC_BF16X2, 30, 1e-4),   # small-N tensor-core path
    (61, 1, chym.PREC_BF16X2, 30, 1e-4),    # the CIM as a map (D = 1)
    (150, 2, chym.PREC_BF16X2, 30, 1e-4),   # large-N tensor-core path
])
def test_map_mode_matches_the_literal_map(N, D, prec, trips, tol):
    """Kernels in map mode (three gains around threshold, one batch) against the literal
    map of Eq. 1 and Eq. 2, relative per (run, component).  FP64: 1e-10.  FP32: 30 trips of
    FP32 rounding (2^-24 each, a few operations deep) stay far below 1e-4.  BF16 hi+lo:
    x = hi + lo + r with |r| <= 2^-18 |x| (two round-to-nearest BF16 steps), and J = +-1 is
    exact, so a trip's coupling term eps J x is off by eps sum_q J_pq r_q: independent
    roundings of about 2^-18 |x| over N terms, i.e. about eps sqrt(N) 2^-18 |x|
    (eps N <= 3 at these gains, so about 1e-6 |x| at N = 100).  The map contracts around
    its fixed points at these gains, so the errors of 30 trips add up to at most
    30 times that, 3e-5; the test takes 1e-4, the mixed-precision bound."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    J = inputs.sk_pm1(N, 17)
    K_th = CAV.threshold(float(np.linalg.eigvalsh(J)[-1]))
    gains = [0.9 * K_th, 1.05 * K_th, 1.15 * K_th]
    for X, A, E in _map_on_gpu(J, D, gains, 5, trips, prec, sigma=1e-3):
        assert np.all(np.isfinite(X))
        scale = max(np.max(np.abs(A)), 1e-300)
        assert rel_err(X, A) <= tol
        s = np.where(A[:, :, 0] >= 0, 1, -1).astype(np.int8)
        sure = np.all(np.abs(A[:, :, 0]) > 1e-2 * scale, axis=1)   # no sign within rounding
        Eo = O.ising_energies(J, s)
        assert np.array_equal(E[sure], Eo[sure])
