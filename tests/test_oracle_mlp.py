"""CPU pins of the FP64 early-exit reference: finite differences of the loss, the
GELU closed form, Adam on a quadratic, and feature special cases."""
import math

import numpy as np
import pytest

import oracle.mlp as M
import oracle.oracle as O
from paper_2308_02329_gb300 import inputs


def _rand_theta(rng, scale=0.3):
    return rng.standard_normal(M.N_PARAMS) * scale


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = _rand_theta(rng)
    F = rng.standard_normal((7, M.N_FEAT))
    y = rng.integers(0, 2, 7).astype(float)
    mean, istd = rng.standard_normal(M.N_FEAT) * 0.1, rng.uniform(0.5, 2.0, M.N_FEAT)
    g = M.grad(theta, F, y, mean, istd)
    eps = 1e-6
    for i in list(rng.choice(M.N_PARAMS, 60, replace=False)) + [0, 1535, 1536, 5695, 5823, 5824]:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (M.loss(tp, F, y, mean, istd) - M.loss(tm, F, y, mean, istd)) / (2 * eps)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_gelu_closed_form():
    z = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    phi = lambda t: 0.5 * (1 + math.erf(t / math.sqrt(2)))
    assert np.allclose(M.gelu(z), [t * phi(t) for t in z], atol=1e-15)
    fd = (M.gelu(z + 1e-6) - M.gelu(z - 1e-6)) / 2e-6
    assert np.allclose(M.gelu_grad(z), fd, atol=1e-8)


def test_adam_reaches_the_minimum_of_a_quadratic():
    c = np.array([1.5, -2.0, 0.25])
    theta, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 3001):
        theta, m, v = M.adam_step(theta, m, v, 2 * (theta - c), t, 0.01)
    assert np.allclose(theta, c, atol=1e-3)


def test_features_special_cases():
    N, D = 16, 3
    J = inputs.sk_pm1(N, 3)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((N, D))
    f = M.features(J, x, x, h=0.7, k_frac=0.1)
    # identical snapshot: no slope, no flips
    assert f[13] == 0 and f[15] == 0 and f[16] == 0
    s = np.where(x[:, 0] >= 0, 1, -1).astype(np.int8)
    assert f[12] == O.ising_energy(J, s) / N
    # quantiles: the extremes are min and max of |x0| / rms and they are sorted
    u = np.abs(x[:, 0]) / math.sqrt(np.mean(x[:, 0] ** 2))
    assert f[0] == pytest.approx(u.min()) and f[11] == pytest.approx(u.max())
    assert np.all(np.diff(f[0:12]) >= 0)
    # one flipped spin in the snapshot: flip fraction 1/N and E slope from the identity
    xs = x.copy()
    xs[4, 0] = -xs[4, 0]
    f2 = M.features(J, x, xs, 0.7, 0.1)
    assert f2[16] == pytest.approx(1 / N)
    ss = s.copy()
    ss[4] = -ss[4]
    assert f2[13] == pytest.approx((O.ising_energy(J, s) - O.ising_energy(J, ss)) / N)
    # a pure component-0 state has no extra-dimension weight; E_hs equals the Ising energy
    x1 = np.zeros((N, D))
    x1[:, 0] = x[:, 0]
    f3 = M.features(J, x1, x1, 0.7, 0.1)
    assert f3[14] == 0 and f3[17] == pytest.approx(f3[12])
    assert f[20] == D / 8 and f[21] == pytest.approx(math.log(N) / math.log(2048))
