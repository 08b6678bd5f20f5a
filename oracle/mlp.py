"""FP64 reference of the learned early exit (test infrastructure only).

The paper has no learned component; the early-exit network reads early-trajectory
features of a run and predicts whether it will end at the Ising ground state.
This module defines, in plain numpy FP64:

* the 24 features of a run at its decision step, from its state x (N x D), an
  earlier snapshot xs of the same run, the couplings J, the pump h and the
  fraction of the schedule reached;
* the network 24 -> 64 -> 64 -> 1 (input standardisation, GELU, logit output),
  its mean binary cross-entropy-with-logits loss, the backward pass and one Adam
  update.

Parameter vector layout (5825 values): W1 [64 x 24] (row = hidden unit), b1 [64],
W2 [64 x 64], b2 [64], W3 [64], b3 [1].
"""
import math

import numpy as np
from scipy.special import erf

import oracle.oracle as O

N_FEAT, H = 24, 64
SIZES = {"W1": (H, N_FEAT), "b1": (H,), "W2": (H, H), "b2": (H,), "W3": (H,), "b3": (1,)}
ORDER = ["W1", "b1", "W2", "b2", "W3", "b3"]
N_PARAMS = sum(int(np.prod(s)) for s in SIZES.values())


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SIZES[k]))
        out[k] = theta[o:o + n].reshape(SIZES[k])
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[k], dtype=np.float64).ravel() for k in ORDER])


# ---------------------------------------------------------------------------
# features
# ---------------------------------------------------------------------------
def features(J, x, xs, h, k_frac):
    """24 features of one run: x, xs are (N, D) states at the decision step and at
    an earlier snapshot."""
    N, D = x.shape
    x0 = x[:, 0]
    rms = math.sqrt(float(np.mean(x0 * x0)))
    u = np.sort(np.abs(x0) / (rms + 1e-30))
    idx = [int(math.floor(j * (N - 1) / 11.0 + 0.5)) for j in range(12)]
    f = np.zeros(N_FEAT)
    f[0:12] = u[idx]
    s = np.where(x0 >= 0, 1, -1).astype(np.int8)
    ss = np.where(xs[:, 0] >= 0, 1, -1).astype(np.int8)
    E = O.ising_energy(J, s)
    Es = O.ising_energy(J, ss)
    f[12] = E / N
    f[13] = (E - Es) / N

    def weight(v):
        tot = float(np.sum(v * v))
        return float(np.sum(v[:, 1:] ** 2)) / tot if (tot > 0 and v.shape[1] > 1) else 0.0
    w, ws = weight(x), weight(xs)
    f[14] = w
    f[15] = w - ws
    f[16] = float(np.mean(s != ss))
    f[17] = O.hyperspin_energy(J, x) / N
    f[18] = float(np.mean(np.sqrt(np.sum(x * x, axis=1))))
    f[19] = h
    f[20] = D / 8.0
    f[21] = math.log(N) / math.log(2048.0)
    f[22] = k_frac
    f[23] = rms
    return f


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------
def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(theta, F, mean, istd):
    """Logits of the rows of F (B x 24) and the cached activations."""
    p = unpack(theta)
    Fs = (np.asarray(F, dtype=np.float64) - mean) * istd
    z1 = Fs @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    logit = h2 @ p["W3"] + p["b3"][0]
    return logit, (Fs, z1, h1, z2, h2)


def loss(theta, F, y, mean, istd):
    """Mean binary cross-entropy with logits."""
    logit, _ = forward(theta, F, mean, istd)
    y = np.asarray(y, dtype=np.float64)
    return float(np.mean(np.maximum(logit, 0) - logit * y + np.log1p(np.exp(-np.abs(logit)))))


def grad(theta, F, y, mean, istd):
    """Gradient of `loss` with respect to the parameter vector (backpropagation)."""
    p = unpack(theta)
    logit, (Fs, z1, h1, z2, h2) = forward(theta, F, mean, istd)
    B = len(logit)
    dlogit = (1.0 / (1.0 + np.exp(-logit)) - np.asarray(y, dtype=np.float64)) / B
    g = {"W3": h2.T @ dlogit, "b3": np.array([dlogit.sum()])}
    dz2 = np.outer(dlogit, p["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ Fs
    g["b1"] = dz1.sum(0)
    return pack(g)


def adam_step(theta, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) at step t >= 1; returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
