"""The CHYM as the discrete round-trip map of the optical cavity (test infrastructure only).

Written literally from Eq. 1, Eq. 2 and the output-coupler relation after Eq. 2, with
the coupling matrices built explicitly as Kronecker products over the D x N optical
parametric oscillators (PO index j = p * D + mu, hyperspin p, component mu):

    C = J_N (x) 1_D                     linear coupling between hyperspins
    W = beta 1_N (x) I_D                I_D: the D x D matrix of ones (nonlinear loss)
    B = K A                             parametric amplification in the NLM
    X = sqrt(b) (C B - b B * (W B^2))   Eq. 1, computed by the FPGA
    Y = a B + sqrt(b) X                 Eq. 2, with a + b = 1
    A' = (1 - d) Y                      the field of the next round trip

Readings (the gain K and the noise are defined in the missing supplement):
  * K is one positive constant per context (the parametric gain of the pump value),
    the same for every PO and round trip;
  * noise, if any, is added to the next field as sigma xi with xi the standard
    normals of the step noise stream (tag 0) of the run, step = round trip.

Plain dense FP64 numpy; sizes up to a few hundred POs.  Only the test suite may
import it; it shares no code with the CUDA path.
"""
import numpy as np

from . import oracle as O


def matrices(J, D, a, beta):
    """(C, W, Q) of the text after Eq. 1 and Eq. 2 for an N x N graph J."""
    J = np.asarray(J, dtype=np.float64)
    N = J.shape[0]
    b = 1.0 - a
    C = np.kron(J, np.eye(D))
    W = beta * np.kron(np.eye(N), np.ones((D, D)))
    Q = a * np.eye(N * D) + b * C
    return C, W, Q


def round_trip(A, C, W, a, d, K):
    """One cavity round trip of the field vector A (length D N), Eq. 1 and Eq. 2."""
    b = 1.0 - a
    B = K * A
    X = np.sqrt(b) * (C @ B - b * B * (W @ (B * B)))
    Y = a * B + np.sqrt(b) * X
    return (1.0 - d) * Y


def run(J, D, a, d, beta, K, seeds, round_trips, init_std=0.1, sigma=0.0, k0=0, A0=None):
    """Fields after `round_trips` round trips for every run (seeded like the Euler
    runs: A(0) = init_std * N(0, 1) from the initial-state stream, then the step
    noise of round trip k added as sigma xi(k)).  Returns A[run, p, mu]."""
    J = np.asarray(J, dtype=np.float64)
    N = J.shape[0]
    C, W, _ = matrices(J, D, a, beta)
    seeds = np.asarray(seeds, dtype=np.uint64)
    A = O.init_state(N, D, seeds, init_std) if A0 is None else np.array(A0, dtype=np.float64)
    out = np.empty_like(A)
    for r, seed in enumerate(seeds):
        v = A[r].reshape(-1).copy()
        for k in range(k0, k0 + round_trips):
            v = round_trip(v, C, W, a, d, K)
            if sigma:
                v = v + sigma * O.normals(int(seed), 0, k, N, D).reshape(-1)
        out[r] = v.reshape(N, D)
    return out


def threshold_gain(J, a, d):
    """Smallest gain at which the zero field loses stability through the top eigenmode
    of J: the linear part of the map is (1 - d) K Q, and Q has the eigenvalues
    a + b lambda_i, so K_th = 1 / ((1 - d) (a + b lambda_max)) whenever
    a + b lambda_max >= |a + b lambda_min| (true for a > 0 and a spectrum symmetric
    about zero, as for the +-1 graphs)."""
    lam = float(np.linalg.eigvalsh(np.asarray(J, dtype=np.float64))[-1])
    return 1.0 / ((1.0 - d) * (a + (1.0 - a) * lam))
