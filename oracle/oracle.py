"""ctypes front end of the FP64 C oracle (test infrastructure only).

Every function states the passage of arXiv 2308.02329 it follows; the C source
``chym_oracle.c`` holds the arithmetic.  Arrays are numpy float64 / int8 /
uint64 with the state laid out as X[run, p, mu] (hyperspin p, component mu).
"""
import ctypes
import os
from dataclasses import dataclass

import numpy as np

from .build import build_oracle

_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        dp = ctypes.POINTER(ctypes.c_double)
        i8p = ctypes.POINTER(ctypes.c_int8)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.oracle_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                      ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
        lib.oracle_round_xy.argtypes = [dp, ctypes.c_int, dp, i8p]
        lib.oracle_round_xy.restype = ctypes.c_double
        lib.oracle_normal.restype = ctypes.c_double
        lib.oracle_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                       ctypes.c_int, ctypes.c_int, dp]
        lib.oracle_alpha.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_int64, ctypes.c_int]
        lib.oracle_alpha.restype = ctypes.c_double
        lib.oracle_init.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p,
                                    ctypes.c_double, dp]
        lib.oracle_drift.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_int64, dp]
        lib.oracle_integrate.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                         u64p, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_int64, dp, ctypes.c_int]
        lib.oracle_readout.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, i8p]
        lib.oracle_ising_energy.argtypes = [dp, ctypes.c_int, i8p]
        lib.oracle_ising_energy.restype = ctypes.c_double
        lib.oracle_hyperspin_energy.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
        lib.oracle_hyperspin_energy.restype = ctypes.c_double
        lib.oracle_ground_state_bruteforce.argtypes = [dp, ctypes.c_int, i8p]
        lib.oracle_ground_state_bruteforce.restype = ctypes.c_double
        lib.oracle_ground_state_mobius.argtypes = [ctypes.c_int, ctypes.c_double,
                                                   ctypes.c_double]
        lib.oracle_ground_state_mobius.restype = ctypes.c_double
        lib.oracle_xy_energy.argtypes = [dp, ctypes.c_int, dp]
        lib.oracle_xy_energy.restype = ctypes.c_double
        lib.oracle_xy_ground_state.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int,
                                               ctypes.c_double, dp]
        lib.oracle_xy_ground_state.restype = ctypes.c_double
        _lib = lib
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


@dataclass
class Params:
    """Model constants of the oracle (the readings are listed in the C header).

    gamma: non-local saturation beta b^2; kappa: local nonlinearity kappa L;
    eps: feedback coupling strength; sigma: diffusion coefficient of the
    additive noise (per-step std sigma sqrt(dt)); init_std: std of x(0).
    """
    dt: float = 0.01
    sigma: float = 1e-3
    init_std: float = 0.1
    gamma: float = 25.0
    kappa: float = 0.1
    eps: float = 0.05


@dataclass
class Schedule:
    """Annealing schedule alpha_mu(k): kind 0 none, kind 1 linear from k_anneal to k_total."""
    kind: int = 1
    k_anneal: int = 0
    k_total: int = 1


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _L().oracle_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32),
                              _p(out, ctypes.c_uint32))
    return out


def normal(seed, tag, k, p, mu, D):
    """Normal of component mu of spin p of a D-component run (see oracle_normal)."""
    return _L().oracle_normal(int(seed), int(tag), int(k), int(p), int(mu), int(D))


def normals(seed, tag, k, N, D):
    out = np.zeros((N, D), dtype=np.float64)
    _L().oracle_normals(int(seed), int(tag), int(k), int(N), int(D), _p(out, ctypes.c_double))
    return out


def alpha(sched: Schedule, k, mu):
    return _L().oracle_alpha(int(sched.kind), int(k), int(sched.k_anneal),
                             int(sched.k_total), int(mu))


def init_state(N, D, seeds, init_std):
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    X = np.zeros((len(seeds), N, D), dtype=np.float64)
    _L().oracle_init(int(N), int(D), len(seeds), _p(seeds, ctypes.c_uint64),
                     float(init_std), _p(X, ctypes.c_double))
    return X


def drift(J, x, h, prm: Params, sched: Schedule, k):
    J = np.ascontiguousarray(J, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    N, D = x.shape
    f = np.zeros_like(x)
    _L().oracle_drift(_p(J, ctypes.c_double), N, D, _p(x, ctypes.c_double), float(h),
                      prm.gamma, prm.kappa, prm.eps, sched.kind, int(k), int(sched.k_anneal),
                      int(sched.k_total), _p(f, ctypes.c_double))
    return f


def integrate(J, X, h_run, seeds, prm: Params, sched: Schedule, k0, steps, threads=0):
    """Euler-Maruyama steps k0..k0+steps-1 of every run, in place on X[run, p, mu]."""
    J = np.ascontiguousarray(J, dtype=np.float64)
    assert X.dtype == np.float64 and X.flags.c_contiguous
    n_runs, N, D = X.shape
    h_run = np.ascontiguousarray(h_run, dtype=np.float64)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    assert len(h_run) == n_runs and len(seeds) == n_runs
    _L().oracle_integrate(_p(J, ctypes.c_double), N, D, n_runs, _p(h_run, ctypes.c_double),
                          _p(seeds, ctypes.c_uint64), prm.dt, prm.sigma, prm.gamma,
                          prm.kappa, prm.eps, sched.kind, int(sched.k_anneal),
                          int(sched.k_total), int(k0), int(steps), _p(X, ctypes.c_double),
                          int(threads))
    return X


def run(J, D, h_run, seeds, prm: Params, sched: Schedule, steps, threads=0):
    """Initialise every run from its seed and integrate `steps` steps from k = 0."""
    J = np.ascontiguousarray(J, dtype=np.float64)
    X = init_state(J.shape[0], D, seeds, prm.init_std)
    return integrate(J, X, h_run, seeds, prm, sched, 0, steps, threads)


def readout(X):
    X = np.ascontiguousarray(X, dtype=np.float64)
    n_runs, N, D = X.shape
    s = np.zeros((n_runs, N), dtype=np.int8)
    _L().oracle_readout(N, D, n_runs, _p(X, ctypes.c_double), _p(s, ctypes.c_int8))
    return s


def ising_energy(J, s):
    J = np.ascontiguousarray(J, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.int8)
    return _L().oracle_ising_energy(_p(J, ctypes.c_double), J.shape[0], _p(s, ctypes.c_int8))


def ising_energies(J, S):
    return np.array([ising_energy(J, s) for s in S], dtype=np.float64)


def round_xy(J, x):
    """Best-axis rounding of one D = 2 state x (N x 2): (energy, spins)."""
    J = np.ascontiguousarray(J, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    s = np.zeros(x.shape[0], dtype=np.int8)
    e = _L().oracle_round_xy(_p(J, ctypes.c_double), J.shape[0], _p(x, ctypes.c_double),
                             _p(s, ctypes.c_int8))
    return e, s


def hyperspin_energy(J, x):
    J = np.ascontiguousarray(J, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    N, D = x.shape
    return _L().oracle_hyperspin_energy(_p(J, ctypes.c_double), N, D, _p(x, ctypes.c_double))


def ground_state_bruteforce(J):
    J = np.ascontiguousarray(J, dtype=np.float64)
    N = J.shape[0]
    s = np.zeros(N, dtype=np.int8)
    e = _L().oracle_ground_state_bruteforce(_p(J, ctypes.c_double), N, _p(s, ctypes.c_int8))
    return e, s


def ground_state_mobius(N, Jr=-1.0, Jg=-1.0):
    return _L().oracle_ground_state_mobius(int(N), float(Jr), float(Jg))


def xy_energy(J, theta):
    """E_XY = -sum_{p,q} J_pq cos(theta_p - theta_q): Eq. 3 with planar unit spins."""
    J = np.ascontiguousarray(J, dtype=np.float64)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    return _L().oracle_xy_energy(_p(J, ctypes.c_double), J.shape[0], _p(th, ctypes.c_double))


def xy_ground_state(J, n_starts=64, seed=0, max_sweeps=20000, tol=1e-14):
    """XY ground-state energy (the reference of the XY machine, text after Fig. 2 and its
    footnote) by multi-start coordinate descent on the angles: n_starts starts from angles
    drawn uniformly on [0, 2 pi) by numpy's PCG64 with `seed`.  Returns (energy, angles)."""
    J = np.ascontiguousarray(J, dtype=np.float64)
    N = J.shape[0]
    th0 = np.random.default_rng(seed).uniform(0.0, 2.0 * np.pi, size=(n_starts, N))
    th0 = np.ascontiguousarray(th0)
    out = np.zeros(N, dtype=np.float64)
    e = _L().oracle_xy_ground_state(_p(J, ctypes.c_double), N, int(n_starts),
                                    _p(th0, ctypes.c_double), int(max_sweeps), float(tol),
                                    _p(out, ctypes.c_double))
    return e, out
