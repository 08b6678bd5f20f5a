"""Seeded synthetic inputs: coupling matrices, run seeds and pump grids.

This module holds no arithmetic of the method; it only draws the instances the
paper's workloads are made of (random +-1 graphs, the Moebius ladder, Gaussian
couplings) and the per-run seeds.  Both the CUDA path and the CPU oracle take
their inputs from here.
"""
import numpy as np

_MASK = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One output of the SplitMix64 generator (Steele, Lea, Flood 2014) for state x."""
    z = (x + 0x9E3779B97F4A7C15) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def run_seeds(instance_seed: int, n_runs: int, offset: int = 0) -> np.ndarray:
    """Per-run 64-bit noise keys: SplitMix64 of (instance_seed << 32) + run index."""
    base = (int(instance_seed) << 32) & _MASK
    return np.array([splitmix64((base + offset + r) & _MASK) for r in range(n_runs)],
                    dtype=np.uint64)


def sk_pm1(N: int, seed: int) -> np.ndarray:
    """Sherrington-Kirkpatrick +-1 couplings: symmetric, zero diagonal, signs uniform."""
    rng = np.random.default_rng(seed)
    U = rng.integers(0, 2, size=(N, N)) * 2 - 1
    J = np.triu(U, 1).astype(np.float64)
    return J + J.T


def gaussian(N: int, seed: int) -> np.ndarray:
    """Symmetric Gaussian couplings J_ij ~ N(0, 1/N), zero diagonal."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((N, N)) / np.sqrt(N)
    J = np.triu(G, 1)
    return J + J.T


def sparse_pm1(N: int, density: float, seed: int) -> np.ndarray:
    """Erdos-Renyi graph of the given edge density, each edge +-1 with equal probability."""
    rng = np.random.default_rng(seed)
    present = rng.random((N, N)) < density
    sign = rng.integers(0, 2, size=(N, N)) * 2 - 1
    J = np.triu(np.where(present, sign, 0), 1).astype(np.float64)
    return J + J.T


def mobius_ladder(N: int, j_ring: float = -1.0, j_rung: float = -1.0) -> np.ndarray:
    """Moebius ladder: ring i ~ i+1 (mod N) with j_ring plus rungs i ~ i+N/2 with j_rung."""
    if N < 6 or N % 2:
        raise ValueError("Moebius ladder needs an even N >= 6")
    J = np.zeros((N, N), dtype=np.float64)
    for i in range(N):
        j = (i + 1) % N
        J[i, j] = J[j, i] = j_ring
    for i in range(N // 2):
        j = i + N // 2
        J[i, j] = J[j, i] = j_rung
    return J


def pump_grid(h_th: float, n_h: int, dh_max: float = 1.0) -> np.ndarray:
    """Pump values h = h_th (1 + dh) for dh evenly spaced over [0, dh_max] (inclusive)."""
    dh = np.linspace(0.0, dh_max, n_h) if n_h > 1 else np.zeros(1)
    return h_th * (1.0 + dh)


def h_per_run(h: np.ndarray, replicas: int) -> np.ndarray:
    """Expand n_h pump values to h-major runs: run = ih * replicas + rep."""
    return np.repeat(np.asarray(h, dtype=np.float64), replicas)


def uneven_instances(n_inst: int, seed: int, n_lo: int = 50, n_hi: int = 2000, dims=(2, 3, 4, 8)):
    """Composition of a batched uneven workload: per instance (N, D, instance seed) with
    N uniform on the integers [n_lo, n_hi] and D uniform over `dims`."""
    rng = np.random.default_rng(seed)
    Ns = rng.integers(n_lo, n_hi + 1, size=n_inst)
    Ds = rng.choice(np.asarray(dims), size=n_inst)
    return [(int(N), int(D), int(seed) * 100003 + i) for i, (N, D) in enumerate(zip(Ns, Ds))]
