"""CPU pins of the FP64 oracle against things other than itself.

Each test checks the oracle against a published known-answer vector, a closed
form of the model, a symmetry of the equations, or brute force, chosen so that a
plausible slip (a dropped term, a wrong sign or index, a transposed operand, a
wrong noise scaling) fails one of them.  No GPU is needed.
"""
import itertools
import os

import numpy as np
import pytest

import oracle.oracle as O
from oracle.stats import energy_histogram, figures_of_merit, hits_per_h
from paper_2308_02329_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Noise generator
# --------------------------------------------------------------------------
def test_philox_known_answers():
    """Philox4x32-10 reproduces the published known-answer vectors."""
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = O.philox4x32_10(r[0:4], r[4:6])
        assert [int(v) for v in out] == r[6:10]


def test_normals_moments_and_independence():
    """Box-Muller normals: mean 0, variance 1, kurtosis 3, no cross-correlation."""
    z = O.normals(seed=0x1234ABCD5678, tag=0, k=7, N=200000, D=5)  # 1e6 samples
    n = z.size
    assert abs(z.mean()) < 5.0 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    kurt = np.mean(z ** 4) / np.mean(z ** 2) ** 2
    assert abs(kurt - 3.0) < 5.0 * np.sqrt(24.0 / n)
    c = np.corrcoef(z.T)
    off = c[~np.eye(5, dtype=bool)]
    assert np.max(np.abs(off)) < 5.0 / np.sqrt(z.shape[0])
    # the two members of a Box-Muller pair are uncorrelated in their squares too
    assert abs(np.corrcoef(z[:, 0] ** 2, z[:, 1] ** 2)[0, 1]) < 5.0 / np.sqrt(z.shape[0])


def test_normals_distinct_streams():
    """Different steps, tags, spins and seeds draw different numbers."""
    a = O.normals(1, 0, 0, 64, 4)
    assert not np.allclose(a, O.normals(1, 0, 1, 64, 4))
    assert not np.allclose(a, O.normals(1, 1, 0, 64, 4))
    assert not np.allclose(a, O.normals(2, 0, 0, 64, 4))
    assert len(np.unique(a)) == a.size
    # steps beyond 2^32 use the high counter word
    assert O.normal(5, 0, 1 << 32, 0, 0, 4) != O.normal(5, 0, 0, 0, 0, 4)
    # component mu and mu + 4 come from different Philox blocks
    b = O.normals(1, 0, 0, 16, 8)
    assert not np.allclose(b[:, :4], b[:, 4:])


def test_normals_block_layout():
    """One Philox block gives four normals: for D >= 3 they belong to one spin
    (components mu = 4 b .. 4 b + 3), for D <= 2 to the 4/D spins that share the
    block, in the order of the element index p D + mu, so that every word is used."""
    def box_muller(w):
        u = (np.asarray(w, dtype=np.float64) + 0.5) / 2.0 ** 32
        r0, r1 = np.sqrt(-2 * np.log(u[0])), np.sqrt(-2 * np.log(u[2]))
        t0, t1 = 2 * np.pi * u[1], 2 * np.pi * u[3]
        return [r0 * np.cos(t0), r0 * np.sin(t0), r1 * np.cos(t1), r1 * np.sin(t1)]
    seed, k = 0x1234567890ABCDEF, 41
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for D in (1, 2, 3, 4, 6):
        z = O.normals(seed, 0, k, 12, D)
        for p in range(12):
            for mu in range(D):
                if D <= 2:
                    per = 4 // D
                    ctr, j = [p // per, 0, k, 0], (p % per) * D + mu
                else:
                    ctr, j = [p, mu // 4, k, 0], mu % 4
                zz = box_muller(O.philox4x32_10(ctr, key))[j]
                assert abs(z[p, mu] - zz) <= 1e-12 * max(1.0, abs(zz))
    # the initial state uses tag 1 in the same layout
    assert O.normals(seed, 1, 0, 4, 2)[1, 0] != O.normals(seed, 0, 0, 4, 2)[1, 0]


# --------------------------------------------------------------------------
# Annealing schedule
# --------------------------------------------------------------------------
def test_alpha_schedule_closed_form():
    s = O.Schedule(kind=1, k_anneal=1500, k_total=3000)
    assert O.alpha(s, 0, 1) == 1.0
    assert O.alpha(s, 1499, 2) == 1.0
    assert O.alpha(s, 1500, 1) == 1.0
    assert O.alpha(s, 2250, 1) == pytest.approx(0.5, abs=1e-15)
    assert O.alpha(s, 2999, 1) == pytest.approx(1.0 / 1500.0, abs=1e-15)
    assert O.alpha(s, 3000, 1) == 0.0
    for k in (0, 1600, 2999, 5000):
        assert O.alpha(s, k, 0) == 1.0  # the surviving component is never annealed
    none = O.Schedule(kind=0, k_anneal=0, k_total=10)
    assert O.alpha(none, 9, 3) == 1.0


# --------------------------------------------------------------------------
# Drift: closed forms and symmetries
# --------------------------------------------------------------------------
def _no_noise(**kw):
    p = O.Params(sigma=0.0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_linear_growth_along_eigenvectors():
    """Near x = 0 each component grows by 1 + dt (h - 1 + eps lambda) per step along an
    eigenvector of J, independently per component (C = J (x) 1_D)."""
    J = inputs.sk_pm1(12, seed=3)
    lam, V = np.linalg.eigh(J)
    prm = _no_noise(gamma=25.0, kappa=0.1, eps=0.07)
    h = 0.8
    x0 = np.zeros((1, 12, 2))
    x0[0, :, 0] = 1e-6 * V[:, -1]  # top eigenvector in component 0
    x0[0, :, 1] = 1e-6 * V[:, 0]   # bottom eigenvector in component 1
    X = x0.copy()
    O.integrate(J, X, [h], [0], prm, O.Schedule(kind=0), 0, 3)
    for mu, l in ((0, lam[-1]), (1, lam[0])):
        g = (1.0 + prm.dt * (h - 1.0 + prm.eps * l)) ** 3
        np.testing.assert_allclose(X[0, :, mu], g * x0[0, :, mu], rtol=1e-9, atol=1e-18)


def test_uncoupled_fixed_points():
    """J = 0: the non-local loss fixes |x_p|^2 = (h-1)/gamma for every D; the local one
    fixes x^2 = (h-1)/(gamma+kappa) for D = 1 and x_mu^2 = (h-1)/kappa when gamma = 0."""
    N = 5
    J = np.zeros((N, N))
    rng = np.random.default_rng(0)
    h = 1.5
    steps = 4000
    X = rng.uniform(0.05, 0.3, size=(2, N, 3))
    O.integrate(J, X, [h, h], [1, 2], _no_noise(gamma=25.0, kappa=0.0), O.Schedule(kind=0),
                0, steps)
    np.testing.assert_allclose((X ** 2).sum(-1), (h - 1) / 25.0, rtol=1e-9)

    X = rng.uniform(0.05, 0.3, size=(1, N, 1))
    O.integrate(J, X, [h], [1], _no_noise(gamma=25.0, kappa=7.0), O.Schedule(kind=0), 0, steps)
    np.testing.assert_allclose(X[..., 0] ** 2, (h - 1) / 32.0, rtol=1e-9)

    X = rng.uniform(0.3, 0.6, size=(1, N, 2))
    O.integrate(J, X, [h], [1], _no_noise(gamma=0.0, kappa=2.0), O.Schedule(kind=0), 0, steps)
    np.testing.assert_allclose(X ** 2, (h - 1) / 2.0, rtol=1e-9)


def test_rotation_equivariance_of_hyperspins():
    """With kappa = 0 and no annealing the equations are O(D) equivariant: the loss
    depends on |x_p| only and J acts on every component alike."""
    J = inputs.sk_pm1(10, seed=11)
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    x0 = 0.1 * rng.standard_normal((1, 10, 3))
    prm = _no_noise(gamma=25.0, kappa=0.0, eps=0.1)
    A = x0.copy()
    B = x0 @ Q.T
    O.integrate(J, A, [0.9], [0], prm, O.Schedule(kind=0), 0, 300)
    O.integrate(J, B, [0.9], [0], prm, O.Schedule(kind=0), 0, 300)
    np.testing.assert_allclose(B, A @ Q.T, rtol=0, atol=1e-13)
    # the local nonlinearity acts per component and must break the symmetry
    prm.kappa = 5.0
    A = x0.copy()
    B = x0 @ Q.T
    O.integrate(J, A, [0.9], [0], prm, O.Schedule(kind=0), 0, 300)
    O.integrate(J, B, [0.9], [0], prm, O.Schedule(kind=0), 0, 300)
    assert np.max(np.abs(B - A @ Q.T)) > 1e-6


def test_z2_and_component_permutation():
    J = inputs.sk_pm1(9, seed=5)
    rng = np.random.default_rng(2)
    x0 = 0.1 * rng.standard_normal((1, 9, 4))
    prm = _no_noise(kappa=0.1, eps=0.1)
    A, B = x0.copy(), -x0
    O.integrate(J, A, [0.95], [0], prm, O.Schedule(kind=0), 0, 200)
    O.integrate(J, B, [0.95], [0], prm, O.Schedule(kind=0), 0, 200)
    assert np.array_equal(B, -A)
    perm = [2, 0, 3, 1]
    C = x0[..., perm].copy()
    O.integrate(J, C, [0.95], [0], prm, O.Schedule(kind=0), 0, 200)
    np.testing.assert_allclose(C, A[..., perm], rtol=0, atol=1e-14)


def test_noise_scaling_is_sigma_sqrt_dt():
    """Free diffusion (J = 0, h = 1, no loss): Var x_K = K sigma^2 dt."""
    N, D, R, K = 8, 4, 500, 50
    prm = O.Params(dt=0.01, sigma=1e-3, gamma=0.0, kappa=0.0, eps=0.0)
    X = np.zeros((R, N, D))
    seeds = inputs.run_seeds(77, R)
    O.integrate(np.zeros((N, N)), X, np.ones(R), seeds, prm, O.Schedule(kind=0), 0, K)
    var = X.var()
    expect = K * prm.sigma ** 2 * prm.dt
    n = X.size
    assert abs(var / expect - 1.0) < 5.0 * np.sqrt(2.0 / n)


def test_initial_state_variance():
    X = O.init_state(50, 4, inputs.run_seeds(3, 200), init_std=0.1)
    n = X.size
    assert abs(X.var() / 0.01 - 1.0) < 5.0 * np.sqrt(2.0 / n)
    assert abs(X.mean()) < 5.0 * 0.1 / np.sqrt(n)


def test_annealing_drives_extra_components_away():
    """After the linear schedule the hyperspins have turned (mostly) into component 0:
    the share of the annealed components mu >= 1 in |x_p| collapses, while without
    annealing it stays of order one."""
    N, D = 12, 3
    J = inputs.sk_pm1(N, seed=21)
    lam = np.linalg.eigvalsh(J)[-1]
    prm = O.Params(eps=0.5 / lam)
    h_th = 1.0 - prm.eps * lam
    K = 3000
    seeds = inputs.run_seeds(9, 8)

    def share(X):
        return np.sqrt((X[..., 1:] ** 2).sum(-1)) / np.sqrt((X ** 2).sum(-1))

    X = O.run(J, D, np.full(8, 1.5 * h_th), seeds, prm, O.Schedule(1, 1500, K), K)
    X0 = O.run(J, D, np.full(8, 1.5 * h_th), seeds, prm, O.Schedule(0, 0, K), K)
    assert np.median(np.sqrt((X ** 2).sum(-1))) > 0.03
    assert np.median(share(X)) < 0.1
    assert np.median(share(X0)) > 0.5


def test_split_integration_equals_single_pass():
    """The noise is counter based: steps [0,K) equal [0,K/2) followed by [K/2,K)."""
    J = inputs.sk_pm1(10, seed=4)
    prm = O.Params(eps=0.06)
    seeds = inputs.run_seeds(5, 6)
    h = np.linspace(0.5, 0.9, 6)
    sch = O.Schedule(1, 100, 300)
    A = O.init_state(10, 3, seeds, prm.init_std)
    B = A.copy()
    O.integrate(J, A, h, seeds, prm, sch, 0, 300, threads=1)
    O.integrate(J, B, h, seeds, prm, sch, 0, 150, threads=3)
    O.integrate(J, B, h, seeds, prm, sch, 150, 150, threads=2)
    assert np.array_equal(A, B)


# --------------------------------------------------------------------------
# Ising energy, readout and ground states
# --------------------------------------------------------------------------
def _all_states(N):
    return np.array(list(itertools.product([1, -1], repeat=N)), dtype=np.int8)


def test_energy_single_flip_identity_and_mod4():
    J = inputs.sk_pm1(15, seed=8)
    rng = np.random.default_rng(3)
    c = -J.sum()
    for _ in range(20):
        s = rng.choice(np.array([-1, 1], dtype=np.int8), size=15)
        e = O.ising_energy(J, s)
        assert (e - c) % 4 == 0
        p = rng.integers(15)
        t = s.copy()
        t[p] = -t[p]
        assert O.ising_energy(J, t) - e == 4 * s[p] * (J[p] @ s)


def test_energy_and_readout_closed_forms():
    N = 7
    ferro = np.ones((N, N)) - np.eye(N)
    assert O.ising_energy(ferro, np.ones(N, dtype=np.int8)) == -N * (N - 1)
    X = np.array([[[0.3], [-0.2], [0.0], [-0.0], [1e-300]]])
    assert O.readout(X).tolist() == [[1, -1, 1, 1, 1]]


def test_bruteforce_against_full_enumeration():
    for N, seed in ((6, 1), (9, 2), (12, 3)):
        for J in (inputs.sk_pm1(N, seed), inputs.gaussian(N, seed), inputs.sparse_pm1(N, 0.4, seed)):
            S = _all_states(N).astype(np.float64)
            E = -np.einsum("ip,pq,iq->i", S, J, S)
            e, s = O.ground_state_bruteforce(J)
            assert e == pytest.approx(E.min(), abs=1e-9)
            assert O.ising_energy(J, s) == pytest.approx(e, abs=1e-9)


def test_bruteforce_known_ground_states():
    N = 10
    ferro = np.ones((N, N)) - np.eye(N)
    assert O.ground_state_bruteforce(ferro)[0] == -N * (N - 1)
    for N in (8, 9):
        ring = np.zeros((N, N))
        for i in range(N):
            ring[i, (i + 1) % N] = ring[(i + 1) % N, i] = -1.0
        expect = -2 * N if N % 2 == 0 else -2 * N + 4
        assert O.ground_state_bruteforce(ring)[0] == expect


@pytest.mark.parametrize("N", [6, 8, 10, 12, 14, 16, 18, 20])
def test_mobius_transfer_matrix_against_bruteforce(N):
    for jr, jg in ((-1.0, -1.0), (1.0, -1.0), (-1.0, 1.0), (0.5, -2.0)):
        J = inputs.mobius_ladder(N, jr, jg)
        assert O.ground_state_mobius(N, jr, jg) == pytest.approx(
            O.ground_state_bruteforce(J)[0], abs=1e-9)


def test_hyperspin_energy_special_cases():
    J = inputs.sk_pm1(11, seed=6)
    rng = np.random.default_rng(4)
    s = rng.choice(np.array([-1, 1], dtype=np.int8), size=11)
    x = (s * rng.uniform(0.1, 2.0, size=11))[:, None]
    assert O.hyperspin_energy(J, x) == pytest.approx(O.ising_energy(J, s), abs=1e-12)
    u = np.tile([0.6, 0.8], (11, 1)) * rng.uniform(0.5, 2, size=(11, 1))
    assert O.hyperspin_energy(J, u) == pytest.approx(-J.sum(), abs=1e-12)
    x3 = rng.standard_normal((11, 3))
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    assert O.hyperspin_energy(J, x3 @ Q.T) == pytest.approx(O.hyperspin_energy(J, x3), abs=1e-12)
    # |sigma| = 1 bounds the energy by sum |J|
    assert abs(O.hyperspin_energy(J, x3)) <= np.abs(J).sum() + 1e-12


# --------------------------------------------------------------------------
# Figures of merit
# --------------------------------------------------------------------------
def test_figures_of_merit_hand_example():
    E_gs = -12.0
    E = np.array([-12, -12, -8, -4,    # h0: 2 of 4 hit
                  -8, -8, -8, -8,      # h1: 0 hits
                  -12, -8, -12, -12])  # h2: 3 hits
    fm = figures_of_merit(E, E_gs, 3)
    assert fm["hits"].tolist() == [2, 0, 3]
    assert fm["P_max"] == 0.75
    assert fm["W_range"] == pytest.approx((0.5 + 0.75) / 2)
    assert fm["W_scan"] == pytest.approx((0.5 + 0.75) / 3)
    assert fm["dE_mean"] == pytest.approx(np.mean(E - E_gs))
    lv, ct = energy_histogram(E)
    assert lv.tolist() == [-12, -8, -4] and ct.tolist() == [5, 6, 1]
    assert hits_per_h([-1.0 + 1e-12, np.nan], -1.0, 2, real_j=True).tolist() == [1, 0]


# --------------------------------------------------------------------------
# Best-axis rounding of XY states (D = 2)
# --------------------------------------------------------------------------
def _grid_round_xy(J, x, n_phi):
    """The lowest Ising energy of the patterns sign(x . u(phi)) over a uniform grid of
    n_phi axes in [0, pi): a brute force that knows nothing of critical angles."""
    best = np.inf
    for phi in (np.arange(n_phi) + 0.5) * np.pi / n_phi:
        s = np.where(x @ np.array([np.cos(phi), np.sin(phi)]) >= 0, 1, -1).astype(np.int8)
        best = min(best, O.ising_energy(J, s))
    return best


def test_round_xy_matches_a_fine_grid_of_axes():
    for seed in range(6):
        rng = np.random.default_rng(seed)
        N = 9
        J = inputs.sk_pm1(N, 100 + seed)
        x = rng.standard_normal((N, 2))
        crit = np.sort(np.mod(np.arctan2(x[:, 1], x[:, 0]) + np.pi / 2, np.pi))
        gaps = np.diff(np.concatenate([crit, [crit[0] + np.pi]]))
        n_phi = 20000
        assert gaps.min() > 2 * np.pi / n_phi    # every pattern interval holds grid points
        e, s = O.round_xy(J, x)
        assert e == _grid_round_xy(J, x, n_phi)
        assert O.ising_energy(J, s) == e


def test_round_xy_invariances():
    rng = np.random.default_rng(3)
    N = 14
    J = inputs.sk_pm1(N, 5)
    x = rng.standard_normal((N, 2))
    e, _ = O.round_xy(J, x)
    # never worse than reading the first component (the axis phi = 0 is a candidate)
    assert e <= O.ising_energy(J, np.where(x[:, 0] >= 0, 1, -1).astype(np.int8))
    # a common rotation of every spin leaves the best axis energy unchanged
    for psi in (0.3, 1.1, 2.9):
        R = np.array([[np.cos(psi), -np.sin(psi)], [np.sin(psi), np.cos(psi)]])
        assert O.round_xy(J, x @ R.T)[0] == e
    # spins already on the first axis: the plain readout is the best pattern (or its flip)
    y = np.stack([np.sign(x[:, 0]) * (1 + rng.random(N)), np.zeros(N)], axis=1)
    e1, s1 = O.round_xy(J, y)
    assert e1 == O.ising_energy(J, np.where(y[:, 0] >= 0, 1, -1).astype(np.int8))
    assert abs(int(s1 @ np.sign(y[:, 0]))) == N
    # a spin of zero length projects to zero and reads +1 on every axis
    z = x.copy()
    z[4] = 0.0
    ez, sz = O.round_xy(J, z)
    assert sz[4] == 1 and O.ising_energy(J, sz) == ez


# --------------------------------------------------------------------------
# XY ground state (reference of the XY machine, D = 2 without annealing)
# --------------------------------------------------------------------------
def _ring(N, j):
    J = np.zeros((N, N))
    for i in range(N):
        J[i, (i + 1) % N] = J[(i + 1) % N, i] = j
    return J


def test_xy_ground_state_closed_forms():
    """Closed forms of the XY ground state in the full double-sum convention of Eq. 3:
    a ferromagnet aligns every spin (E = -N(N-1)); an antiferromagnetic ring of odd N
    cannot alternate, and its best compromise turns each bond by pi - pi/N
    (E = -2N cos(pi/N)); an even antiferromagnetic ring alternates (E = -2N)."""
    for N in (2, 5, 10):
        J = np.ones((N, N)) - np.eye(N)
        assert O.xy_ground_state(J, n_starts=8)[0] == pytest.approx(-N * (N - 1), rel=1e-12)
    for N in (3, 5, 7, 9, 15):
        e, th = O.xy_ground_state(_ring(N, -1.0), n_starts=16)
        assert e == pytest.approx(-2 * N * np.cos(np.pi / N), rel=1e-10)
        assert O.xy_energy(_ring(N, -1.0), th) == pytest.approx(e, rel=1e-14)
    for N in (4, 8, 12):
        assert O.xy_ground_state(_ring(N, -1.0), n_starts=16)[0] == pytest.approx(-2 * N, rel=1e-10)
    # a ferromagnetic ring and the AF triangle (-3 against the Ising -2)
    assert O.xy_ground_state(_ring(6, 1.0), n_starts=4)[0] == pytest.approx(-12, rel=1e-12)
    assert O.xy_ground_state(_ring(3, -1.0), n_starts=4)[0] == pytest.approx(-3, rel=1e-10)


def test_xy_ground_state_bounds_the_ising_one():
    """XY spins include the Ising states (theta in {0, pi}), so E_XY,GS <= E_Ising,GS, with
    equality on an unfrustrated graph (a gauge transform tau_p tau_q |J_pq| of a
    ferromagnet, whose Ising and XY ground states both reach -sum |J|)."""
    for seed in range(4):
        for J in (inputs.sk_pm1(12, 40 + seed), inputs.sparse_pm1(14, 0.4, 50 + seed),
                  inputs.gaussian(10, 60 + seed)):
            e_xy = O.xy_ground_state(J, n_starts=32, seed=seed)[0]
            e_is = O.ground_state_bruteforce(J)[0]
            assert e_xy <= e_is + 1e-12 * abs(e_is)
        rng = np.random.default_rng(seed)
        tau = rng.choice([-1.0, 1.0], size=11)
        A = np.abs(inputs.gaussian(11, 70 + seed))
        J = A * np.outer(tau, tau)
        e_xy = O.xy_ground_state(J, n_starts=16, seed=seed)[0]
        assert e_xy == pytest.approx(-np.sum(A), rel=1e-10)
        assert O.ground_state_bruteforce(J)[0] == pytest.approx(-np.sum(A), rel=1e-12)


def test_xy_ground_state_against_a_grid_of_angles():
    """Brute force on tiny inputs: with theta_0 = 0 (a common rotation keeps E), a grid of
    the other angles comes within the curvature bound of the minimiser's energy and never
    below it.  E(grid) - E_min <= |H| (N-1) h^2 / 8 with |H| <= 4 max_p sum_q |J_pq|."""
    n = 72
    g = np.arange(n) * (2 * np.pi / n)
    for seed in range(3):
        J = inputs.gaussian(4, 80 + seed)
        e_min, th = O.xy_ground_state(J, n_starts=32, seed=seed)
        t1, t2, t3 = np.meshgrid(g, g, g, indexing="ij")
        T = [np.zeros_like(t1), t1, t2, t3]
        E = np.zeros_like(t1)
        for p in range(4):
            for q in range(4):
                E -= J[p, q] * np.cos(T[p] - T[q])
        e_grid = float(E.min())
        bound = 4 * np.max(np.sum(np.abs(J), axis=1)) * 3 * (2 * np.pi / n) ** 2 / 8
        assert e_min <= e_grid + 1e-12
        assert e_grid - e_min <= bound
        # the minimiser's angles: every spin is aligned with its local field
        f = J @ np.stack([np.cos(th), np.sin(th)], axis=1)
        cross = f[:, 0] * np.sin(th) - f[:, 1] * np.cos(th)
        assert np.max(np.abs(cross)) < 1e-6
