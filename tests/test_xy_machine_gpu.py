"""The XY machine (D = 2, no annealing) against the XY ground state, on the GPU.

The text after Fig. 2 (mode I: D = 2, kappa L = 1e-3, beta b^2 = 25, no dimensional
annealing) compares the hyperspin energy E_hs of Eq. 3 reached by the XY machine with
the XY ground-state energy of the same graph, found by a numerical minimiser (its
footnote).  Every planar state has E_hs >= E_XY,GS, and the machine's best runs come
close to it.  The reference here is the oracle's multi-start minimiser
(oracle_xy_ground_state), pinned on the CPU by closed forms, the Ising bound and a
grid of angles; E_hs is evaluated by the oracle from the GPU's final states.
"""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2308_02329_gb300 import chym, inputs

pytestmark = pytest.mark.gpu

# bound on the best run's relative gap 1 - E_hs / E_XY,GS over the scan below; the
# paper reports below 0.14 % with its own (unpublished) graph and constants
BEST_GAP = 0.005


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chym.lib()


def _mode_one(J, prec, n_h, reps, steps, seed):
    ctx = chym.Context(J, 2)
    prm = chym.Params(eps=0.5 / ctx.lambda_max(), kappa=1e-3, gamma=25.0, prec=prec)
    ctx.run(prm, inputs.pump_grid(0.5, n_h), inputs.run_seeds(seed, n_h * reps), steps,
            chym.Schedule(0, 0, steps))
    X, k = ctx.get_state()
    assert k == steps
    ctx.close()
    return np.array([O.hyperspin_energy(J, x) for x in X])


@pytest.mark.parametrize("prec", [chym.PREC_FP64, chym.PREC_FP32, chym.PREC_BF16X2])
def test_xy_machine_mode_one_reaches_the_xy_ground_state(prec):
    """A 20 % sparse N = 100 graph (reading of the random graphs of the size study):
    16 pumps over the scanned range x 64 replicas, 20000 steps.  No run goes below the
    XY ground state; the best run comes within BEST_GAP of it."""
    J = inputs.sparse_pm1(100, 0.2, 3)
    e_xy = O.xy_ground_state(J, n_starts=64, seed=1)[0]
    E = _mode_one(J, prec, 16, 64, 20000, 0xA11CE)
    assert np.all(np.isfinite(E))
    assert np.all(E >= e_xy - 1e-9 * abs(e_xy))
    gap = 1.0 - E.min() / e_xy
    print(f"XY machine prec={prec}: E_XY,GS {e_xy:.6f}, best E_hs {E.min():.6f}, gap {gap:.2e}")
    assert gap <= BEST_GAP


@pytest.mark.parametrize("graph", ["mobius", "sk"])
def test_benchmark_xy_contexts_stay_above_the_xy_ground_state(graph):
    """The D = 2 contexts of the N = 100 benchmark (Moebius ladder and SK +-1, mode I,
    BF16 hi+lo): every final state's E_hs is at or above E_XY,GS."""
    J = inputs.mobius_ladder(100) if graph == "mobius" else inputs.sk_pm1(100, 0xC0FFEE + 1)
    e_xy = O.xy_ground_state(J, n_starts=64, seed=2)[0]
    E = _mode_one(J, chym.PREC_BF16X2, 32, 32, 20000, 0xB0B)
    assert np.all(np.isfinite(E))
    assert np.all(E >= e_xy - 1e-9 * abs(e_xy))
    print(f"{graph}: E_XY,GS {e_xy:.6f}, best E_hs {E.min():.6f}, gap {1 - E.min() / e_xy:.2e}")
