"""The bounded-wait failure path of the tensor-core kernels, exercised without a fault.

Every device-side wait of the tensor-core step kernels (mbarrier phases of the
products, TMA copies, the accumulator hand-over) gives up after a limit, raises the
context's status word, drains the work the CTA issued and frees its tensor memory.
CHYM_FLAG_TEST_STALL makes that happen on purpose: the thread that issues a step's
products withholds the signal that they are complete (nothing else sets it), and the
limit drops to 2 ms.  The next synchronising call must report CHYM_ETIMEOUT, clear the
word, and leave the context usable: a restart from the seeds gives exactly the states
and energies of a fresh context.  No trap, fault or unbounded wait is involved.
"""
import time

import numpy as np
import pytest

from paper_2308_02329_gb300 import chym, inputs
from tests.helpers import make_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chym.lib()


def _params(eps, prec, stall):
    return chym.Params(eps=eps, prec=prec, flags=chym.FLAG_TEST_STALL if stall else 0)


@pytest.mark.parametrize("N,D,prec", [(100, 4, chym.PREC_BF16X2),   # small-N kernel
                                      (48, 2, chym.PREC_BF16X2),
                                      (300, 3, chym.PREC_BF16X2),   # large-N kernel
                                      (260, 4, chym.PREC_FP8)])
def test_stalled_products_time_out_and_the_context_recovers(N, D, prec):
    J, eps, h, seeds = make_case(N, D, 2, 8, 5 + N)
    sch = chym.Schedule(1, 10, 20)
    ctx = chym.Context(J, D)
    ctx.run(_params(eps, prec, False), h, seeds, 2, sch)   # operand images built, kernels loaded
    ctx.energy()
    t0 = time.perf_counter()
    ctx.run(_params(eps, prec, True), h, seeds, 3, sch)
    with pytest.raises(chym.ChymError) as e:
        ctx.energy()
    elapsed = time.perf_counter() - t0
    assert e.value.status == chym.ETIMEOUT
    assert elapsed < 1.9   # the short limit ran out, not the 2 s one
    # the status word is cleared and a restart from the seeds runs normally
    ctx.run(_params(eps, prec, False), h, seeds, 20, sch)
    X, k = ctx.get_state()
    E = ctx.energy()
    ref = chym.Context(J, D)
    ref.run(_params(eps, prec, False), h, seeds, 20, sch)
    assert k == 20
    assert np.array_equal(X, ref.get_state()[0])
    assert np.array_equal(E, ref.energy())
    ctx.close()
    ref.close()


def test_stalled_batch_reports_the_timeout_and_recovers():
    """A batch with a small-N and a large-N context, both stalled: chym_batch_status
    reports CHYM_ETIMEOUT once; afterwards the batch integrates exactly as the contexts
    do alone."""
    specs = [(inputs.sk_pm1(90, 3), 3), (inputs.sk_pm1(200, 2), 2)]

    def make():
        out = []
        for k, (J, D) in enumerate(specs):
            c = chym.Context(J, D)
            eps = 0.5 / c.lambda_max()
            sch = chym.Schedule(1, 10, 30)
            c.run(_params(eps, chym.PREC_BF16X2, False), inputs.pump_grid(0.5, 2),
                  inputs.run_seeds(91 + k, 24), 0, sch)
            out.append((c, eps, sch))
        return out

    batched = make()
    b = chym.Batch([c for c, _, _ in batched])
    b.run([_params(e, chym.PREC_BF16X2, True) for _, e, _ in batched], [s for _, _, s in batched], 4)
    with pytest.raises(chym.ChymError) as err:
        b.status()
    assert err.value.status == chym.ETIMEOUT
    b.status()   # cleared
    # restart every context from its seeds and integrate normally
    for k, (c, eps, sch) in enumerate(batched):
        c.run(_params(eps, chym.PREC_BF16X2, False), inputs.pump_grid(0.5, 2),
              inputs.run_seeds(91 + k, 24), 0, sch)
    b.run([_params(e, chym.PREC_BF16X2, False) for _, e, _ in batched], [s for _, _, s in batched], 30)
    b.status()
    b.close()
    for (c, eps, sch), (ca, _, _) in zip(make(), batched):
        c.run(_params(eps, chym.PREC_BF16X2, False), None, None, 30, sch)
        assert np.array_equal(c.get_state()[0], ca.get_state()[0])
        c.close()
        ca.close()
