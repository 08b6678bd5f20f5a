"""The allocation-free statistics entry point against chym_stats.

chym_stats_noalloc serves callers that cannot allocate device memory where they
need the statistics (a framework owning the device pool, fixed-budget real-time
loops, code that must not trigger cudaMalloc's implicit synchronisation).  It
keeps its result block in a fixed device array inside the library, so this test
checks it against the context-based chym_stats on two calls in a row, with
different inputs, through the C ABI.  The file is named so pytest collects it last.
"""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2308_02329_gb300 import chym
from tests.helpers import make_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chym.lib()
    return torch


def _energies(torch, N, D, n_h, reps, seed, steps, kind=chym.J_PM1, graph="sk"):
    J, eps, h, seeds = make_case(N, D, n_h, reps, seed, graph)
    ctx = chym.Context(J, D, kind)
    ctx.run(chym.Params(eps=eps, prec=chym.PREC_FP32), h, seeds, steps,
            chym.Schedule(1, steps // 2, steps))
    d_E = torch.empty(n_h * reps, dtype=torch.float64, device="cuda")
    ctx.energy_device(d_E.data_ptr(), 0, 0)
    torch.cuda.synchronize()
    return J, ctx, d_E


def _same(a, b):
    if "hits" in a:
        assert a["hits"].tolist() == b["hits"].tolist()
    if "hist" in a or "hist" in b:
        assert a["hist"].tolist() == b["hist"].tolist()
    for k in ("P_max", "W_range", "W_scan", "dE_mean", "best_E"):
        assert a[k] == pytest.approx(b[k], rel=1e-12, abs=1e-12)
    for k in ("best_run", "n_finite", "n_hits"):
        assert a[k] == b[k]


def test_stats_noalloc_matches_chym_stats_twice(torch_cuda):
    torch = torch_cuda
    # call 1: +-1 couplings, exact ground state, 64-bin histogram
    J1, c1, d_E1 = _energies(torch, 16, 2, 4, 16, 5, 1500)
    E1_gs = O.ground_state_bruteforce(J1)[0]
    ref1 = c1.stats(E1_gs, n_bins=64)
    got1 = chym.stats_noalloc(d_E1.data_ptr(), 64, 4, chym.J_PM1, E1_gs, n_bins=64)
    _same(got1, ref1)
    assert ref1["n_hits"] > 0
    # call 2: different sizes and real couplings; nothing of call 1 may leak through
    J2, c2, d_E2 = _energies(torch, 24, 3, 3, 7, 9, 400, kind=chym.J_REAL, graph="gauss")
    E2 = d_E2.cpu().numpy()
    E2_gs = float(E2.min())
    ref2 = c2.stats(E2_gs, n_bins=16)
    got2 = chym.stats_noalloc(d_E2.data_ptr(), 21, 3, chym.J_REAL, E2_gs, n_bins=16)
    _same(got2, ref2)
    # and call 1's inputs again, without a histogram
    got3 = chym.stats_noalloc(d_E1.data_ptr(), 64, 4, chym.J_PM1, E1_gs)
    _same(got3, c1.stats(E1_gs))
    c1.close()
    c2.close()


def test_stats_noalloc_rejects_sizes_beyond_its_array(torch_cuda):
    torch = torch_cuda
    d_E = torch.zeros(8192, dtype=torch.float64, device="cuda")
    with pytest.raises(chym.ChymError) as e:
        chym.stats_noalloc(d_E.data_ptr(), 8192, 8192, chym.J_PM1, 0.0)
    assert e.value.status == chym.EINVAL and "4096" in str(e.value)
    with pytest.raises(chym.ChymError) as e:
        chym.stats_noalloc(d_E.data_ptr(), 8192, 8, chym.J_PM1, 0.0, n_bins=70000)
    assert e.value.status == chym.EINVAL


def test_stats_noalloc_without_a_hits_buffer_over_many_pumps(torch_cuda):
    # no per-pump buffer from the caller and more pumps than one 64-count slice: the
    # figures that need every per-pump count (P_max, W) must still match chym_stats
    torch = torch_cuda
    n_h, reps = 96, 4
    J, c, d_E = _energies(torch, 16, 2, n_h, reps, 11, 1500)
    E_gs = O.ground_state_bruteforce(J)[0]
    ref = c.stats(E_gs, n_bins=32)
    assert ref["n_hits"] > 0
    for _ in range(2):
        got = chym.stats_noalloc(d_E.data_ptr(), n_h * reps, n_h, chym.J_PM1, E_gs, n_bins=32,
                                 with_hits=False)
        assert "hits" not in got
        _same(got, ref)
    c.close()
