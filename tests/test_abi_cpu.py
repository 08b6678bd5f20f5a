"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point declared in include/*.h, and rejects invalid arguments before any
device work (no GPU needed)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2308_02329_gb300 import build as lib_build
from paper_2308_02329_gb300 import chym, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names |= set(re.findall(r"CHYM_API\s+[\w\s\*]*?\b(chym_\w+)\s*\(", src))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    path = lib_build.build()
    L = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/ but not exported"
    assert set(names) == set(chym.EXPORTS) | (set(names) - set(chym.EXPORTS))
    for n in chym.EXPORTS:
        assert n in names


def test_create_rejects_invalid_couplings_without_gpu():
    with pytest.raises(chym.ChymError) as e:
        chym.Context(np.ones((4, 4)), 2)
    assert e.value.status == chym.EINVAL
    J = inputs.sk_pm1(6, 1)
    J[0, 1] = 0.5
    with pytest.raises(chym.ChymError) as e:
        chym.Context(J, 2)
    assert e.value.status == chym.EINVAL and "symmetric" in str(e.value)
    J = inputs.sk_pm1(6, 1)
    J[0, 1] = J[1, 0] = 2.0
    with pytest.raises(chym.ChymError) as e:
        chym.Context(J, 2, chym.J_PM1)
    assert e.value.status == chym.EINVAL
    with pytest.raises(chym.ChymError) as e:
        chym.Context(inputs.sk_pm1(6, 1), 9)
    assert e.value.status == chym.EINVAL
    with pytest.raises(chym.ChymError) as e:
        chym.Context(np.zeros((0, 0)), 2)
    assert e.value.status == chym.EINVAL


def test_null_context_calls_are_rejected():
    L = chym.lib()
    assert L.chym_destroy(None) == chym.OK
    assert L.chym_info(None, None, None, None) == chym.EINVAL
    assert L.chym_energy(None, None, None, None) == chym.EINVAL
    assert b"NULL" in L.chym_last_error()
