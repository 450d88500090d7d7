"""CPU checks of the C-ABI library: it builds, loads, exports every symbol
include/smm.h declares, and its host-side quadrature matches the oracle."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2304_07386_gb300 import build as B
    from paper_2304_07386_gb300.smm import load_library
    B.build()
    return load_library()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(smm_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"smm_create", "smm_sweep", "smm_moments", "smm_moment_solve", "smm_iterate", "smm_destroy"} <= names
    for n in names:
        assert hasattr(lib, n), n


def test_quadrature_matches_oracle(lib):
    from oracle.quadrature import level_symmetric_2d
    from paper_2304_07386_gb300 import smm_quadrature
    for N in (2, 4, 6, 8, 10, 12):
        om, w = smm_quadrature(N)
        om2, w2 = level_symmetric_2d(N)
        assert np.array_equal(om, om2)
        assert np.max(np.abs(w - w2)) < 1e-12


def test_invalid_arguments_rejected(lib):
    from paper_2304_07386_gb300 import SMMError, smm_quadrature
    with pytest.raises(SMMError):
        smm_quadrature(5)
