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


def test_struct_layouts_match_the_header(tmp_path):
    """The Python mirror of every struct in include/smm.h has the header's size
    and field offsets (a C program compiled against the header prints them)."""
    import ctypes
    import shutil
    import subprocess
    from paper_2304_07386_gb300 import smm as S
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [S.smm_mesh, S.smm_options, S.smm_info, S.smm_stats]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "smm.h"', "int main(void) {"]
    for st in structs:
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (st.__name__, st.__name__))
        for name, _ in st._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (st.__name__, name, st.__name__, name))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st in structs:
        assert got[(st.__name__, "sizeof")] == ctypes.sizeof(st), st.__name__
        for name, _ in st._fields_:
            assert got[(st.__name__, name)] == getattr(st, name).offset, (st.__name__, name)


def test_default_options(lib):
    """The defaults the header documents: FP64 sweep with cached inverses,
    multigrid CG with degree-3 Chebyshev smoothing run as one device-side loop."""
    from paper_2304_07386_gb300 import smm as S
    from paper_2304_07386_gb300 import smm_default_options
    o = smm_default_options()
    assert o.sweep_precision == S.SMM_SWEEP_FP64 and o.sweep_solver == S.SMM_SOLVER_CACHED_INVERSE
    assert o.precond == S.SMM_PRECOND_MULTIGRID
    assert o.mg_smoother == S.SMM_SMOOTHER_CHEBYSHEV and o.mg_smooth_steps == 3
    assert o.cg_device_loop == 1 and o.sweep_tiles == 1 and o.negative_flux_fixup == 0
    assert o.moment_discretization == S.SMM_MOMENT_IP
    assert o.cg_tol_adaptive == 0.0 and o.cycle_lagging == 1 and o.cg_guess_extrapolate == 1


class _FakeDeviceBuffer:
    """Just enough of a CUDA float64 tensor for the binding's pointer checks
    (no device is touched: only the checks before a C call run)."""

    def __init__(self, numel, dtype="torch.float64"):
        self._numel, self.dtype, self.is_cuda = numel, dtype, True

    def is_contiguous(self):
        return True

    def numel(self):
        return self._numel

    def data_ptr(self):
        return 4096


class _FakeHandle:
    def __init__(self, n_phi):
        self._n = n_phi

    def n_phi(self):
        return self._n


def test_binding_rejects_buffers_of_the_wrong_size():
    """The C calls take bare device pointers, so the binding checks each
    buffer's element count against the layout the header states before the
    call: a short buffer would be read or written past its end."""
    from paper_2304_07386_gb300 import smm as S
    assert S._devbuf(None, 10, "phi") is None
    assert S._devbuf(_FakeDeviceBuffer(10), 10, "phi").value == 4096
    for bad in (9, 11):
        with pytest.raises(ValueError, match="phi"):
            S._devbuf(_FakeDeviceBuffer(bad), 10, "phi")
    with pytest.raises(ValueError):
        S._devbuf(_FakeDeviceBuffer(10, "torch.float32"), 10, "phi")
    hs = [_FakeHandle(8), _FakeHandle(12)]
    arr = S._ptr_array(hs, [_FakeDeviceBuffer(8), None])
    assert arr[0] == 4096 and arr[1] is None
    with pytest.raises(ValueError, match=r"phi\[1\]"):
        S._ptr_array(hs, [_FakeDeviceBuffer(8), _FakeDeviceBuffer(8)])
    with pytest.raises(ValueError, match="expected 2 buffers"):
        S._ptr_array(hs, [_FakeDeviceBuffer(8)])
