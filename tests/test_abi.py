"""The C ABI library on a machine without a GPU: it loads, exports every
function include/*.h declares, and its host-only logic (element matrix,
edof table, filter stencil, argument checks) agrees with the oracle.  No
device work is requested here."""
import ctypes as C
import re
from pathlib import Path

import numpy as np
import pytest

from oracle import fem, filter as cone

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    names = set()
    for hdr in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", hdr.read_text(), flags=re.S)
        names.update(re.findall(r"\b(mfto_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def mf():
    from paper_2604_18020_gb300 import build, mfto
    build.build()
    return mfto


def test_every_declared_symbol_is_exported(mf):
    lib = mf.lib()
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding knows every one of them
    assert set(names) <= set(mf.SIGNATURES), set(names) - set(mf.SIGNATURES)


def test_unit_ke_matches_oracle(mf):
    for nu, h in [(0.3, 1.0), (0.3, 2.0), (0.0, 0.5), (0.45, 1.0)]:
        a = mf.unit_ke(1.0, nu, h)
        b = fem.ke_gauss(1.0, nu, h)
        assert np.abs(a - b).max() <= 1e-15 * max(1.0, np.abs(b).max()) * 4


def test_edof_bit_exact(mf):
    for shape in [(1, 1, 1), (2, 1, 1), (5, 3, 4), (24, 12, 12)]:
        assert np.array_equal(mf.edof(*shape).astype(np.int64), fem.edof_table_fast(*shape))


@pytest.mark.parametrize("rmin", [0.9, 1.5, 2.0, 2.7, 3.0, 4.5])
def test_filter_stencil_bit_exact(mf, rmin):
    off, w = mf.filter_stencil(rmin)
    ref = cone.stencil(rmin)
    assert off.tolist() == [[dx, dy, dz] for dx, dy, dz, _ in ref]
    assert np.array_equal(w, np.array([x[3] for x in ref]))


def test_argument_checks_without_device(mf):
    lib = mf.lib()
    p = mf.default_params()
    assert (p.E0, p.Emin, p.nu, p.penal, p.rtol, p.maxit) == (1.0, 1e-9, 0.3, 3.0, 1e-8, 10000)
    out = C.c_void_p()
    fixed = np.zeros(8, dtype=np.uint8)
    for mesh in [mf.Mesh(0, 1, 1, 1.0), mf.Mesh(1, -2, 1, 1.0), mf.Mesh(1, 1, 1, 0.0),
                 mf.Mesh(2000, 2000, 2000, 1.0)]:          # last: n_dof > INT32_MAX
        assert lib.mfto_create(C.byref(mesh), C.byref(p), fixed.ctypes.data, None,
                               C.byref(out)) == mf.INVALID_ARG
        assert not out.value
    bad = mf.default_params(nu=0.5)
    assert lib.mfto_create(C.byref(mf.Mesh(1, 1, 1, 1.0)), C.byref(bad), fixed.ctypes.data,
                           None, C.byref(out)) == mf.INVALID_ARG
    assert lib.mfto_unit_ke(1.0, 0.6, 1.0, np.zeros(576).ctypes.data) == mf.INVALID_ARG
    n = C.c_int32()
    assert lib.mfto_filter_stencil(1.5, 3, None, None, C.byref(n)) == mf.INVALID_ARG
    assert n.value == 19
