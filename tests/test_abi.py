"""The C-ABI library loads and exports every entry point include/symtensor.h declares (no GPU)."""
import ctypes
import os
import re

from tests.conftest import ROOT


def _declared():
    text = open(os.path.join(ROOT, "include", "symtensor.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sym_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_1203_2222_gb300 import _lib
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(_lib.lib, n), n
        assert ctypes.cast(getattr(_lib.lib, n), ctypes.c_void_p).value


def test_version_and_error_reporting():
    from paper_1203_2222_gb300 import _lib
    assert b"sm_103a" in _lib.lib.sym_version()
    h = ctypes.c_void_p()
    rc = _lib.lib.sym_tensor_create(7, 0, None, 0, None, ctypes.byref(h))
    assert rc == _lib.SYM_ERR_ARG
    assert b"group" in _lib.lib.sym_last_error()


def test_bad_legs_are_rejected():
    import pytest
    from paper_1203_2222_gb300 import SymError, Structure, U1, SU2
    with pytest.raises(SymError):
        Structure(U1, [([0, 0], [1, 1], 1)])          # labels must increase
    with pytest.raises(SymError):
        Structure(U1, [([0], [0], 1)])                # degeneracy >= 1
    with pytest.raises(SymError):
        Structure(SU2, [([0, 1], [1, 1], 2)])         # direction +-1
    with pytest.raises(SymError):
        Structure(SU2, [([1], [1], 1)] * 3, tree=[(0, 2), (3, 1)])  # not planar
