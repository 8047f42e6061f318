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


def test_raw_abi_error_codes():
    """Error paths of the C ABI called directly (independent binding; the
    planner runs host-only with SYM_PLAN_DRYRUN=1, so no GPU is needed)."""
    import ctypes

    from tests import abi_raw as R
    os.environ["SYM_PLAN_DRYRUN"] = "1"
    try:
        lib = R.load()
        q = [-1, 0, 1]
        rc, a = R.tensor(lib, R.SYM_U1, [(q, [2, 3, 1], 1), (q, [1, 2, 2], -1)])
        assert rc == R.SYM_OK and R.numel(lib, a) == 2 * 1 + 3 * 2 + 1 * 2
        rc, b = R.tensor(lib, R.SYM_U1, [(q, [1, 2, 3], 1), (q, [1, 1, 1], -1)])  # leg 0 differs from a's leg 1
        assert rc == R.SYM_OK
        c, p = ctypes.c_void_p(), ctypes.c_void_p()
        # contracted legs must carry the same labels and degeneracies with opposite directions
        rc = lib.sym_contract_plan(a, b, 1, R.ints([1]), R.ints([0]), None, R.SYM_PREC_FP64, ctypes.byref(c),
                                   ctypes.byref(p))
        assert rc == R.SYM_ERR_INCOMPATIBLE_LEGS and b"same labels" in lib.sym_last_error()
        rc, d = R.tensor(lib, R.SYM_U1, [(q, [2, 3, 1], 1), (q, [2, 3, 1], -1)])  # d's leg 1 pairs with its leg 0
        assert rc == R.SYM_OK
        # bad precision, repeated pair, NULL outputs
        assert lib.sym_contract_plan(d, d, 1, R.ints([1]), R.ints([0]), None, 9, ctypes.byref(c),
                                     ctypes.byref(p)) == R.SYM_ERR_ARG
        assert lib.sym_contract_plan(d, d, 2, R.ints([1, 1]), R.ints([0, 0]), None, R.SYM_PREC_FP64,
                                     ctypes.byref(c), ctypes.byref(p)) == R.SYM_ERR_ARG
        assert lib.sym_contract_plan(d, d, 1, R.ints([1]), R.ints([0]), None, R.SYM_PREC_FP64, None,
                                     None) == R.SYM_ERR_ARG
        # a valid plan built host-only refuses to run
        assert lib.sym_contract_plan(d, d, 1, R.ints([1]), R.ints([0]), None, R.SYM_PREC_FP64, ctypes.byref(c),
                                     ctypes.byref(p)) == R.SYM_OK
        assert lib.sym_contract(p, None, None, None, None) == R.SYM_ERR_UNSUPPORTED
        assert lib.sym_plan_destroy(p) == R.SYM_OK and lib.sym_tensor_destroy(c) == R.SYM_OK
        # the eigendecomposition needs the column legs to be the row legs reversed
        e, nb, nev = ctypes.c_void_p(), ctypes.c_int(), ctypes.c_int64()
        assert lib.sym_eig_plan(b, 1, ctypes.byref(e), ctypes.byref(nb), ctypes.byref(nev)) == \
            R.SYM_ERR_INCOMPATIBLE_LEGS
        rc, s = R.tensor(lib, R.SYM_U1, [(q, [2, 3, 1], -1), (q, [2, 3, 1], 1)])
        assert lib.sym_eig_plan(s, 1, ctypes.byref(e), ctypes.byref(nb), ctypes.byref(nev)) == R.SYM_OK
        assert nb.value == 3 and nev.value == 6
        assert lib.sym_svd_destroy(e) == R.SYM_OK
        # SU(2): a tree that is not planar is refused
        rc, _ = R.tensor(lib, R.SYM_SU2, [([1], [1], 1)] * 3, tree=[(0, 2), (3, 1)])
        assert rc == R.SYM_ERR_ARG
        for h in (a, b, d, s):
            assert lib.sym_tensor_destroy(h) == R.SYM_OK
    finally:
        del os.environ["SYM_PLAN_DRYRUN"]


def test_fuse_of_several_legs_is_the_iterated_pairwise_fuse():
    """The structure sym_fuse_n_plan returns equals that of n-1 pairwise
    fuses, and a chained plan runs all of them (host-only plans)."""
    import subprocess
    import sys
    code = (
        "import paper_1203_2222_gb300 as P\n"
        "for g, legs in ((P.U1, [([-1, 0, 1], [2, 1, 2], 1), ([0, 1], [1, 2], 1), ([-1, 0], [2, 1], 1), "
        "([0], [3], -1)]), (P.SU2, [([0, 1, 2], [2, 1, 1], 1), ([0, 1], [1, 2], 1), ([1, 2], [2, 1], 1), "
        "([0, 1, 2, 3], [1, 2, 1, 1], 1)])):\n"
        "    S = P.Structure(g, legs)\n"
        "    a = P.fuse_plan(S, 0, P.FP64, nlegs=3).out\n"
        "    b = P.fuse_plan(P.fuse_plan(S, 0, P.FP64).out, 0, P.FP64).out\n"
        "    assert a.legs == b.legs and a.numel == b.numel, (a.legs, b.legs)\n"
        "print('ok')\n")
    env = dict(os.environ, SYM_PLAN_DRYRUN="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr
