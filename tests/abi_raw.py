"""A second, independent ctypes binding of libsymtensor.so written from
include/symtensor.h alone (test helper): the raw C-ABI tests call the library
through it, not through the package's own binding."""
import ctypes
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_1203_2222_gb300", "_build", "libsymtensor.so")

SYM_OK, SYM_ERR_ARG, SYM_ERR_INCOMPATIBLE_LEGS, SYM_ERR_UNSUPPORTED = 0, -1, -2, -7
SYM_U1, SYM_SU2 = 1, 2
SYM_PREC_FP64, SYM_PREC_BF16X3 = 1, 2


class Leg(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("labels", ctypes.POINTER(ctypes.c_int)),
                ("degens", ctypes.POINTER(ctypes.c_int)), ("dir", ctypes.c_int)]


P, I, IP, LP, DP = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64), \
    ctypes.POINTER(ctypes.c_double)
PP = ctypes.POINTER(ctypes.c_void_p)


def load():
    lib = ctypes.CDLL(LIB)
    sigs = {
        "sym_last_error": ([], ctypes.c_char_p),
        "sym_tensor_create": ([I, I, ctypes.POINTER(Leg), I, IP, PP], I),
        "sym_tensor_destroy": ([P], I),
        "sym_tensor_info": ([P, IP, IP, LP, LP], I),
        "sym_tensor_tree": ([P, IP], I),
        "sym_permute_plan": ([P, IP, IP, I, PP, PP], I),
        "sym_plan_execute": ([P, P, P, P], I),
        "sym_contract_plan": ([P, P, I, IP, IP, IP, I, PP, PP], I),
        "sym_contract": ([P, P, P, P, P], I),
        "sym_contract_backward": ([P, P, P, P, P, P, P], I),
        "sym_plan_destroy": ([P], I),
        "sym_device_status": ([], I),
        "sym_eig_plan": ([P, I, PP, IP, LP], I),
        "sym_eig_execute": ([P, P, P, P], I),
        "sym_svd_destroy": ([P], I),
    }
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes, f.restype = args, res
    return lib


def ints(values):
    values = [int(v) for v in values]
    return (ctypes.c_int * max(len(values), 1))(*values)


def tensor(lib, group, legs, total=0, tree=None):
    """sym_tensor_create from (labels, degens, dir) legs; returns (rc, handle)."""
    arr = (Leg * max(len(legs), 1))()
    keep = []
    for i, (lab, deg, d) in enumerate(legs):
        la, de = ints(lab), ints(deg)
        keep += [la, de]
        arr[i].n, arr[i].labels, arr[i].degens, arr[i].dir = len(lab), la, de, int(d)
    tr = None if tree is None else ints([x for node in tree for x in node])
    h = ctypes.c_void_p()
    rc = lib.sym_tensor_create(group, len(legs), arr, total, tr, ctypes.byref(h))
    return rc, h


def numel(lib, h):
    n = ctypes.c_int64()
    assert lib.sym_tensor_info(h, None, None, ctypes.byref(n), None) == SYM_OK
    return n.value
