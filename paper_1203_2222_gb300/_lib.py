"""ctypes binding of ``libsymtensor.so`` (include/symtensor.h): argument marshalling only.

The library is built in-tree by ``paper_1203_2222_gb300/build.py``.  If it is
missing, importing this module raises: there is no fallback path.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# SYMTENSOR_LIB selects another build of the same library (e.g. an
# instrumented one); the default is the in-tree build.
LIB_PATH = os.environ.get("SYMTENSOR_LIB") or os.path.join(HERE, "_build", "libsymtensor.so")

SYM_OK = 0
SYM_ERR_ARG = -1
SYM_ERR_INCOMPATIBLE_LEGS = -2
SYM_ERR_CUDA = -4
SYM_ERR_TIMEOUT = -5
SYM_ERR_OOM = -6
SYM_ERR_UNSUPPORTED = -7
SYM_ERR_NUMERIC = -8
SYM_U1 = 1
SYM_SU2 = 2
SYM_Z2F = 3
SYM_SU2U1 = 4
SYM_PREC_FP64 = 1
SYM_PREC_BF16X3 = 2

ERR_NAMES = {
    SYM_ERR_ARG: "SYM_ERR_ARG", SYM_ERR_INCOMPATIBLE_LEGS: "SYM_ERR_INCOMPATIBLE_LEGS",
    SYM_ERR_CUDA: "SYM_ERR_CUDA", SYM_ERR_TIMEOUT: "SYM_ERR_TIMEOUT", SYM_ERR_OOM: "SYM_ERR_OOM",
    SYM_ERR_UNSUPPORTED: "SYM_ERR_UNSUPPORTED", SYM_ERR_NUMERIC: "SYM_ERR_NUMERIC",
}


class SymError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class sym_leg(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("labels", ctypes.POINTER(ctypes.c_int)),
                ("degens", ctypes.POINTER(ctypes.c_int)), ("dir", ctypes.c_int)]


TUNE_FIELDS = ("tc_min_mn", "tc_min_k", "tc_max_k", "direct_max", "direct_chunk", "rows_spans", "splitk_ctas",
               "thin_slice", "tc_order", "tc_group", "direct_mixed", "tc_all")


class sym_tune(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int) for f in TUNE_FIELDS]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_1203_2222_gb300/build.py` "
                      "(or __graft_entry__.build())")

lib = ctypes.CDLL(LIB_PATH)

_P = ctypes.c_void_p
_I = ctypes.c_int
_IP = ctypes.POINTER(ctypes.c_int)
_LP = ctypes.POINTER(ctypes.c_int64)
_DP = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "sym_last_error": ([], ctypes.c_char_p),
    "sym_version": ([], ctypes.c_char_p),
    "sym_tensor_create": ([_I, _I, ctypes.POINTER(sym_leg), _I, _IP, ctypes.POINTER(_P)], _I),
    "sym_tensor_destroy": ([_P], _I),
    "sym_tensor_info": ([_P, _IP, _IP, _LP, _LP], _I),
    "sym_tensor_leg": ([_P, _I, _IP, _IP, _IP, _IP], _I),
    "sym_tensor_tree": ([_P, _IP], _I),
    "sym_tensor_sectors": ([_P, _IP, _LP], _I),
    "sym_permute_plan": ([_P, _IP, _IP, _I, ctypes.POINTER(_P), ctypes.POINTER(_P)], _I),
    "sym_fuse_plan": ([_P, _I, _I, ctypes.POINTER(_P), ctypes.POINTER(_P)], _I),
    "sym_fuse_n_plan": ([_P, _I, _I, _I, ctypes.POINTER(_P), ctypes.POINTER(_P)], _I),
    "sym_split_plan": ([_P, _I, ctypes.POINTER(sym_leg), _I, ctypes.POINTER(_P), ctypes.POINTER(_P)], _I),
    "sym_plan_execute": ([_P, _P, _P, _P], _I),
    "sym_contract_plan": ([_P, _P, _I, _IP, _IP, _IP, _I, ctypes.POINTER(_P), ctypes.POINTER(_P)], _I),
    "sym_contract_batch_plan": ([_I, ctypes.POINTER(_P), ctypes.POINTER(_P), _I, _IP, _IP, _I,
                                 ctypes.POINTER(_P), _LP, ctypes.POINTER(_P)], _I),
    "sym_contract": ([_P, _P, _P, _P, _P], _I),
    "sym_contract_backward": ([_P, _P, _P, _P, _P, _P, _P], _I),
    "sym_plan_stats": ([_P, _DP, _LP, _LP, _LP], _I),
    "sym_plan_launches": ([_P, _IP], _I),
    "sym_plan_profile": ([_P, _I], _I),
    "sym_plan_profile_read": ([_P, _I, _IP, _DP, _DP, _DP], _I),
    "sym_plan_profile_kernel": ([_P, _I, _IP, _DP, _DP, _DP], _I),
    "sym_plan_destroy": ([_P], _I),
    "sym_plan_gemm_shapes": ([_P, _IP, _IP], _I),
    "sym_device_status": ([], _I),
    "sym_wait_probe": ([_I, _I], _I),
    "sym_su2_F": ([_I, _I, _I, _I, _I, _I, _DP], _I),
    "sym_contract_noalloc": ([_P, _P, _I, _IP, _IP, _I, _P, _P, _P, _P], _I),
    "sym_su2_gamma": ([_I, _IP, _IP, _IP, _IP, _IP, _IP, _DP, _IP, _IP], _I),
    "sym_tune_get": ([ctypes.POINTER(sym_tune)], _I),
    "sym_tune_set": ([ctypes.POINTER(sym_tune)], _I),
    "sym_tune_epoch": ([_IP], _I),
    "sym_svd_plan": ([_P, _I, ctypes.POINTER(_P), _IP, _LP], _I),
    "sym_svd_blocks": ([_P, _IP, _IP, _IP], _I),
    "sym_svd_execute": ([_P, _P, _P, _P], _I),
    "sym_svd_stats": ([_P, _I, _IP, _LP], _I),
    "sym_svd_truncation": ([_P, _DP, ctypes.c_int64, ctypes.c_double, _IP], _I),
    "sym_svd_bond": ([_P, _IP, ctypes.POINTER(_P), ctypes.POINTER(_P)], _I),
    "sym_svd_factors": ([_P, _I, _P, _P, _P, _P], _I),
    "sym_svd_destroy": ([_P], _I),
    "sym_eig_plan": ([_P, _I, ctypes.POINTER(_P), _IP, _LP], _I),
    "sym_eig_execute": ([_P, _P, _P, _P], _I),
    "sym_eig_truncation": ([_P, _DP, ctypes.c_int64, ctypes.c_double, _IP], _I),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def check(rc):
    if rc != SYM_OK:
        raise SymError(rc, lib.sym_last_error().decode())
    return rc


def int_array(values):
    values = [int(v) for v in values]
    return (ctypes.c_int * max(len(values), 1))(*values)


def leg_array(legs):
    """legs: sequence of (labels, degens, dir) -> (ctypes array, keep-alive list)."""
    keep = []
    arr = (sym_leg * max(len(legs), 1))()
    for i, (labels, degens, d) in enumerate(legs):
        la, de = int_array(labels), int_array(degens)
        keep += [la, de]
        arr[i].n = len(labels)
        arr[i].labels = la
        arr[i].degens = de
        arr[i].dir = int(d)
    return arr, keep


def tree_array(nodes):
    if nodes is None:
        return None
    flat = [c for nd in nodes for c in nd]
    return int_array(flat)
