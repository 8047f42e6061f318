"""GPU parity through the bare C ABI: every call below goes through an
independent ctypes binding written from include/symtensor.h (tests/abi_raw.py),
not through the package.  Device buffers come from torch (plumbing only).

  * U(1) contraction with multi-tile ragged sectors: sym_contract_plan,
    sym_contract, sym_contract_backward, FP64 (1e-12) and split-BF16 (2e-5);
  * SU(2) permute into another tree: sym_permute_plan + sym_plan_execute;
  * symmetric eigendecomposition: sym_eig_plan + sym_eig_execute;
each against the FP64 oracle."""
import ctypes

import numpy as np
import pytest

import abi_raw as R

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _rel(x, y):
    return float(np.linalg.norm(np.asarray(x) - np.asarray(y)) / max(np.linalg.norm(y), 1e-300))


@pytest.mark.parametrize("prec,dtype,tol", [(R.SYM_PREC_FP64, torch.float64, 1e-12),
                                            (R.SYM_PREC_BF16X3, torch.float32, 2e-5)], ids=["fp64", "bf16x3"])
def test_raw_u1_contraction_forward_and_backward(prec, dtype, tol):
    from oracle import contract as oc
    from oracle import u1
    lib = R.load()
    q = [-1, 0, 1]
    la = [(q, [70, 150, 33], -1), (q, [5, 9, 2], 1), (q, [90, 140, 61], 1)]
    lb = [(q, [90, 140, 61], -1), (q, [100, 131, 7], 1)]
    rc, A = R.tensor(lib, R.SYM_U1, la)
    assert rc == R.SYM_OK
    rc, B = R.tensor(lib, R.SYM_U1, lb)
    assert rc == R.SYM_OK
    C, plan = ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.sym_contract_plan(A, B, 1, R.ints([2]), R.ints([0]), None, prec, ctypes.byref(C),
                                 ctypes.byref(plan)) == R.SYM_OK, lib.sym_last_error()
    rng = np.random.default_rng(21)
    a = torch.as_tensor(rng.standard_normal(R.numel(lib, A))).to(dtype).cuda()
    b = torch.as_tensor(rng.standard_normal(R.numel(lib, B))).to(dtype).cuda()
    nc = R.numel(lib, C)
    c = torch.empty(nc, dtype=dtype, device="cuda")
    assert lib.sym_contract(plan, _ptr(a), _ptr(b), _ptr(c), _stream()) == R.SYM_OK, lib.sym_last_error()
    dc = torch.as_tensor(rng.standard_normal(nc)).to(dtype).cuda()
    da, db = torch.empty_like(a), torch.empty_like(b)
    assert lib.sym_contract_backward(plan, _ptr(a), _ptr(b), _ptr(dc), _ptr(da), _ptr(db), _stream()) == R.SYM_OK
    torch.cuda.synchronize()
    assert lib.sym_device_status() == R.SYM_OK
    oA = ([u1.Leg(*l) for l in la], 0, a.double().cpu().numpy())
    oB = ([u1.Leg(*l) for l in lb], 0, b.double().cpu().numpy())
    _, _, c_ref, _ = oc.contract("u1", oA, oB, [2], [0])
    dA_ref, dB_ref, _ = oc.contract_grad("u1", oA, oB, [2], [0], dc.double().cpu().numpy())
    assert _rel(c.double().cpu().numpy(), c_ref) <= tol
    assert _rel(da.double().cpu().numpy(), dA_ref) <= tol
    assert _rel(db.double().cpu().numpy(), dB_ref) <= tol
    for h in (plan,):
        assert lib.sym_plan_destroy(h) == R.SYM_OK
    for h in (A, B, C):
        assert lib.sym_tensor_destroy(h) == R.SYM_OK


def test_raw_su2_permute_into_another_tree():
    from oracle import contract as oc
    from oracle import su2
    lib = R.load()
    sp = [0, 1, 2, 3]
    legs = [(sp, [2, 1, 1, 1], 1), (sp, [1, 2, 1, 1], -1), (sp, [1, 1, 2, 1], 1), (sp, [1, 1, 1, 2], 1)]
    tree_in = [(1, 2), (0, 4), (5, 3)]
    rc, T = R.tensor(lib, R.SYM_SU2, legs, tree=tree_in)
    assert rc == R.SYM_OK
    perm, tree_out = [2, 0, 3, 1], [(0, 1), (2, 3), (4, 5)]
    O, plan = ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.sym_permute_plan(T, R.ints(perm), R.ints([x for n in tree_out for x in n]), R.SYM_PREC_FP64,
                                ctypes.byref(O), ctypes.byref(plan)) == R.SYM_OK, lib.sym_last_error()
    t = torch.as_tensor(np.random.default_rng(22).standard_normal(R.numel(lib, T))).cuda()
    o = torch.empty(R.numel(lib, O), dtype=torch.float64, device="cuda")
    assert lib.sym_plan_execute(plan, _ptr(t), _ptr(o), _stream()) == R.SYM_OK
    torch.cuda.synchronize()
    oT = ([su2.Leg(*l) for l in legs], tree_in, t.cpu().numpy())
    _, _, ref, resid = oc.permute("su2", oT, perm, tree_out)
    assert resid < 1e-12
    assert _rel(o.cpu().numpy(), ref) <= 1e-12
    assert lib.sym_plan_destroy(plan) == R.SYM_OK
    for h in (T, O):
        assert lib.sym_tensor_destroy(h) == R.SYM_OK


def test_raw_eigendecomposition():
    from oracle import eig as oeig
    from oracle import u1
    lib = R.load()
    q = [-2, -1, 0, 1]
    legs = [(q, [20, 33, 41, 12], -1), (q, [20, 33, 41, 12], 1)]
    ol = [u1.Leg(*l) for l in legs]
    n = u1.layout(ol, 0)[2]
    d = u1.embed(ol, 0, np.random.default_rng(23).standard_normal(n))
    vals, _ = u1.extract(ol, 0, 0.5 * (d + d.T))
    rc, T = R.tensor(lib, R.SYM_U1, legs)
    assert rc == R.SYM_OK
    plan, nb, nev = ctypes.c_void_p(), ctypes.c_int(), ctypes.c_int64()
    assert lib.sym_eig_plan(T, 1, ctypes.byref(plan), ctypes.byref(nb), ctypes.byref(nev)) == R.SYM_OK
    t = torch.as_tensor(vals).cuda()
    lam = torch.empty(nev.value, dtype=torch.float64, device="cuda")
    assert lib.sym_eig_execute(plan, _ptr(t), _ptr(lam), _stream()) == R.SYM_OK
    torch.cuda.synchronize()
    assert lib.sym_device_status() == R.SYM_OK
    fac, _ = oeig.eig("u1", (ol, 0, vals), 1)
    ref = np.concatenate([fac[x][1] for x in sorted(fac)])  # blocks in ascending label, |lambda| descending
    got = lam.cpu().numpy()
    assert len(got) == len(ref)
    lmax = float(np.max(np.abs(ref)))
    off = 0
    for x in sorted(fac):
        k = len(fac[x][1])
        assert np.max(np.abs(np.sort(got[off:off + k]) - np.sort(ref[off:off + k]))) <= 1e-12 * lmax
        off += k
    assert lib.sym_svd_destroy(plan) == R.SYM_OK
    assert lib.sym_tensor_destroy(T) == R.SYM_OK


@pytest.mark.parametrize("prec,dtype", [(R.SYM_PREC_FP64, torch.float64), (R.SYM_PREC_BF16X3, torch.float32)],
                         ids=["fp64", "bf16x3"])
def test_raw_sectors_without_contributions_are_written_as_zeros(prec, dtype):
    """C's sector (a = 1, b = 1) is allowed by charge conservation but no
    block of A has a = 1, so nothing contributes to it: the library must
    write it as zeros (the outputs start as NaN here), and likewise the
    gradient blocks of A and B that receive nothing."""
    from oracle import contract as oc
    from oracle import u1
    lib = R.load()
    la = [([0, 1], [2, 3], 1), ([0], [2], -1)]   # A: only the block a = 0
    lb = [([0], [2], 1), ([0, 1], [3, 2], -1)]   # B: only the block b = 0
    rc, A = R.tensor(lib, R.SYM_U1, la)
    assert rc == R.SYM_OK
    rc, B = R.tensor(lib, R.SYM_U1, lb)
    assert rc == R.SYM_OK
    C, plan = ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.sym_contract_plan(A, B, 1, R.ints([1]), R.ints([0]), None, prec, ctypes.byref(C),
                                 ctypes.byref(plan)) == R.SYM_OK
    nc = R.numel(lib, C)
    assert nc == 2 * 3 + 3 * 2  # sectors (0, 0) and (1, 1)
    rng = np.random.default_rng(24)
    a = torch.as_tensor(rng.standard_normal(R.numel(lib, A))).to(dtype).cuda()
    b = torch.as_tensor(rng.standard_normal(R.numel(lib, B))).to(dtype).cuda()
    c = torch.full((nc,), float("nan"), dtype=dtype, device="cuda")
    assert lib.sym_contract(plan, _ptr(a), _ptr(b), _ptr(c), _stream()) == R.SYM_OK
    dc = torch.as_tensor(rng.standard_normal(nc)).to(dtype).cuda()
    da = torch.full_like(a, float("nan"))
    db = torch.full_like(b, float("nan"))
    assert lib.sym_contract_backward(plan, _ptr(a), _ptr(b), _ptr(dc), _ptr(da), _ptr(db), _stream()) == R.SYM_OK
    torch.cuda.synchronize()
    assert lib.sym_device_status() == R.SYM_OK
    for t in (c, da, db):
        assert not torch.isnan(t).any()
    assert torch.all(c[6:] == 0)
    oA = ([u1.Leg(*l) for l in la], 0, a.double().cpu().numpy())
    oB = ([u1.Leg(*l) for l in lb], 0, b.double().cpu().numpy())
    _, _, c_ref, _ = oc.contract("u1", oA, oB, [1], [0])
    dA_ref, dB_ref, _ = oc.contract_grad("u1", oA, oB, [1], [0], dc.double().cpu().numpy())
    tol = 1e-12 if dtype == torch.float64 else 2e-5
    assert _rel(c.double().cpu().numpy(), c_ref) <= tol
    assert _rel(da.double().cpu().numpy(), dA_ref) <= tol
    assert _rel(db.double().cpu().numpy(), dB_ref) <= tol
    assert lib.sym_plan_destroy(plan) == R.SYM_OK
    for h in (A, B, C):
        assert lib.sym_tensor_destroy(h) == R.SYM_OK


def test_raw_empty_tensors():
    """A tensor whose total charge no sector reaches has no blocks; its
    contraction plans, runs (nothing to launch) and leaves the buffers alone."""
    lib = R.load()
    rc, A = R.tensor(lib, R.SYM_U1, [([0], [3], 1), ([0], [2], -1)], total=1)  # a - k = 1: impossible
    assert rc == R.SYM_OK and R.numel(lib, A) == 0
    rc, B = R.tensor(lib, R.SYM_U1, [([0], [2], 1), ([0], [4], -1)])
    assert rc == R.SYM_OK and R.numel(lib, B) == 8
    C, plan = ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.sym_contract_plan(A, B, 1, R.ints([1]), R.ints([0]), None, R.SYM_PREC_BF16X3, ctypes.byref(C),
                                 ctypes.byref(plan)) == R.SYM_OK, lib.sym_last_error()
    assert R.numel(lib, C) == 0
    a = torch.full((1,), 7.0, device="cuda")
    b = torch.ones(8, device="cuda")
    c = torch.full((1,), 7.0, device="cuda")
    db = torch.full((8,), 7.0, device="cuda")
    assert lib.sym_contract(plan, _ptr(a), _ptr(b), _ptr(c), _stream()) == R.SYM_OK
    assert lib.sym_contract_backward(plan, _ptr(a), _ptr(b), _ptr(c), _ptr(a), _ptr(db), _stream()) == R.SYM_OK
    torch.cuda.synchronize()
    assert lib.sym_device_status() == R.SYM_OK
    assert float(c[0]) == 7.0 and float(a[0]) == 7.0
    assert torch.all(db == 0)  # B's gradient is a real tensor: nothing reaches it, so it is zero
    assert lib.sym_plan_destroy(plan) == R.SYM_OK
    for h in (A, B, C):
        assert lib.sym_tensor_destroy(h) == R.SYM_OK
