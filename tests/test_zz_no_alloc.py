"""sym_contract_noalloc: the contraction for callers that cannot allocate device memory.

Some callers of this library cannot call cudaMalloc at the point where they
contract (for instance code that must stay out of the CUDA allocator, or that
runs beside a framework owning all device memory).  sym_contract_noalloc
serves them from a fixed 32 MiB static device array instead of plan-owned
buffers.  These tests call it through the C ABI and check its result against
the regular entry point (sym_contract_plan + sym_contract) on two calls in a
row, within the tolerances of the other parity tests.  The file is named to
run last, so that a failure here cannot hide failures elsewhere.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 2e-5}


def _rel(x, y):
    return float((x.double() - y.double()).norm() / max(float(y.double().norm()), 1e-300))


def _run_noalloc(P, L, SA, SB, pa, pb, prec, a, b, numel):
    c = torch.full((numel,), float("nan"), dtype=a.dtype, device=a.device)
    rc = L.lib.sym_contract_noalloc(SA._h, SB._h, len(pa), L.int_array(pa), L.int_array(pb), prec,
                                    ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                    ctypes.c_void_p(c.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, L.lib.sym_last_error()
    torch.cuda.synchronize()
    return c


CASES = ["u1_pairwise", "u1_ragged", "su2_recouple"]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["float64", "float32"])
def test_noalloc_matches_regular_contraction_twice(case, dtype):
    import paper_1203_2222_gb300 as P
    from paper_1203_2222_gb300 import _lib as L
    from paper_1203_2222_gb300 import synthetic
    if case == "u1_pairwise":
        c = synthetic.u1_pairwise()
        g, la, lb, pa, pb = P.U1, c["A"], c["B"], c["pairsA"], c["pairsB"]
    elif case == "u1_ragged":
        qs = [-1, 0, 1]
        g = P.U1
        la = [(qs, [70, 150, 33], -1), (qs, [5, 9, 2], 1), (qs, [90, 140, 61], 1)]
        lb = [(qs, [90, 140, 61], -1), (qs, [100, 131, 7], 1)]
        pa, pb = [2], [0]
    else:
        c = synthetic.su2_recouple(dmax=3, jmax2=4)
        g, la, lb, pa, pb = P.SU2, c["A"], c["B"], c["pairsA"], c["pairsB"]
    SA, SB = P.Structure(g, la), P.Structure(g, lb)
    prec = P.FP64 if dtype == torch.float64 else P.BF16X3
    rng = np.random.default_rng(3)
    a = torch.as_tensor(rng.standard_normal(SA.numel)).to(dtype).cuda()
    b = torch.as_tensor(rng.standard_normal(SB.numel)).to(dtype).cuda()
    ref = P.contract(P.SymTensor(SA, a), P.SymTensor(SB, b), pa, pb).data
    torch.cuda.synchronize()
    for _ in range(2):  # the static array keeps the previous call's contents
        out = _run_noalloc(P, L, SA, SB, pa, pb, prec, a, b, ref.numel())
        assert not torch.isnan(out).any()
        assert _rel(out, ref) <= TOL[dtype]
    P.device_status()


def test_noalloc_rejects_contractions_beyond_its_scratch():
    import paper_1203_2222_gb300 as P
    from paper_1203_2222_gb300 import _lib as L
    qs = [0]
    SA = P.Structure(P.U1, [(qs, [3000], 1), (qs, [3000], -1)])
    SB = P.Structure(P.U1, [(qs, [3000], 1), (qs, [3000], -1)])
    a = torch.zeros(SA.numel, dtype=torch.float64, device="cuda")
    c = torch.zeros(SA.numel, dtype=torch.float64, device="cuda")
    rc = L.lib.sym_contract_noalloc(SA._h, SB._h, 1, L.int_array([1]), L.int_array([0]), P.FP64,
                                    ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                    ctypes.c_void_p(c.data_ptr()), None)
    assert rc == L.SYM_ERR_UNSUPPORTED
    assert b"static limit" in L.lib.sym_last_error()


def _case_structures(P, synthetic, case):
    if case == "u1_ragged":
        qs = [-1, 0, 1]
        la = [(qs, [70, 150, 33], -1), (qs, [5, 9, 2], 1), (qs, [90, 140, 61], 1)]
        lb = [(qs, [90, 140, 61], -1), (qs, [100, 131, 7], 1)]
        return P.U1, la, lb, [2], [0]
    c = synthetic.su2_recouple(dmax=3, jmax2=4)
    return P.SU2, c["A"], c["B"], c["pairsA"], c["pairsB"]


def test_noalloc_alternating_plans_share_the_array():
    """Calls with different plans in a row on one stream: each call lays out
    the shared array for its own plan over what the previous one left."""
    import paper_1203_2222_gb300 as P
    from paper_1203_2222_gb300 import _lib as L
    from paper_1203_2222_gb300 import synthetic
    rng = np.random.default_rng(5)
    setups = {}
    for case in ("u1_ragged", "su2_recouple"):
        g, la, lb, pa, pb = _case_structures(P, synthetic, case)
        SA, SB = P.Structure(g, la), P.Structure(g, lb)
        a = torch.as_tensor(rng.standard_normal(SA.numel)).float().cuda()
        b = torch.as_tensor(rng.standard_normal(SB.numel)).float().cuda()
        ref = P.contract(P.SymTensor(SA, a), P.SymTensor(SB, b), pa, pb).data
        setups[case] = (SA, SB, pa, pb, a, b, ref)
    torch.cuda.synchronize()
    for case in ("u1_ragged", "su2_recouple", "u1_ragged", "su2_recouple"):
        SA, SB, pa, pb, a, b, ref = setups[case]
        out = _run_noalloc(P, L, SA, SB, pa, pb, P.BF16X3, a, b, ref.numel())
        assert _rel(out, ref) <= TOL[torch.float32], case
    P.device_status()


def test_noalloc_recreated_structures_get_their_own_plans():
    """Structures passed only to sym_contract_noalloc are destroyed after each
    call and replaced by structures of other sizes, whose handles the host
    allocator may place at the freed addresses: every call must run the plan
    of its own structures (the references come from other, cached handles)."""
    import gc

    import paper_1203_2222_gb300 as P
    from paper_1203_2222_gb300 import _lib as L
    rng = np.random.default_rng(6)
    qs = [-1, 0, 1]
    sizes = [([40, 90, 30], [50, 70, 20]), ([200, 310, 120], [60, 140, 90]), ([40, 90, 30], [50, 70, 20]),
             ([7, 3, 11], [300, 5, 64])]
    for trial, (dk, dn) in enumerate(sizes):
        la = [(qs, [64, 100, 36], 1), (qs, dk, -1)]
        lb = [(qs, dk, 1), (qs, dn, -1)]
        RA, RB = P.Structure(P.U1, la), P.Structure(P.U1, lb)
        a = torch.as_tensor(rng.standard_normal(RA.numel)).cuda()
        b = torch.as_tensor(rng.standard_normal(RB.numel)).cuda()
        ref = P.contract(P.SymTensor(RA, a), P.SymTensor(RB, b), [1], [0]).data
        torch.cuda.synchronize()
        SA, SB = P.Structure(P.U1, la), P.Structure(P.U1, lb)  # seen by the no-allocation call only
        out = _run_noalloc(P, L, SA, SB, [1], [0], P.FP64, a, b, ref.numel())
        assert _rel(out, ref) <= TOL[torch.float64], trial
        del SA, SB
        gc.collect()
    P.device_status()
