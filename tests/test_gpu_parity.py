"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

Tolerances (relative Frobenius error against the oracle):
  FP64 path            1e-12
  split-BF16 x3 path   2e-5   (inputs are the float32 values the GPU holds,
                               cast to float64 for the oracle)
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import contract as oc  # noqa: E402
from oracle import su2 as osu2  # noqa: E402
from oracle import su2u1 as osu2u1  # noqa: E402
from oracle import u1 as ou1  # noqa: E402
from oracle import z2f as oz2f  # noqa: E402

TOL = {torch.float64: 1e-12, torch.float32: 2e-5}


def _lib():
    import paper_1203_2222_gb300 as P
    return P


def rel(x, y):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    ny = np.linalg.norm(y)
    return float(np.linalg.norm(x - y) / (ny if ny > 0 else 1.0))


def _oleg(group, l):
    return {"u1": ou1.Leg, "su2": osu2.Leg, "z2f": oz2f.Leg, "su2u1": osu2u1.Leg}[group](*l)


def _otree(group, S, legs_spec):
    if group in ("u1", "z2f"):
        return S.total
    tree = S.tree if S.tree is not None else osu2.left_comb(len(legs_spec))
    return (tree, S.total) if group == "su2u1" else tree


def _make(group, legs, seed, dtype, total=0, tree=None):
    P = _lib()
    S = P.Structure({"u1": P.U1, "su2": P.SU2, "z2f": P.Z2F, "su2u1": P.SU2U1}[group], legs, total=total, tree=tree)
    vals = np.random.default_rng(seed).standard_normal(S.numel)
    T = P.SymTensor.from_numpy(S, vals, dtype=dtype)
    host = T.data.double().cpu().numpy()  # exactly what the GPU holds
    return S, T, host


def _contract_case(group, la, lb, pa, pb, dtype, QA=0, QB=0, ta=None, tb=None, tree_c=None, grad=True, seed=0):
    P = _lib()
    SA, A, a = _make(group, la, seed, dtype, QA, ta)
    SB, B, b = _make(group, lb, seed + 1, dtype, QB, tb)
    A.data.requires_grad_(grad)
    B.data.requires_grad_(grad)
    C = P.contract(A, B, pa, pb, tree_c=tree_c)
    torch.cuda.synchronize()
    oA = ([_oleg(group, l) for l in la], _otree(group, SA, la), a)
    oB = ([_oleg(group, l) for l in lb], _otree(group, SB, lb), b)
    tree_of_c = C.structure.tree if group in ("su2", "su2u1") else None
    lc, tc, c_ref, resid = oc.contract(group, oA, oB, pa, pb, tree_c=tree_of_c)
    assert resid < 1e-10
    assert C.structure.numel == len(c_ref)
    c = C.data.detach().double().cpu().numpy()
    err = rel(c, c_ref)
    assert err <= TOL[dtype], f"forward rel err {err:.3e}"
    if grad:
        g = np.random.default_rng(seed + 2).standard_normal(C.structure.numel)
        gt = torch.as_tensor(g).to(dtype).cuda()
        C.data.backward(gt)
        torch.cuda.synchronize()
        g_used = gt.double().cpu().numpy()
        dA_ref, dB_ref, r2 = oc.contract_grad(group, oA, oB, pa, pb, g_used, tree_c=tree_of_c)
        assert r2 < 1e-10
        eA = rel(A.data.grad.double().cpu().numpy(), dA_ref)
        eB = rel(B.data.grad.double().cpu().numpy(), dB_ref)
        assert eA <= TOL[dtype], f"dA rel err {eA:.3e}"
        assert eB <= TOL[dtype], f"dB rel err {eB:.3e}"
    P.device_status()
    return err


DTYPES = [torch.float64, torch.float32]
DTYPE_IDS = ["float64", "float32"]


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_u1_pairwise_workload(dtype):
    from paper_1203_2222_gb300 import synthetic
    c = synthetic.u1_pairwise()
    _contract_case("u1", c["A"], c["B"], c["pairsA"], c["pairsB"], dtype)


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_u1_ragged_multi_tile(dtype):
    # sector matrices spanning several 128-tiles with ragged tails in m, n and k
    qs = [-1, 0, 1]
    la = [(qs, [70, 150, 33], -1), (qs, [5, 9, 2], 1), (qs, [90, 140, 61], 1)]
    lb = [(qs, [90, 140, 61], -1), (qs, [100, 131, 7], 1)]
    _contract_case("u1", la, lb, [2], [0], dtype, QA=0, QB=0)


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_u1_long_reduction_split_k(dtype):
    # thin outputs with reductions of several thousand: split across CTAs
    qs = [-1, 0, 1]
    la = [(qs, [5000, 6000, 4500], -1), (qs, [1, 2, 1], 1)]
    lb = [(qs, [5000, 6000, 4500], 1), (qs, [1, 1, 2], 1)]
    _contract_case("u1", la, lb, [0], [0], dtype)


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_u1_permuted_pairs_and_charges(dtype):
    qs = [-2, -1, 0, 1, 2]
    la = [(qs, [1, 2, 3, 2, 1], 1), (qs, [2, 1, 2, 1, 2], -1), (qs, [3, 1, 1, 2, 1], 1), (qs, [1, 1, 2, 2, 1], -1)]
    lb = [(qs, [1, 1, 2, 2, 1], 1), (qs, [2, 3, 1, 1, 1], 1), (qs, [3, 1, 1, 2, 1], -1)]
    # contract A3<->B0 and A2<->B2 (pairs out of order), nonzero total charges
    _contract_case("u1", la, lb, [3, 2], [0, 2], dtype, QA=1, QB=-2)


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_u1_edge_cases(dtype):
    qs = [0]
    # single sector, 1x1 blocks
    _contract_case("u1", [(qs, [1], 1), (qs, [1], -1)], [(qs, [1], 1), (qs, [1], 1)], [1], [0], dtype)
    # full contraction to a scalar
    la = [([-1, 0, 1], [2, 3, 1], 1), ([-1, 0, 1], [1, 2, 2], -1)]
    lb = [([-1, 0, 1], [2, 3, 1], -1), ([-1, 0, 1], [1, 2, 2], 1)]
    _contract_case("u1", la, lb, [0, 1], [0, 1], dtype)
    # outer product (no pairs)
    _contract_case("u1", la, [([-1, 0, 1], [2, 1, 3], 1)], [], [], dtype, QB=1)


# Sectors whose matrix of B is at most 4 x 4 are contracted directly on the
# blocks (no matrix form); the cases below put every sector there.
MPO = ([-1, 0, 1], [1, 3, 1])
PHYS = ([0, 1], [1, 1])


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_u1_mpo_step_direct(dtype):
    # T[a, w, s, b] . W[w, s, s', w'] over (w, s): contracted legs in the middle
    # of T, free-leg strides that vary with the MPO charge on both sides
    qs = [-2, -1, 0, 1, 2]
    bond_in, bond_out = (qs, [7, 19, 33, 21, 5], -1), (qs, [6, 17, 40, 23, 9], 1)
    la = [bond_in, (*MPO, -1), (*PHYS, -1), bond_out]
    lb = [(*MPO, 1), (*PHYS, -1), (*PHYS, 1), (*MPO, -1)]
    _contract_case("u1", la, lb, [1, 2], [0, 2], dtype)


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_u1_mpo_split_contracted_legs_direct(dtype):
    # T[a, s2, b, s1, w] . W[w, s, s', w'] over T(1, 4) <-> W(2, 0): the
    # contracted legs sit on both sides of free legs
    qs = [-2, -1, 0, 1, 2]
    la = [(qs, [4, 11, 20, 9, 3], -1), (*PHYS, -1), (qs, [5, 13, 17, 12, 6], 1), (*PHYS, 1), (*MPO, 1)]
    lb = [(*MPO, -1), (*PHYS, 1), (*PHYS, 1), (*MPO, 1)]
    _contract_case("u1", la, lb, [1, 4], [2, 0], dtype, QA=1)


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_u1_tiny_b_with_missing_blocks_direct(dtype):
    # B's sector matrices have structurally absent blocks (total charge 1 and a
    # leg without every charge), m large with a ragged box, k = n = 1 sectors
    la = [([-1, 0, 1, 2], [37, 64, 129, 3], 1), ([-1, 0, 1], [1, 2, 1], -1)]
    lb = [([-1, 0, 1], [1, 2, 1], 1), ([0, 2], [1, 2], 1)]
    _contract_case("u1", la, lb, [1], [0], dtype, QB=1)


# Fermion parity (the thesis's outlook): permutations carry the swap signs;
# a contraction is A's contracted legs permuted last, B's first, then the
# blockwise product.
PAR = [0, 1]


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_z2f_contraction_with_swap_signs(dtype):
    # contracted legs out of order on both sides: odd legs are exchanged
    la = [(PAR, [23, 17], 1), (PAR, [9, 14], -1), (PAR, [30, 11], 1), (PAR, [12, 19], 1)]
    lb = [(PAR, [12, 19], -1), (PAR, [40, 25], 1), (PAR, [9, 14], 1)]
    _contract_case("z2f", la, lb, [3, 1], [0, 2], dtype, QA=1, QB=0)


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_z2f_multi_tile_and_edge_cases(dtype):
    # sector matrices spanning several 128-tiles (tensor-core and CUDA-core kernels)
    la = [(PAR, [150, 70], 1), (PAR, [5, 3], -1), (PAR, [90, 140], 1)]
    lb = [(PAR, [90, 140], -1), (PAR, [100, 37], 1)]
    _contract_case("z2f", la, lb, [2], [0], dtype, QA=0, QB=1)
    # three contracted pairs in reversed order, total parity odd on both sides
    la = [(PAR, [3, 2], 1), (PAR, [2, 3], 1), (PAR, [4, 1], -1), (PAR, [1, 2], 1)]
    lb = [(PAR, [1, 2], -1), (PAR, [4, 1], 1), (PAR, [2, 3], -1), (PAR, [2, 2], 1)]
    _contract_case("z2f", la, lb, [3, 2, 1], [0, 1, 2], dtype, QA=1, QB=1)
    # full contraction to a scalar and an outer product
    la = [(PAR, [2, 3], 1), (PAR, [3, 1], -1)]
    lb = [(PAR, [2, 3], -1), (PAR, [3, 1], 1)]
    _contract_case("z2f", la, lb, [0, 1], [0, 1], dtype, QA=1, QB=1)
    _contract_case("z2f", la, [(PAR, [2, 2], 1)], [], [], dtype, QA=1, QB=1)


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_z2f_permute_and_fuse(dtype):
    legs = [(PAR, [2, 3], 1), (PAR, [3, 1], -1), (PAR, [1, 2], 1), (PAR, [2, 2], -1)]
    _transform_case("z2f", legs, "permute", ([2, 0, 3, 1], None), dtype)
    _transform_case("z2f", legs, "permute", ([3, 2, 1, 0], None), dtype)
    legs = [(PAR, [2, 3], 1), (PAR, [3, 1], 1), (PAR, [1, 2], -1)]
    _transform_case("z2f", legs, "fuse", (0,), dtype)


SU2_TREES = [None, [(1, 2), (0, 4), (5, 3)], [(0, 1), (2, 3), (4, 5)]]


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
@pytest.mark.parametrize("ti", range(len(SU2_TREES)))
def test_su2_recoupling_contraction(dtype, ti):
    # the recoupling workload at reduced size: 2j <= 4, degeneracies 1..3
    from paper_1203_2222_gb300 import synthetic
    c = synthetic.su2_recouple(dmax=3, jmax2=4)
    _contract_case("su2", c["A"], c["B"], c["pairsA"], c["pairsB"], dtype, ta=SU2_TREES[ti])


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_su2_mixed_directions_and_output_tree(dtype):
    sp = [0, 1, 2, 3]
    la = [(sp, [2, 1, 2, 1], -1), (sp, [1, 2, 1, 1], 1), (sp, [2, 2, 1, 1], -1), (sp, [1, 1, 2, 1], 1)]
    lb = [(sp, [1, 2, 1, 1], -1), (sp, [2, 2, 1, 1], 1), (sp, [1, 1, 1, 2], 1)]
    _contract_case("su2", la, lb, [1, 2], [0, 1], dtype, ta=[(1, 2), (0, 4), (5, 3)])
    # requested output tree different from the natural one
    _contract_case("su2", la, lb, [1, 2], [0, 1], dtype, tree_c=[(1, 2), (0, 3)])


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_su2_matrix_and_edge_cases(dtype):
    sp = [0, 1, 2, 3]
    m = [(sp, [3, 2, 2, 1], -1), (sp, [3, 2, 2, 1], 1)]
    n = [(sp, [3, 2, 2, 1], -1), (sp, [2, 1, 3, 2], 1)]
    _contract_case("su2", m, n, [1], [0], dtype)
    # full contraction to a scalar and a rank-1 result
    a = [(sp, [2, 1, 1, 1], 1), (sp, [1, 2, 1, 1], 1)]
    b = [(sp, [2, 1, 1, 1], -1), (sp, [1, 2, 1, 1], -1)]
    _contract_case("su2", a, b, [0, 1], [0, 1], dtype)
    c3 = [(sp, [2, 1, 1, 1], 1), (sp, [1, 2, 1, 1], 1), ([0, 2], [2, 1], 1)]
    _contract_case("su2", c3, b, [0, 1], [0, 1], dtype)


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_su2_large_sectors_multi_tile(dtype):
    # sector matrices of a few hundred rows/cols: several tiles with ragged tails
    sp = [0, 1, 2]
    la = [(sp, [40, 35, 9], 1), (sp, [13, 7, 5], 1), (sp, [31, 22, 17], 1)]
    lb = [(sp, [31, 22, 17], -1), (sp, [29, 15, 11], 1)]
    _contract_case("su2", la, lb, [2], [0], dtype, grad=True)


# ----------------------------------------------------------- transforms ------

def _transform_case(group, legs, op, args, dtype, tree=None, seed=5, total=0):
    P = _lib()
    S, T, t = _make(group, legs, seed, dtype, total, tree)
    oT = ([_oleg(group, l) for l in legs], _otree(group, S, legs), t)
    if op == "permute":
        out = P.permute(T, args[0], args[1])
        lo, to, ref, resid = oc.permute(group, oT, args[0], out.structure.tree if group in ("su2", "su2u1") else None)
    elif op == "fuse":
        out = P.fuse(T, args[0])
        lo, to, ref, resid = oc.fuse(group, oT, args[0], out.structure.tree if group in ("su2", "su2u1") else None)
        assert [tuple(l.labels) for l in lo] == [tuple(l[0]) for l in out.structure.legs]
        assert [tuple(l.degens) for l in lo] == [tuple(l[1]) for l in out.structure.legs]
    torch.cuda.synchronize()
    assert resid < 1e-10
    err = rel(out.data.double().cpu().numpy(), ref)
    assert err <= TOL[dtype] if dtype == torch.float64 else err <= 1e-6, err
    return S, T, out


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_permute(dtype):
    qs = [-1, 0, 1]
    u = [(qs, [2, 3, 1], 1), (qs, [1, 2, 2], -1), (qs, [3, 1, 2], 1), (qs, [2, 2, 1], -1)]
    _transform_case("u1", u, "permute", ([2, 0, 3, 1], None), dtype)
    sp = [0, 1, 2, 3]
    s = [(sp, [2, 1, 1, 1], 1), (sp, [1, 2, 1, 1], -1), (sp, [1, 1, 2, 1], 1), (sp, [1, 1, 1, 2], 1)]
    _transform_case("su2", s, "permute", ([2, 0, 3, 1], None), dtype)
    _transform_case("su2", s, "permute", ([0, 2, 1, 3], [(0, 1), (2, 3), (4, 5)]), dtype,
                    tree=[(1, 2), (0, 4), (5, 3)])


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_su2_transforms_many_positions(dtype):
    # standalone SU(2) permute, fuse and split whose blocks span several
    # fused recoupling items (blocks up to 12^4 positions; items of 512 to
    # 2048 positions with ragged last ones) and whose leg spins give 1 to 5
    # source labels per set of legs; fuses of inner legs (1, 2) and (2, 3)
    # take the destination's fused-leg dimension as its row stride
    P = _lib()
    sp = [0, 1, 2]
    for legs in ([(sp, [12, 9, 7], 1), (sp, [9, 7, 12], -1), (sp, [7, 12, 9], -1), (sp, [12, 7, 9], -1)],
                 [([3, 4], [6, 5], 1), ([2, 3, 4], [3, 6, 4], 1), ([3, 4], [5, 6], 1), ([2, 4], [6, 5], 1)]):
        _transform_case("su2", legs, "permute", ([0, 2, 1, 3], [(0, 1), (2, 3), (4, 5)]), dtype)
        _transform_case("su2", legs, "permute", ([3, 1, 0, 2], None), dtype)
        for f in (1, 2):
            S, T, F = _transform_case("su2", legs, "fuse", (f,), dtype)
            back = P.split(F, f, [legs[f], legs[f + 1]])
            torch.cuda.synchronize()
            err = rel(back.data.double().cpu().numpy(), T.data.double().cpu().numpy())
            assert err <= (1e-13 if dtype == torch.float64 else 1e-6), (f, err)


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_fuse_then_split_roundtrip(dtype):
    P = _lib()
    for group, legs in [
        ("u1", [([-1, 0, 1], [2, 3, 1], 1), ([-1, 0, 1], [1, 2, 2], 1), ([-2, -1, 0, 1, 2], [1, 1, 2, 1, 1], -1)]),
        ("su2", [([0, 1, 2], [2, 1, 1], 1), ([0, 1, 2], [1, 2, 1], 1), ([0, 1, 2, 3, 4], [1, 1, 2, 1, 1], 1)]),
        ("su2", [([0, 1, 2], [2, 1, 1], -1), ([0, 1, 2], [1, 2, 1], -1), ([0, 1, 2, 3, 4], [1, 1, 2, 1, 1], 1)]),
    ]:
        S, T, F = _transform_case(group, legs, "fuse", (0,), dtype)
        back = P.split(F, 0, [legs[0], legs[1]])
        torch.cuda.synchronize()
        err = rel(back.data.double().cpu().numpy(), T.data.double().cpu().numpy())
        assert err <= (1e-13 if dtype == torch.float64 else 1e-6), (group, err)


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_backward_after_another_forward_on_the_same_plan(dtype):
    # The backward reads the tensor-core operand forms its forward gathered
    # unless the plan has run a forward on other inputs since; then it
    # gathers them again.  Interleave two forwards and check both gradients.
    P = _lib()
    qs = [-1, 0, 1]
    la = [(qs, [70, 150, 33], -1), (qs, [5, 9, 2], 1), (qs, [90, 140, 61], 1)]
    lb = [(qs, [90, 140, 61], -1), (qs, [100, 131, 7], 1)]
    runs = []
    for seed in (0, 10):
        SA, A, a = _make("u1", la, seed, dtype)
        SB, B, b = _make("u1", lb, seed + 1, dtype)
        A.data.requires_grad_(True)
        B.data.requires_grad_(True)
        runs.append((A, B, a, b, P.contract(A, B, [2], [0])))
    for i, (A, B, a, b, C) in enumerate(runs):
        g = np.random.default_rng(20 + i).standard_normal(C.structure.numel)
        gt = torch.as_tensor(g).to(dtype).cuda()
        C.data.backward(gt)
        torch.cuda.synchronize()
        oA = ([_oleg("u1", l) for l in la], 0, a)
        oB = ([_oleg("u1", l) for l in lb], 0, b)
        dA_ref, dB_ref, _ = oc.contract_grad("u1", oA, oB, [2], [0], gt.double().cpu().numpy())
        assert rel(A.data.grad.double().cpu().numpy(), dA_ref) <= TOL[dtype]
        assert rel(B.data.grad.double().cpu().numpy(), dB_ref) <= TOL[dtype]
    P.device_status()


# ------------------------------------------------- SU(2) x U(1) (composite) --

# labels (q, 2j); odd charges carry half-integer spins, like a spinful
# particle number; directions mixed; nonzero total charges
CQ = [(-1, 1), (0, 0), (0, 2), (1, 1), (2, 0)]


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_su2u1_contraction(dtype):
    la = [(CQ, [2, 1, 2, 1, 1], 1), (CQ, [1, 2, 1, 2, 1], -1), (CQ, [2, 2, 1, 1, 2], 1), (CQ, [1, 1, 2, 1, 1], -1)]
    lb = [(CQ, [2, 2, 1, 1, 2], -1), (CQ, [1, 1, 2, 1, 1], 1), (CQ, [2, 1, 1, 2, 1], 1)]
    _contract_case("su2u1", la, lb, [2, 3], [0, 1], dtype, QA=2, QB=-2)
    _contract_case("su2u1", la, lb, [2, 3], [0, 1], dtype, QA=0, QB=0, ta=[(1, 2), (0, 4), (5, 3)])
    _contract_case("su2u1", la, lb, [2, 3], [0, 1], dtype, QA=2, QB=0, tree_c=[(1, 2), (0, 3)])


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_su2u1_large_sectors_multi_tile(dtype):
    # sector matrices of a few hundred rows and columns: tensor-core tiles with ragged tails
    la = [(CQ, [30, 41, 12, 25, 9], 1), (CQ, [7, 5, 3, 6, 2], 1), (CQ, [60, 52, 49, 55, 48], 1)]
    lb = [(CQ, [60, 52, 49, 55, 48], -1), (CQ, [70, 64, 30, 66, 20], 1)]
    _contract_case("su2u1", la, lb, [2], [0], dtype, QA=2, QB=-2)


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_su2u1_permute_fuse_split(dtype):
    P = _lib()
    s = [(CQ, [2, 1, 1, 1, 1], 1), (CQ, [1, 2, 1, 1, 2], -1), (CQ, [1, 1, 2, 1, 1], 1), (CQ, [1, 1, 1, 2, 1], 1)]
    _transform_case("su2u1", s, "permute", ([2, 0, 3, 1], None), dtype, total=2)
    _transform_case("su2u1", s, "permute", ([0, 2, 1, 3], [(0, 1), (2, 3), (4, 5)]), dtype, tree=[(1, 2), (0, 4), (5, 3)])
    for legs in ([(CQ, [2, 1, 1, 1, 1], 1), (CQ, [1, 2, 1, 1, 2], 1), (CQ, [1, 1, 2, 1, 1], -1)],
                 [(CQ, [2, 1, 1, 1, 1], -1), (CQ, [1, 2, 1, 1, 2], -1), (CQ, [1, 1, 2, 1, 1], 1)]):
        for total in (0, 2):
            S, T, F = _transform_case("su2u1", legs, "fuse", (0,), dtype, total=total)
            back = P.split(F, 0, [legs[0], legs[1]])
            torch.cuda.synchronize()
            err = rel(back.data.double().cpu().numpy(), T.data.double().cpu().numpy())
            assert err <= (1e-13 if dtype == torch.float64 else 1e-6), err


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_su2_high_spins(dtype):
    # legs of spin 7 to 8 (2j = 14..16, the largest the workloads use, node
    # spins up to 2j = 32 inside A's comb tree), recoupled into the matrix tree
    hi = [14, 15, 16]
    la = [(hi, [1, 2, 1], 1), (hi, [2, 1, 1], 1), (hi, [1, 1, 2], 1), ([0, 1, 2], [1, 1, 1], 1)]
    lb = [(hi, [2, 1, 1], -1), ([0, 1, 2], [1, 1, 1], -1), ([13, 14, 15, 16], [1, 1, 2, 1], 1)]
    _contract_case("su2", la, lb, [1, 3], [0, 1], dtype)


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_fuse_several_legs(dtype):
    # sym_fuse_n_plan: legs first..first+n-1 fused pairwise from the left in
    # one plan (its steps chained through plan-owned scratch), against the
    # oracle's pairwise fuse applied n-1 times
    P = _lib()
    cases = [
        ("u1", [([-1, 0, 1], [2, 1, 2], 1), ([0, 1], [1, 2], 1), ([-1, 0], [2, 1], 1), ([-2, 0, 2], [1, 2, 1], -1)],
         0, 3),
        ("u1", [([0, 1], [2, 1], -1), ([-1, 0, 1], [1, 2, 1], 1), ([0, 1], [1, 2], 1), ([0, 1], [2, 1], 1),
                ([-1, 0, 1, 2, 3], [1, 1, 2, 1, 1], -1)], 1, 3),
        ("su2", [([0, 1, 2], [2, 1, 1], 1), ([0, 1], [1, 2], 1), ([1, 2], [2, 1], 1), ([0, 1, 2, 3], [1, 2, 1, 1], 1)],
         0, 3),
        ("su2", [([0, 1, 2], [1, 1, 1], -1), ([0, 1, 2], [2, 1, 1], -1), ([0, 1], [1, 1], -1), ([1, 2], [1, 1], -1),
                 ([0, 1, 2, 3, 4], [1, 1, 2, 1, 1], 1)], 0, 4),
    ]
    for group, legs, first, n in cases:
        S, T, t = _make(group, legs, 31, dtype)
        out = P.fuse(T, first, nlegs=n)
        torch.cuda.synchronize()
        oT = ([_oleg(group, l) for l in legs], _otree(group, S, legs), t)
        for _ in range(n - 1):
            lo, to, data, resid = oc.fuse(group, oT, first)
            assert resid < 1e-10
            oT = (lo, to, data)
        assert [tuple(l.labels) for l in oT[0]] == [tuple(l[0]) for l in out.structure.legs]
        assert [tuple(l.degens) for l in oT[0]] == [tuple(l[1]) for l in out.structure.legs]
        err = rel(out.data.double().cpu().numpy(), oT[2])
        assert err <= (TOL[dtype] if dtype == torch.float64 else 1e-6), (group, first, n, err)
    P.device_status()
