"""GPU parity of rank-5 and rank-6 SU(2) tensors (the library's largest rank):
permute, fuse, split and contraction with non-comb input and output trees,
small degeneracies, against the FP64 oracle's dense embeddings.

Thesis: Ch. 6, PERMUTE and NEWTREE for arbitrary trees (Eq. Gamma, Eq.
permsu2), FUSE/SPLIT, and the contraction of Ch. 5 (Eq. blockmult) after the
recoupling into matrix form.  The blocks of these tensors have 5 or 6 dims;
the gathers fold them into the box kernel's boxes of at most 4 dims.

Tolerances as in test_gpu_parity.py: FP64 1e-12; split-BF16 x3 2e-5 for
contractions; pure data movement in FP32 1e-6 (the recoupling sums run in
FP32 on FP32 copies of the FP64 coefficients).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from test_gpu_parity import DTYPE_IDS, DTYPES, _contract_case, _transform_case, rel  # noqa: E402

SP = [0, 1, 2]
# non-comb trees over 5 and 6 legs (node ids k, k+1, ...; children adjacent ranges, left first)
TREE5 = [(1, 2), (0, 5), (3, 4), (6, 7)]
TREE5B = [(0, 1), (2, 3), (5, 6), (7, 4)]
TREE6 = [(0, 1), (2, 3), (4, 5), (6, 7), (9, 8)]
TREE6B = [(1, 2), (3, 4), (0, 6), (8, 7), (9, 5)]


def _legs5(dirs=(1, 1, -1, 1, -1)):
    degs = [[1, 2, 2], [2, 1, 1], [1, 1, 2], [2, 2, 1], [1, 2, 1]]
    return [(SP, d, s) for d, s in zip(degs, dirs)]


def _legs6(dirs=(1, -1, 1, 1, -1, 1)):
    degs = [[1, 1, 2], [2, 1, 1], [1, 2, 1], [1, 1, 1], [2, 1, 1], [1, 1, 2]]
    return [(SP, d, s) for d, s in zip(degs, dirs)]


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_rank5_permute_between_non_comb_trees(dtype):
    legs = _legs5()
    _transform_case("su2", legs, "permute", ([3, 0, 4, 1, 2], TREE5B), dtype, tree=TREE5)
    _transform_case("su2", legs, "permute", ([0, 2, 1, 3, 4], None), dtype, tree=TREE5B)
    _transform_case("su2", legs, "permute", ([4, 3, 2, 1, 0], TREE5), dtype)


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_rank6_permute_between_non_comb_trees(dtype):
    legs = _legs6()
    _transform_case("su2", legs, "permute", ([0, 2, 1, 3, 5, 4], TREE6), dtype)
    _transform_case("su2", legs, "permute", ([3, 0, 5, 1, 4, 2], TREE6B), dtype, tree=TREE6)
    _transform_case("su2", legs, "permute", ([5, 4, 3, 2, 1, 0], None), dtype, tree=TREE6B)


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_rank5_and_rank6_fuse_and_split(dtype):
    import paper_1203_2222_gb300 as P
    # fusing legs that share no node of the comb needs a recoupling (NEWTREE) first
    legs5 = _legs5(dirs=(1, 1, 1, -1, -1))
    _transform_case("su2", legs5, "fuse", (1,), dtype)
    _transform_case("su2", legs5, "fuse", (3,), dtype)
    legs6 = _legs6(dirs=(1, 1, -1, -1, 1, 1))
    _transform_case("su2", legs6, "fuse", (2,), dtype)
    _transform_case("su2", legs6, "fuse", (4,), dtype)
    # split a rank-5 tensor's fused leg back to rank 6: the round trip is exact
    S, T, F = _transform_case("su2", legs6, "fuse", (0,), dtype)
    back = P.split(F, 0, [legs6[0], legs6[1]])
    torch.cuda.synchronize()
    err = rel(back.data.double().cpu().numpy(), T.data.double().cpu().numpy())
    assert err <= (1e-13 if dtype == torch.float64 else 1e-6), err


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_rank5_contractions_with_non_comb_trees(dtype):
    la = _legs5(dirs=(1, 1, -1, 1, -1))
    # B's first legs are the duals of A's legs 3 and 1 (pairs out of order)
    lb = [(SP, la[3][1], -1), (SP, la[1][1], -1), (SP, [1, 1, 1], 1), ([1], [2], 1)]
    _contract_case("su2", la, lb, [3, 1], [0, 1], dtype, ta=TREE5, tb=[(1, 2), (0, 4), (5, 3)])
    # rank-5 result (3 free legs of A + 2 of B) in a requested non-comb tree
    _contract_case("su2", la, lb, [3, 1], [0, 1], dtype, ta=TREE5B, tree_c=[(1, 2), (0, 5), (3, 4), (6, 7)])


@pytest.mark.parametrize("dtype", DTYPES, ids=DTYPE_IDS)
def test_rank6_contractions(dtype):
    la = _legs6()
    # rank 6 x rank 2 -> rank 6: one pair, A in a balanced tree, C requested in another
    lb = [(SP, la[2][1], -1), (SP, [2, 1, 1], 1)]
    _contract_case("su2", la, lb, [2], [0], dtype, ta=TREE6, tree_c=TREE6B)
    # rank 6 x rank 4 over three pairs -> rank 4 (3 free legs of A + 1 of B)
    lb = [(SP, la[5][1], -1), (SP, la[1][1], 1), (SP, la[3][1], -1), (SP, [1, 2, 1], 1)]
    _contract_case("su2", la, lb, [5, 1, 3], [0, 1, 2], dtype, ta=TREE6B)
