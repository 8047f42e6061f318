"""Pins of the blockwise SVD oracle (oracle/svd.py) against the plain dense SVD
and the mathematics of the singular value decomposition, independent of the
GPU path."""
import numpy as np
import pytest

from oracle import svd, u1, z2f


def _t(group, legs, total, seed):
    m = u1 if group == "u1" else z2f
    n = m.layout(legs, total)[2]
    return (legs, total, np.random.default_rng(seed).standard_normal(n))


def _u1_rank4():
    return [u1.Leg([-1, 0, 1], [2, 3, 1], 1), u1.Leg([0, 1], [2, 2], 1),
            u1.Leg([-1, 0, 2], [1, 2, 2], -1), u1.Leg([0, 1], [1, 3], -1)]


def _z2f_rank3():
    return [z2f.Leg([0, 1], [3, 2], 1), z2f.Leg([0, 1], [1, 2], -1), z2f.Leg([0, 1], [2, 3], 1)]


CASES = [("u1", _u1_rank4, 0, 2), ("u1", _u1_rank4, 1, 1), ("u1", _u1_rank4, -1, 3),
         ("z2f", _z2f_rank3, 0, 1), ("z2f", _z2f_rank3, 1, 2)]


def _dense(group, T):
    legs, total, data = T
    return svd._mod(group).embed(legs, total, data)


def _bond_matrix(group, U, V):
    """Dense U as (rows, bond) and dense V as (bond, cols)."""
    du, dv = _dense(group, U), _dense(group, V)
    return du.reshape(-1, du.shape[-1]), dv.reshape(dv.shape[0], -1)


def _all_values(fac):
    return np.sort(np.concatenate([fac[x][1] for x in fac]))[::-1]


@pytest.mark.parametrize("group,legs,total,nrow", CASES)
def test_singular_values_are_those_of_the_dense_matrix(group, legs, total, nrow):
    # the block-diagonal form is a permutation of the dense matrix's rows and
    # columns (zero blocks aside), so the union of the blocks' singular values
    # is the dense matrix's nonzero spectrum
    T = _t(group, legs(), total, 3)
    fac, _ = svd.svd(group, T, nrow)
    ours = _all_values(fac)
    dense = np.linalg.svd(svd.matrix(group, T, nrow), compute_uv=False)
    assert np.allclose(ours, dense[:len(ours)], rtol=1e-12, atol=1e-12)
    assert np.all(dense[len(ours):] < 1e-12)


@pytest.mark.parametrize("group,legs,total,nrow", CASES)
def test_factors_rebuild_the_tensor_and_are_orthonormal(group, legs, total, nrow):
    T = _t(group, legs(), total, 5)
    fac, _ = svd.svd(group, T, nrow)
    keep = svd.truncation({x: f[1] for x, f in fac.items()})
    U, kept, V = svd.factors(group, T, nrow, keep)
    Um, Vm = _bond_matrix(group, U, V)
    S = np.concatenate([kept[x] for x in sorted(kept)])  # bond order: labels ascending
    assert np.allclose(Um @ np.diag(S) @ Vm, svd.matrix(group, T, nrow), atol=1e-12)
    assert np.allclose(Um.T @ Um, np.eye(len(S)), atol=1e-12)
    assert np.allclose(Vm @ Vm.T, np.eye(len(S)), atol=1e-12)
    # U and V are symmetric tensors in their own right: nothing outside their blocks
    m = u1 if group == "u1" else z2f
    for legsX, tot, d in (U, V):
        assert m.extract(legsX, tot, m.embed(legsX, tot, d))[1] == 0.0
    # absorbing S into either factor gives the same product
    U1, _, V1 = svd.factors(group, T, nrow, keep, absorb=1)
    U2, _, V2 = svd.factors(group, T, nrow, keep, absorb=2)
    for A, B in ((U1, V1), (U2, V2)):
        Am, Bm = _bond_matrix(group, A, B)
        assert np.allclose(Am @ Bm, svd.matrix(group, T, nrow), atol=1e-12)


@pytest.mark.parametrize("group,legs,total,nrow", CASES)
def test_truncation_is_the_best_low_rank_approximation(group, legs, total, nrow):
    # Eckart-Young: keeping the chi largest singular values of the whole
    # matrix is optimal in the Frobenius norm, the error being the norm of
    # the discarded values -- the dense matrix's own optimum
    T = _t(group, legs(), total, 7)
    M = svd.matrix(group, T, nrow)
    dense = np.linalg.svd(M, compute_uv=False)
    fac, _ = svd.svd(group, T, nrow)
    for chi in (1, 3, len(_all_values(fac)) // 2):
        keep = svd.truncation({x: f[1] for x, f in fac.items()}, chi=chi)
        assert sum(keep.values()) == chi
        U, kept, V = svd.factors(group, T, nrow, keep, absorb=1)
        Um, Vm = _bond_matrix(group, U, V)
        err = np.linalg.norm(M - Um @ Vm)
        assert err == pytest.approx(np.sqrt(np.sum(dense[chi:] ** 2)), rel=1e-10, abs=1e-12)


def test_cutoff_keeps_values_above_the_threshold():
    T = _t("u1", _u1_rank4(), 0, 9)
    fac, _ = svd.svd("u1", T, 2)
    vals = _all_values(fac)
    cut = 0.5 * (vals[3] + vals[4]) / vals[0]
    keep = svd.truncation({x: f[1] for x, f in fac.items()}, cutoff=cut)
    assert sum(keep.values()) == 4
    keep = svd.truncation({x: f[1] for x, f in fac.items()}, chi=2, cutoff=cut)
    assert sum(keep.values()) == 2


def test_one_charge_is_the_plain_svd():
    # with one label per leg the matrix has a single block: the dense matrix
    legs = [u1.Leg([0], [4], 1), u1.Leg([0], [3], 1), u1.Leg([0], [5], -1)]
    T = _t("u1", legs, 0, 11)
    fac, bd = svd.svd("u1", T, 2)
    assert list(fac) == [0]
    M = T[2].reshape(12, 5)
    assert np.array_equal(bd[0][0], M)
    assert np.allclose(fac[0][1], np.linalg.svd(M, compute_uv=False), rtol=1e-14)


def test_diagonal_blocks_give_their_absolute_values():
    # a rank-2 U(1) tensor with diagonal blocks: the singular values are the
    # absolute diagonal entries, sorted within each block
    legs = [u1.Leg([-1, 0, 1], [2, 3, 1], 1), u1.Leg([-1, 0, 1], [2, 3, 1], -1)]
    diag = {-1: [0.5, -2.0], 0: [3.0, -1.0, 0.25], 1: [-7.0]}
    data = np.concatenate([np.diag(diag[q]).reshape(-1) for q in (-1, 0, 1)])
    fac, _ = svd.svd("u1", (legs, 0, data), 1)
    for q in (-1, 0, 1):
        assert np.allclose(fac[q][1], sorted(np.abs(diag[q]), reverse=True), rtol=0, atol=1e-15)
    keep = svd.truncation({x: f[1] for x, f in fac.items()}, chi=2)
    assert keep == {-1: 0, 0: 1, 1: 1}  # 7 and 3


def test_block_labels_follow_the_row_legs():
    # U(1): block x collects exactly the tensor blocks whose row charges sum
    # (with directions) to x; total charge 1 moves the column partner by 1
    legs = _u1_rank4()
    T = _t("u1", legs, 1, 13)
    bd = svd.block_diagonal("u1", T, 2)
    secs = u1.layout(legs, 1)[0]
    for s in secs:
        x = legs[0].labels[s[0]] + legs[1].labels[s[1]]
        assert x in bd
        rt = tuple(s[:2])
        assert any(t == rt for t, _, _ in bd[x][1])
        cq = -legs[2].labels[s[2]] - legs[3].labels[s[3]]
        assert x + cq == 1


# ---- SU(2): rank-2 tensors, the block-diagonal form of Eq. svd0

SU2_DIRS = [(1, -1), (1, 1), (-1, -1), (-1, 1)]


def _su2_tensor(dirs, seed):
    from oracle import su2
    legs = [su2.Leg([0, 1, 2, 3], [3, 2, 4, 2], dirs[0]), su2.Leg([0, 1, 2, 3], [2, 3, 3, 1], dirs[1])]
    tree = su2.left_comb(2)
    n = su2.layout(legs, tree)[2]
    return (legs, tree, np.random.default_rng(seed).standard_normal(n))


@pytest.mark.parametrize("dirs", SU2_DIRS)
def test_su2_values_are_the_dense_spectrum_with_multiplicity(dirs):
    # the dense matrix is the direct sum over spins of the stored block over
    # sqrt(2j+1) times an orthogonal (2j+1)-dimensional map
    T = _su2_tensor(dirs, 31)
    fac, _ = svd.svd("su2", T, 1)
    keep = svd.truncation({x: f[1] for x, f in fac.items()}, group="su2")
    ours = np.sort(svd.dense_values("su2", {x: fac[x][1][:keep[x]] for x in fac}))[::-1]
    dense = np.linalg.svd(svd.matrix("su2", T, 1), compute_uv=False)
    assert np.allclose(ours, dense[:len(ours)], rtol=1e-12, atol=1e-12)
    assert np.all(dense[len(ours):] < 1e-12)


@pytest.mark.parametrize("dirs", SU2_DIRS)
def test_su2_factors_rebuild_the_tensor_and_are_isometries(dirs):
    T = _su2_tensor(dirs, 33)
    fac, _ = svd.svd("su2", T, 1)
    keep = svd.truncation({x: f[1] for x, f in fac.items()}, group="su2")
    U, kept, V = svd.factors("su2", T, 1, keep)
    Um, Vm = _bond_matrix("su2", U, V)
    S = svd.dense_values("su2", kept)
    assert np.allclose(Um @ np.diag(S) @ Vm, svd.matrix("su2", T, 1), atol=1e-12)
    assert np.allclose(Um.T @ Um, np.eye(len(S)), atol=1e-12)
    assert np.allclose(Vm @ Vm.T, np.eye(len(S)), atol=1e-12)
    from oracle import su2
    for legsX, tree, d in (U, V):
        assert su2.extract(legsX, tree, su2.embed(legsX, tree, d))[1] < 1e-12
    for absorb in (1, 2):
        A, _, B = svd.factors("su2", T, 1, keep, absorb=absorb)
        Am, Bm = _bond_matrix("su2", A, B)
        assert np.allclose(Am @ Bm, svd.matrix("su2", T, 1), atol=1e-12)


def test_su2_truncation_counts_multiplets():
    # chi counts dense singular values: a spin-j value costs 2j+1 of it, and
    # when a whole multiplet fits the error is the dense optimum
    T = _su2_tensor((1, -1), 35)
    M = svd.matrix("su2", T, 1)
    dense = np.linalg.svd(M, compute_uv=False)
    fac, _ = svd.svd("su2", T, 1)
    for chi in (1, 4, 9, 20):
        keep = svd.truncation({x: f[1] for x, f in fac.items()}, chi=chi, group="su2")
        n = sum(k * (x + 1) for x, k in keep.items())
        assert n <= chi
        U, kept, V = svd.factors("su2", T, 1, keep, absorb=1)
        Um, Vm = _bond_matrix("su2", U, V)
        err = np.linalg.norm(M - Um @ Vm)
        assert err == pytest.approx(np.sqrt(np.sum(dense[n:] ** 2)), rel=1e-10, abs=1e-12)
