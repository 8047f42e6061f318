"""Pins of the SU(2) x U(1) oracle (oracle/su2u1.py): it reduces to the SU(2)
oracle when every charge is 0 and to the U(1) oracle when every spin is 0,
its tensors are invariant under both groups, and contraction, permutation,
fusion and the gradient keep that invariance and agree with the dense
definitions."""
import numpy as np
import pytest

from oracle import contract as oc
from oracle import su2, su2u1, u1


def _rand(legs, tot, seed):
    n = su2u1.layout(legs, tot)[2]
    return np.random.default_rng(seed).standard_normal(n)


def _legs_a():
    return [su2u1.Leg([(-1, 1), (0, 0), (0, 2), (1, 1)], [2, 1, 2, 1], 1),
            su2u1.Leg([(0, 0), (1, 1)], [2, 1], 1),
            su2u1.Leg([(-1, 1), (0, 0), (1, 1), (1, 3)], [1, 2, 2, 1], -1)]


def test_zero_charges_reduce_to_su2():
    spins = [[0, 1, 2], [1, 3], [0, 2]]
    degs = [[2, 1, 3], [1, 2], [2, 2]]
    dirs = [1, -1, 1]
    for tree in (su2.left_comb(3), [(1, 2), (0, 3)]):
        L = [su2u1.Leg([(0, j) for j in sp], d, r) for sp, d, r in zip(spins, degs, dirs)]
        S = [su2.Leg(sp, d, r) for sp, d, r in zip(spins, degs, dirs)]
        data = _rand(L, (tree, 0), 1)
        assert su2u1.layout(L, (tree, 0))[2] == su2.layout(S, tree)[2]
        assert np.array_equal(su2u1.embed(L, (tree, 0), data), su2.embed(S, tree, data))


def test_zero_spins_reduce_to_u1():
    charges = [[-1, 0, 2], [0, 1], [-1, 0, 1, 3]]
    degs = [[2, 1, 3], [1, 2], [2, 2, 1, 1]]
    dirs = [1, 1, -1]
    for Q in (0, 1, -2):
        L = [su2u1.Leg([(q, 0) for q in c], d, r) for c, d, r in zip(charges, degs, dirs)]
        U = [u1.Leg(c, d, r) for c, d, r in zip(charges, degs, dirs)]
        tot = (su2.left_comb(3), Q)
        data = _rand(L, tot, 2)
        assert su2u1.layout(L, tot)[2] == u1.layout(U, Q)[2]
        assert np.allclose(su2u1.embed(L, tot, data), u1.embed(U, Q, data), atol=1e-15)


@pytest.mark.parametrize("Q", [0, 2])  # odd charges carry half-integer spins here, so Q is even
def test_embeddings_are_invariant_and_a_random_tensor_is_not(Q):
    legs = _legs_a()
    for tree in (su2.left_comb(3), [(1, 2), (0, 3)]):
        tot = (tree, Q)
        d = su2u1.embed(legs, tot, _rand(legs, tot, 3))
        assert np.linalg.norm(d) > 1.0
        assert su2u1.invariance_residual(legs, tot, d) < 1e-12
        b, r = su2u1.extract(legs, tot, d)
        assert r < 1e-12
    noise = np.random.default_rng(4).standard_normal(d.shape)
    assert su2u1.invariance_residual(legs, tot, noise) > 1e-2
    assert su2u1.extract(legs, tot, noise)[1] > 1e-2


def test_contraction_conserves_both_symmetries():
    A = (_legs_a(), (su2.left_comb(3), 2), _rand(_legs_a(), (su2.left_comb(3), 2), 5))
    lb = [_legs_a()[2].dual(), su2u1.Leg([(-1, 1), (0, 0), (0, 2)], [1, 2, 1], 1)]
    tB = (su2.left_comb(2), -2)
    B = (lb, tB, _rand(lb, tB, 6))
    assert A[2].size and B[2].size
    legsC, tC, c, resid = oc.contract("su2u1", A, B, [2], [0])
    assert resid < 1e-12
    assert tC[1] == 0
    dense = np.tensordot(su2u1.embed(*A), su2u1.embed(*B), axes=([2], [0]))
    assert np.allclose(su2u1.embed(legsC, tC, c), dense, atol=1e-12)
    assert su2u1.invariance_residual(legsC, tC, dense) < 1e-12


def test_permute_round_trip_and_fuse_isometry():
    legs = _legs_a()
    tot = (su2.left_comb(3), 0)
    data = _rand(legs, tot, 7)
    T = (legs, tot, data)
    l2, t2, d2, r2 = oc.permute("su2u1", T, [2, 0, 1])
    assert r2 < 1e-12
    l3, t3, d3, r3 = oc.permute("su2u1", (l2, t2, d2), [1, 2, 0])
    assert r3 < 1e-12 and np.allclose(d3, data, atol=1e-12)
    # fusion is an orthogonal change of basis: the dense norm is kept
    lf, tf, df, rf = oc.fuse("su2u1", T, 0)
    assert rf < 1e-12
    assert np.linalg.norm(su2u1.embed(lf, tf, df)) == pytest.approx(np.linalg.norm(su2u1.embed(*T)), rel=1e-12)
    # fused labels: charges add, spins couple; degeneracies count the pairs
    ld, _ = su2u1.fused_leg(su2u1.Leg([(0, 1), (1, 0)], [2, 1], 1), su2u1.Leg([(0, 1), (1, 1)], [1, 3], 1))
    # (0,1)x(0,1) -> (0,0), (0,2), 2 x 1 each; (0,1)x(1,1) -> (1,0), (1,2), 2 x 3 each;
    # (1,0)x(0,1) -> (1,1), 1 x 1; (1,0)x(1,1) -> (2,1), 1 x 3
    assert ld.labels == [(0, 0), (0, 2), (1, 0), (1, 1), (1, 2), (2, 1)]
    assert ld.degens == [2, 2, 6, 1, 6, 3]


def test_gradient_matches_finite_differences():
    la = _legs_a()
    ta = (su2.left_comb(3), 0)
    lb = [la[2].dual(), su2u1.Leg([(0, 0), (1, 1)], [1, 2], -1)]
    tb = (su2.left_comb(2), 0)
    a, b = _rand(la, ta, 8), _rand(lb, tb, 9)
    legsC, tC, c, _ = oc.contract("su2u1", (la, ta, a), (lb, tb, b), [2], [0])
    g = np.random.default_rng(10).standard_normal(c.size)
    dA, dB, _ = oc.contract_grad("su2u1", (la, ta, a), (lb, tb, b), [2], [0], g)
    h = 1e-6
    rng = np.random.default_rng(11)
    for x, dx, which in ((a, dA, 0), (b, dB, 1)):
        v = rng.standard_normal(x.size)
        plus = [a, b]
        minus = [a, b]
        plus[which] = x + h * v
        minus[which] = x - h * v
        fp = oc.contract("su2u1", (la, ta, plus[0]), (lb, tb, plus[1]), [2], [0])[2] @ g
        fm = oc.contract("su2u1", (la, ta, minus[0]), (lb, tb, minus[1]), [2], [0])[2] @ g
        assert (fp - fm) / (2 * h) == pytest.approx(dx @ v, rel=1e-6, abs=1e-8)
