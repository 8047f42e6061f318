"""Pins of the fermion-parity oracle (oracle/z2f.py) against what the thesis
prints and what the Z2 grading fixes, independent of the GPU path."""
import itertools

import numpy as np
import pytest

from oracle import u1, z2f
from tests.conftest import read_golden


def _rand(legs, P, seed):
    n = z2f.layout(legs, P)[2]
    return np.random.default_rng(seed).standard_normal(n)


def test_swap_tensor_is_the_printed_table():
    # a rank-2 tensor with one state of each parity per leg: exchanging its
    # legs multiplies the element (p, p') by the swap tensor R(p, p')
    for row in read_golden("z2f_swap.txt"):
        p, q, r, value = row.split()
        p, q, r, value = int(p), int(q), int(r), float(value)
        assert r == (p + q) % 2
        assert z2f.swap(p, q) == value
        legs = [z2f.Leg([0, 1], [1, 1], 1), z2f.Leg([0, 1], [1, 1], 1)]
        T = np.zeros((2, 2))
        T[p, q] = 1.0
        data, resid = z2f.extract(legs, r, T)
        assert resid == 0.0
        _, _, out, resid = z2f.permute((legs, r, data), [1, 0])
        assert resid == 0.0
        assert np.allclose(z2f.embed(legs, r, out), value * T.T)


def test_permutations_compose():
    # the signs form a representation: permuting by p1 then p2 equals
    # permuting once by the composite; and p followed by its inverse is the identity
    legs = [z2f.Leg([0, 1], [2, 1], 1), z2f.Leg([0, 1], [1, 2], -1), z2f.Leg([0, 1], [2, 2], 1),
            z2f.Leg([0, 1], [1, 1], -1)]
    data = _rand(legs, 1, 0)
    rng = np.random.default_rng(1)
    for _ in range(12):
        p1 = list(rng.permutation(4))
        p2 = list(rng.permutation(4))
        l1, P1, d1, _ = z2f.permute((legs, 1, data), p1)
        _, _, d12, _ = z2f.permute((l1, P1, d1), p2)
        comp = [p1[i] for i in p2]
        _, _, dc, _ = z2f.permute((legs, 1, data), comp)
        assert np.allclose(d12, dc)
        inv = list(np.argsort(p1))
        _, _, back, _ = z2f.permute((l1, P1, d1), inv)
        assert np.allclose(back, data)


def test_odd_vectors_anticommute():
    # u and v supported on odd states only: exchanging the legs of u (x) v gives -(v (x) u)
    leg = z2f.Leg([0, 1], [2, 3], 1)
    rng = np.random.default_rng(2)
    u = np.concatenate([np.zeros(2), rng.standard_normal(3)])
    v = np.concatenate([np.zeros(2), rng.standard_normal(3)])
    T = np.outer(u, v)
    data, resid = z2f.extract([leg, leg], 0, T)
    assert resid == 0.0
    _, _, out, _ = z2f.permute(([leg, leg], 0, data), [1, 0])
    assert np.allclose(z2f.embed([leg, leg], 0, out), -np.outer(v, u))


def test_even_sector_only_is_bosonic():
    # legs with parity 0 only: permutation is a plain transpose and a
    # contraction the plain dense one (the U(1) oracle with one charge)
    la = [z2f.Leg([0], [3], 1), z2f.Leg([0], [4], -1), z2f.Leg([0], [2], 1)]
    lb = [z2f.Leg([0], [2], -1), z2f.Leg([0], [5], 1)]
    a, b = _rand(la, 0, 3), _rand(lb, 0, 4)
    _, _, p, _ = z2f.permute((la, 0, a), [2, 0, 1])
    assert np.allclose(z2f.embed([la[2], la[0], la[1]], 0, p), np.transpose(z2f.embed(la, 0, a), [2, 0, 1]))
    _, _, c, _ = z2f.contract((la, 0, a), (lb, 0, b), [2], [0])
    ua = [u1.Leg([0], [l.degens[0]], l.dir) for l in la]
    ub = [u1.Leg([0], [l.degens[0]], l.dir) for l in lb]
    ref = np.tensordot(u1.embed(ua, 0, a), u1.embed(ub, 0, b), axes=([2], [0])).reshape(-1)
    assert np.allclose(c, ref)


def test_contraction_is_permute_then_matrix_product():
    # contracting A's legs (3, 1) with B's (0, 2) equals permuting A into
    # (free, contracted) order and B into (contracted, free) order by the
    # oracle's own permute, then summing a plain product over the contracted index
    la = [z2f.Leg([0, 1], [2, 1], 1), z2f.Leg([0, 1], [1, 2], -1), z2f.Leg([0, 1], [2, 2], 1),
          z2f.Leg([0, 1], [1, 3], 1)]
    lb = [z2f.Leg([0, 1], [1, 3], -1), z2f.Leg([0, 1], [2, 1], 1), z2f.Leg([0, 1], [1, 2], 1)]
    a, b = _rand(la, 1, 5), _rand(lb, 0, 6)
    legsC, PC, c, resid = z2f.contract((la, 1, a), (lb, 0, b), [3, 1], [0, 2])
    assert resid < 1e-12 and PC == 1
    la2, _, a2, _ = z2f.permute((la, 1, a), [0, 2, 3, 1])
    lb2, _, b2, _ = z2f.permute((lb, 0, b), [0, 2, 1])
    Ad, Bd = z2f.embed(la2, 1, a2), z2f.embed(lb2, 0, b2)
    ref = np.einsum("xycd,cdz->xyz", Ad, Bd)
    assert np.allclose(z2f.embed(legsC, PC, c), ref)
    # a pair of odd contracted legs exchanged on both sides: the signs cancel
    # only when both permutations reverse the same pairs, so they matter here
    sg = z2f.sign_field(la, [0, 2, 3, 1])
    assert (sg < 0).any()


def test_gradient_against_finite_differences():
    la = [z2f.Leg([0, 1], [2, 1], 1), z2f.Leg([0, 1], [1, 2], -1), z2f.Leg([0, 1], [2, 1], 1)]
    lb = [z2f.Leg([0, 1], [2, 1], -1), z2f.Leg([0, 1], [2, 1], -1), z2f.Leg([0, 1], [1, 2], 1)]
    a, b = _rand(la, 1, 7), _rand(lb, 0, 8)
    _, PC, c, _ = z2f.contract((la, 1, a), (lb, 0, b), [2, 0], [0, 1])
    g = np.random.default_rng(9).standard_normal(c.size)
    dA, dB, resid = z2f.contract_grad((la, 1, a), (lb, 0, b), [2, 0], [0, 1], g)
    assert resid < 1e-12
    f = lambda aa, bb: float(g @ z2f.contract((la, 1, aa), (lb, 0, bb), [2, 0], [0, 1])[2])
    h = 1e-6
    for i in range(a.size):
        e = np.zeros(a.size)
        e[i] = h
        assert abs((f(a + e, b) - f(a - e, b)) / (2 * h) - dA[i]) < 1e-7
    for i in range(b.size):
        e = np.zeros(b.size)
        e[i] = h
        assert abs((f(a, b + e) - f(a, b - e)) / (2 * h) - dB[i]) < 1e-7


def test_sectors_conserve_parity_and_fuse_adds_mod_2():
    legs = [z2f.Leg([0, 1], [1, 2], 1), z2f.Leg([0, 1], [2, 1], 1), z2f.Leg([0, 1], [1, 1], -1)]
    for P in (0, 1):
        for s in z2f.sectors(legs, P):
            assert sum(l.labels[i] for l, i in zip(legs, s)) % 2 == P
    data = _rand(legs, 1, 10)
    l2, P2, out, resid = z2f.fuse((legs, 1, data), 0)
    assert resid == 0.0 and l2[0].labels == [0, 1] and l2[0].degens == [1 * 2 + 2 * 1, 1 * 1 + 2 * 2]
    # fusing reorders nothing: the norm is kept
    assert np.isclose(np.linalg.norm(out), np.linalg.norm(data))
