"""Host-side library logic against the oracle (no GPU): sector tables bit-exact,
recoupling coefficients and Gamma matrices against brute-force CG contraction."""
import itertools

import numpy as np
import pytest

from oracle import cg as ocg
from oracle import su2 as osu2
from oracle import u1 as ou1
from paper_1203_2222_gb300 import SU2, U1, Structure, su2_F, su2_gamma
from paper_1203_2222_gb300 import synthetic


def _check_u1(legs, Q):
    S = Structure(U1, legs, total=Q)
    lab, off = S.sectors()
    secs, offs, n = ou1.layout([ou1.Leg(*l) for l in legs], Q)
    assert S.numel == n and S.nsec == len(secs)
    assert [tuple(r) for r in lab.tolist()] == [tuple(s) for s in secs]
    assert off.tolist() == offs + [n]


def _check_su2(legs, tree):
    S = Structure(SU2, legs, tree=tree)
    lab, off = S.sectors()
    k = len(legs)
    secs, offs, n = osu2.layout([osu2.Leg(*l) for l in legs], tree if tree is not None else osu2.left_comb(k))
    assert S.numel == n and S.nsec == len(secs)
    got = [(tuple(r[:k]), tuple(r[k:])) for r in lab.tolist()]
    assert got == [(tuple(s[0]), tuple(s[1])) for s in secs]
    assert off.tolist() == offs + [n]


def test_u1_sector_tables_match_oracle():
    rng = np.random.default_rng(0)
    for rank in range(0, 5):
        for Q in (-1, 0, 2):
            legs = [([-2, -1, 0, 1, 3], rng.integers(1, 4, 5).tolist(), int(rng.choice([1, -1])))
                    for _ in range(rank)]
            _check_u1(legs, Q)


def test_u1_workload_tables_match_oracle():
    c = synthetic.u1_pairwise()
    _check_u1(c["A"], 0)
    _check_u1(c["B"], 0)
    m = synthetic.u1_mps_heff(D=256, qmax=6, sigma=2.0)
    for name in ("L", "A", "W", "R"):
        _check_u1(m[name], 0)


TREES4 = [None, [(1, 2), (0, 4), (5, 3)], [(0, 1), (2, 3), (4, 5)], [(2, 3), (1, 4), (0, 5)],
          [(1, 2), (4, 3), (0, 5)]]


@pytest.mark.parametrize("tree", TREES4)
def test_su2_sector_tables_match_oracle(tree):
    rng = np.random.default_rng(1)
    legs = [([0, 1, 2, 3, 4], rng.integers(1, 4, 5).tolist(), int(rng.choice([1, -1]))) for _ in range(4)]
    _check_su2(legs, tree)


def test_su2_small_ranks_match_oracle():
    _check_su2([([0, 2], [1, 2], 1)], None)
    _check_su2([([0, 1, 2], [1, 2, 1], 1), ([1, 2], [2, 1], -1)], None)
    _check_su2([([0, 1, 2], [1, 2, 1], 1)] * 3, None)
    _check_su2([([0, 1, 2], [1, 2, 1], 1)] * 5, [(0, 1), (2, 3), (5, 6), (7, 4)])


def test_recoupling_F_matches_oracle():
    for jd, je, ja, jb, jc, J in itertools.product(range(4), repeat=6):
        assert su2_F(jd, je, ja, jb, jc, J) == pytest.approx(
            ocg.recoupling_F(jd, je, ja, jb, jc, J), abs=1e-14)


def _workload_F_args(rng, n):
    """Arguments (jd, je, ja, jb, jc, J) of F as the large-sector workload
    uses them: legs ja, jb, jc with 2j <= 8, node spins jd, je, J <= 16."""
    out = []
    while len(out) < n:
        ja, jb, jc = (int(x) for x in rng.integers(0, 9, size=3))
        jd, je, J = (int(x) for x in rng.integers(0, 17, size=3))
        if (ocg.triangle(ja, jb, jd) and ocg.triangle(jd, jc, J) and ocg.triangle(jb, jc, je)
                and ocg.triangle(ja, je, J)):
            out.append((jd, je, ja, jb, jc, J))
    return out


def test_recoupling_F_exact_at_workload_spins():
    """The library's F (Racah's single sum over long-double factorials)
    against exact values (sympy's 6j in rational arithmetic, Ch. 5 Eq. sixj
    with the sign and normalisation of Eq. f) across the workload's spins,
    including the largest coupled spins, where the sum's cancellation is
    worst."""
    wigner = pytest.importorskip("sympy.physics.wigner")
    from sympy import Rational, sqrt as ssqrt
    rng = np.random.default_rng(21)
    args = _workload_F_args(rng, 400)
    args += [a for a in itertools.product([14, 15, 16], [14, 15, 16], [7, 8], [7, 8], [7, 8], [14, 15, 16])
             if ocg.triangle(a[2], a[3], a[0]) and ocg.triangle(a[0], a[4], a[5]) and ocg.triangle(a[3], a[4], a[1])
             and ocg.triangle(a[2], a[1], a[5])]
    for jd, je, ja, jb, jc, J in args:
        six = wigner.wigner_6j(*(Rational(x, 2) for x in (ja, jb, jd, jc, J, je)))
        exact = (-1) ** ((ja + jb + jc + J) // 2) * ssqrt((jd + 1) * (je + 1)) * six
        want = float(exact.evalf(30))
        assert su2_F(jd, je, ja, jb, jc, J) == pytest.approx(want, abs=1e-14), (jd, je, ja, jb, jc, J)


def test_recoupling_F_matches_oracle_at_workload_spins():
    """The library's F against the oracle's F (four CG tensors contracted,
    Ch. 5 Eq. f with the fourth-factor reading) at the workload's spins."""
    rng = np.random.default_rng(22)
    for jd, je, ja, jb, jc, J in _workload_F_args(rng, 120):
        assert su2_F(jd, je, ja, jb, jc, J) == pytest.approx(
            ocg.recoupling_F(jd, je, ja, jb, jc, J), abs=1e-14), (jd, je, ja, jb, jc, J)


def _brute_gamma(spins, tree_in, perm, tree_out):
    k = len(spins)
    legs = [osu2.Leg([s], [1], 1) for s in spins]
    legs_o = [legs[p] for p in perm]
    ti = tree_in if tree_in is not None else osu2.left_comb(k)
    to = tree_out if tree_out is not None else osu2.left_comb(k)
    si = osu2.sectors(legs, ti)
    so = osu2.sectors(legs_o, to)
    G = np.zeros((len(so), len(si)))
    for i, a in enumerate(si):
        qa = np.transpose(osu2.structure_tensor(legs, ti, a), perm)
        for o, b in enumerate(so):
            G[o, i] = np.sum(qa * osu2.structure_tensor(legs_o, to, b))
    return G, [s[1] for s in si], [s[1] for s in so]


GAMMA_CASES = [
    ([1, 1, 2], None, [1, 0, 2], None),
    ([2, 2, 2], None, [2, 0, 1], None),
    ([1, 2, 3], None, [0, 2, 1], [(1, 2), (0, 3)]),
    ([2, 2, 2, 2], None, [0, 2, 1, 3], [(0, 1), (2, 3), (4, 5)]),
    ([1, 3, 2, 4], None, [3, 1, 0, 2], None),
    ([4, 4, 4, 4], [(1, 2), (0, 4), (5, 3)], [2, 3, 0, 1], [(2, 3), (1, 4), (0, 5)]),
    ([1, 1, 1, 1], None, [0, 1, 2, 3], [(1, 2), (4, 3), (0, 5)]),
    ([2, 1, 1, 2, 2], None, [4, 0, 3, 1, 2], [(0, 1), (2, 3), (6, 4), (5, 7)]),
    ([3, 3, 2, 2, 2], [(0, 1), (2, 3), (5, 6), (7, 4)], [1, 0, 2, 4, 3], None),
    # the large-sector workload's recoupling at its largest leg spins (2j = 8, node spins to 16)
    ([8, 8, 8, 8], None, [0, 2, 1, 3], [(0, 1), (2, 3), (4, 5)]),
    ([7, 8, 5, 6], None, [0, 2, 1, 3], [(0, 1), (2, 3), (4, 5)]),
    ([8, 7, 8, 5], [(1, 2), (0, 4), (5, 3)], [3, 1, 2, 0], None),
    # rank 6 (the library's largest): comb to a balanced tree, and back through a permutation
    ([1, 1, 1, 1, 2, 2], None, [0, 2, 1, 3, 5, 4], [(0, 1), (2, 3), (4, 5), (6, 7), (9, 8)]),
    ([2, 1, 1, 2, 1, 1], [(0, 1), (2, 3), (4, 5), (6, 7), (9, 8)], [3, 0, 5, 1, 4, 2], None),
]


@pytest.mark.parametrize("case", range(len(GAMMA_CASES)))
def test_gamma_matches_brute_force_cg_contraction(case):
    spins, ti, perm, to = GAMMA_CASES[case]
    G, li, lo = su2_gamma(spins, ti, perm, to)
    Gb, bli, blo = _brute_gamma(spins, ti, perm, to)
    assert [tuple(r) for r in li.tolist()] == [tuple(r) for r in bli]
    assert [tuple(r) for r in lo.tolist()] == [tuple(r) for r in blo]
    assert G.shape == Gb.shape and G.size > 0
    assert np.allclose(G, Gb, atol=1e-13)
    # Gamma between orthonormal bases is orthogonal
    assert np.allclose(G @ G.T, np.eye(G.shape[0]), atol=1e-12)


def test_gamma_random_cases_match_brute_force():
    rng = np.random.default_rng(7)
    n = 0
    while n < 12:
        k = int(rng.integers(3, 6))
        spins = rng.integers(0, 4, k).tolist()
        perm = rng.permutation(k).tolist()
        G, _, _ = su2_gamma(spins, None, perm, None)
        if G.size == 0:
            continue
        Gb, _, _ = _brute_gamma(spins, None, perm, None)
        assert np.allclose(G, Gb, atol=1e-13), (spins, perm)
        n += 1
