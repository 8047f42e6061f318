"""Pins of the oracle's coupling coefficients (Ch. 5) against printed values and identities."""
import itertools
from math import sqrt

import numpy as np
import pytest

from oracle import cg as cgm
from tests.conftest import read_golden


def _spins(maxj2):
    return range(0, maxj2 + 1)


def test_printed_half_half_values():
    # Ch. 5, Example 6: the six printed CG values for 1/2 x 1/2
    for row in read_golden("cg_half_half.txt"):
        a = row.split()
        args = [int(x) for x in a[:6]]
        assert cgm.cg(*args) == pytest.approx(float(a[6]), abs=1e-15)


def test_printed_omega_matrices():
    # Ch. 5, Example 10 (Eq. eg101): omega_0, omega_1, omega_2
    for row in read_golden("omega.txt"):
        j2, rest = row.split(None, 1)
        j2 = int(j2)
        m = np.array([[float(x) for x in r.split()] for r in rest.split(";")])
        assert np.allclose(cgm.omega(j2), m / sqrt(j2 + 1), atol=1e-15)


def test_printed_generators():
    # Ch. 5, Examples 2-3: Jz and Jx (= (J+ + J-)/2) in the ascending basis
    s2 = 1 / sqrt(2)
    for row in read_golden("generators.txt"):
        name, j2, rest = row.split(None, 2)
        m = np.array([[s2 if x == "s2" else float(x) for x in r.split()]
                      for r in rest.split(";")])
        jz, jp, jm = cgm.generators(int(j2))
        got = jz if name == "Jz" else 0.5 * (jp + jm)
        assert np.allclose(got, m, atol=1e-15)


def test_singlet_formula():
    # Ch. 5, Eq. singletomega: <j m; j -m | 0 0> = (-1)^(j-m)/sqrt(2j+1)
    for j2 in _spins(9):
        for m2 in range(-j2, j2 + 1, 2):
            want = (-1) ** ((j2 - m2) // 2) / sqrt(j2 + 1)
            assert cgm.cg(j2, m2, j2, -m2, 0, 0) == pytest.approx(want, abs=1e-15)


def test_cg_orthogonality_both_ways():
    # Ch. 5, Eq. cgunitary
    for ja2, jb2 in itertools.product(_spins(5), _spins(5)):
        blocks = [cgm.cg_tensor(ja2, jb2, jc2).reshape((ja2 + 1) * (jb2 + 1), jc2 + 1)
                  for jc2 in range(abs(ja2 - jb2), ja2 + jb2 + 1, 2)]
        U = np.concatenate(blocks, axis=1)  # product basis x coupled basis
        assert U.shape[0] == U.shape[1]
        assert np.allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-14)
        assert np.allclose(U @ U.T, np.eye(U.shape[0]), atol=1e-14)


def test_coupled_states_obey_ladder_relations():
    # The coupled vectors |jc mc> = sum C |ma mb> (Eq. cg) must be eigenvectors of
    # the total Jz and be connected by the total J+ with the factor of
    # Eq. irrepladder; with the highest-weight coefficient <ja ja; jb jc-ja|jc jc>
    # positive (the phase the printed 1/2 x 1/2 values use) this fixes every sign.
    for ja2, jb2 in itertools.product(_spins(4), _spins(4)):
        za, pa, _ = cgm.generators(ja2)
        zb, pb, _ = cgm.generators(jb2)
        Jz = np.kron(za, np.eye(jb2 + 1)) + np.kron(np.eye(ja2 + 1), zb)
        Jp = np.kron(pa, np.eye(jb2 + 1)) + np.kron(np.eye(ja2 + 1), pb)
        for jc2 in range(abs(ja2 - jb2), ja2 + jb2 + 1, 2):
            c = cgm.cg_tensor(ja2, jb2, jc2).reshape(-1, jc2 + 1)
            jc = jc2 / 2
            for i in range(jc2 + 1):
                m = -jc + i
                assert np.allclose(Jz @ c[:, i], m * c[:, i], atol=1e-13)
                up = c[:, i + 1] * sqrt(jc * (jc + 1) - m * (m + 1)) if i < jc2 else 0 * c[:, i]
                assert np.allclose(Jp @ c[:, i], up, atol=1e-13)
            if ja2 + jb2 >= jc2 and abs(jc2 - ja2) <= jb2:
                assert cgm.cg(ja2, ja2, jb2, jc2 - ja2, jc2, jc2) > 0


def test_cg_against_sympy():
    wigner = pytest.importorskip("sympy.physics.wigner")
    from sympy import S
    for ja2, jb2 in itertools.product(_spins(4), _spins(4)):
        for jc2 in range(abs(ja2 - jb2), ja2 + jb2 + 1, 2):
            for ma2 in range(-ja2, ja2 + 1, 2):
                for mb2 in range(-jb2, jb2 + 1, 2):
                    if abs(ma2 + mb2) > jc2:
                        continue
                    ref = float(wigner.clebsch_gordan(S(ja2) / 2, S(jb2) / 2, S(jc2) / 2,
                                                      S(ma2) / 2, S(mb2) / 2, S(ma2 + mb2) / 2))
                    assert cgm.cg(ja2, ma2, jb2, mb2, jc2, ma2 + mb2) == pytest.approx(ref, abs=1e-14)


def test_swap_relation():
    # Ch. 5, Eq. braid3: C_{b,a->c} = (-1)^(ja+jb-jc) C_{a,b->c}
    for ja2, jb2 in itertools.product(_spins(5), _spins(5)):
        for jc2 in range(abs(ja2 - jb2), ja2 + jb2 + 1, 2):
            r = (-1) ** ((ja2 + jb2 - jc2) // 2)
            lhs = cgm.cg_tensor(jb2, ja2, jc2).transpose(1, 0, 2)
            assert np.allclose(lhs, r * cgm.cg_tensor(ja2, jb2, jc2), atol=1e-15)


def test_cup_cap_identity():
    # Ch. 5, Eq. wiggle
    for j2 in _spins(8):
        assert np.allclose(cgm.cup(j2) @ cgm.cap(j2), np.eye(j2 + 1), atol=1e-14)
        assert np.allclose(cgm.cap(j2) @ cgm.cup(j2), np.eye(j2 + 1), atol=1e-14)


def _sixj(a, b, c, d, e, f):
    return cgm.sixj_from_F(a, b, c, d, e, f)


def _admissible(a, b, c, d, e, f):
    return (cgm.triangle(a, b, c) and cgm.triangle(a, e, f)
            and cgm.triangle(d, b, f) and cgm.triangle(d, e, c))


def test_sixj_zero_argument_closed_form():
    # {a b c; 0 c b} = (-1)^(a+b+c) / sqrt((2b+1)(2c+1))
    for a, b, c in itertools.product(_spins(4), _spins(4), _spins(4)):
        if not cgm.triangle(a, b, c):
            continue
        want = (-1) ** ((a + b + c) // 2) / sqrt((b + 1) * (c + 1))
        assert _sixj(a, b, c, 0, c, b) == pytest.approx(want, abs=1e-14)


def test_sixj_tetrahedral_symmetry():
    rng = np.random.default_rng(5)
    n = 0
    while n < 40:
        a, b, c, d, e, f = (int(x) for x in rng.integers(0, 5, size=6))
        if not _admissible(a, b, c, d, e, f):
            continue
        n += 1
        v = _sixj(a, b, c, d, e, f)
        cols = [(a, d), (b, e), (c, f)]
        for perm in itertools.permutations(range(3)):
            pc = [cols[p] for p in perm]
            # column permutations, and swapping upper/lower in two columns
            for flip in [(0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1)]:
                col = [(y, x) if fl else (x, y) for (x, y), fl in zip(pc, flip)]
                w = _sixj(col[0][0], col[1][0], col[2][0], col[0][1], col[1][1], col[2][1])
                assert w == pytest.approx(v, abs=1e-13)


def test_sixj_orthogonality():
    # sum_x (2x+1)(2f+1) {a b x; c d f}{a b x; c d f'} = delta_{f f'}
    for a, b, c, d in itertools.product(_spins(3), _spins(3), _spins(3), _spins(3)):
        fs = [f for f in range(0, 9) if cgm.triangle(a, d, f) and cgm.triangle(c, b, f)]
        xs = [x for x in range(0, 9) if cgm.triangle(a, b, x) and cgm.triangle(c, d, x)]
        for f, f2 in itertools.product(fs, fs):
            s = sum((x + 1) * (f + 1) * _sixj(a, b, x, c, d, f) * _sixj(a, b, x, c, d, f2)
                    for x in xs)
            assert s == pytest.approx(1.0 if f == f2 else 0.0, abs=1e-13)


def test_sixj_against_sympy():
    wigner = pytest.importorskip("sympy.physics.wigner")
    from sympy import S
    rng = np.random.default_rng(11)
    n = 0
    while n < 60:
        a, b, c, d, e, f = (int(x) for x in rng.integers(0, 7, size=6))
        if not _admissible(a, b, c, d, e, f):
            continue
        n += 1
        ref = float(wigner.wigner_6j(*(S(x) / 2 for x in (a, b, c, d, e, f))))
        assert _sixj(a, b, c, d, e, f) == pytest.approx(ref, abs=1e-13)


def test_F_is_orthogonal_matrix():
    # Ch. 5, Eq. fmove: F relates two orthonormal bases
    for ja, jb, jc, J in itertools.product(_spins(3), _spins(3), _spins(3), _spins(5)):
        Ds = [d for d in range(0, 7) if cgm.triangle(ja, jb, d) and cgm.triangle(d, jc, J)]
        Es = [e for e in range(0, 7) if cgm.triangle(jb, jc, e) and cgm.triangle(ja, e, J)]
        if not Ds:
            continue
        F = np.array([[cgm.recoupling_F(d, e, ja, jb, jc, J) for e in Es] for d in Ds])
        assert F.shape[0] == F.shape[1]
        assert np.allclose(F @ F.T, np.eye(len(Ds)), atol=1e-13)


# The large-sector SU(2) workload couples leg spins 2j <= 8 into node spins
# 2e <= 16: the recoupling coefficients it uses have three arguments <= 8
# (the legs a, b and the spectator d) and three <= 16 (c, e, f).
def _workload_sixj_args(rng, n):
    out = []
    while len(out) < n:
        a, b, d = (int(x) for x in rng.integers(0, 9, size=3))
        c, e, f = (int(x) for x in rng.integers(0, 17, size=3))
        if _admissible(a, b, c, d, e, f):
            out.append((a, b, c, d, e, f))
    return out


def test_sixj_zero_argument_closed_form_at_workload_spins():
    for a, b, c in itertools.product(_spins(8), _spins(16), _spins(16)):
        if not cgm.triangle(a, b, c):
            continue
        want = (-1) ** ((a + b + c) // 2) / sqrt((b + 1) * (c + 1))
        assert _sixj(a, b, c, 0, c, b) == pytest.approx(want, abs=1e-14)


def test_sixj_against_sympy_at_workload_spins():
    wigner = pytest.importorskip("sympy.physics.wigner")
    from sympy import S
    rng = np.random.default_rng(12)
    args = _workload_sixj_args(rng, 150) + [(8, 8, 16, 8, 8, 16), (7, 8, 15, 8, 7, 16), (8, 8, 16, 8, 16, 8)]
    for a, b, c, d, e, f in args:
        if not _admissible(a, b, c, d, e, f):
            continue
        ref = float(wigner.wigner_6j(*(S(x) / 2 for x in (a, b, c, d, e, f))).evalf(30))
        assert _sixj(a, b, c, d, e, f) == pytest.approx(ref, abs=1e-14), (a, b, c, d, e, f)


def test_sixj_orthogonality_at_workload_spins():
    # sum_x (2x+1)(2f+1) {a b x; c d f}{a b x; c d f'} = delta_{f f'}, legs up to 2j = 8
    rng = np.random.default_rng(13)
    for _ in range(6):
        a, b, c, d = (int(x) for x in rng.integers(0, 9, size=4))
        if (a + b + c + d) % 2:
            d = max(d - 1, 0) if d else 1
        fs = [f for f in range(0, 17) if cgm.triangle(a, d, f) and cgm.triangle(c, b, f)]
        xs = [x for x in range(0, 17) if cgm.triangle(a, b, x) and cgm.triangle(c, d, x)]
        for f, f2 in itertools.product(fs, fs):
            s = sum((x + 1) * (f + 1) * _sixj(a, b, x, c, d, f) * _sixj(a, b, x, c, d, f2) for x in xs)
            assert s == pytest.approx(1.0 if f == f2 else 0.0, abs=1e-13)
