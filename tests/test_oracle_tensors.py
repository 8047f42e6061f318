"""Pins of the oracle's tensor definitions against what the thesis and the mathematics fix."""
import itertools
from math import sqrt

import numpy as np
import pytest

from oracle import cg as cgm
from oracle import contract as oc
from oracle import su2, u1
from tests.conftest import read_golden


def _rng(s=0):
    return np.random.default_rng(s)


def _rand_u1_legs(rng, dirs, qs=(-1, 0, 1)):
    return [u1.Leg(list(qs), [int(x) for x in rng.integers(1, 3, len(qs))], d) for d in dirs]


def _rand_su2_legs(rng, dirs, spins=(0, 1, 2)):
    return [su2.Leg(list(spins), [int(x) for x in rng.integers(1, 3, len(spins))], d) for d in dirs]


# ---------------------------------------------------------------- U(1) -----------

def test_u1_dense_product_conserves_charge():
    # a dense product of two charge-conserving tensors has no weight outside the
    # result's allowed sectors (nothing in the dense contraction enforces this)
    rng = _rng(1)
    for QA, QB in [(0, 0), (1, -2), (2, 1)]:
        la = _rand_u1_legs(rng, [1, -1, 1])
        lb = [la[2].dual()] + _rand_u1_legs(rng, [1, -1])
        a = rng.standard_normal(u1.layout(la, QA)[2])
        b = rng.standard_normal(u1.layout(lb, QB)[2])
        _, _, _, resid = oc.contract("u1", (la, QA, a), (lb, QB, b), [2], [0])
        assert resid < 1e-12
        # and a generic dense tensor does violate it
        dense = rng.standard_normal([l.dim for l in la])
        assert u1.extract(la, QA, dense)[1] > 0.1


def test_u1_single_charge_is_dense():
    rng = _rng(2)
    la = [u1.Leg([0], [3], 1), u1.Leg([0], [4], -1), u1.Leg([0], [2], 1)]
    lb = [la[1].dual(), u1.Leg([0], [5], -1)]
    a = rng.standard_normal(24)
    b = rng.standard_normal(20)
    _, _, c, _ = oc.contract("u1", (la, 0, a), (lb, 0, b), [1], [0])
    want = np.einsum("ijk,jl->ikl", a.reshape(3, 4, 2), b.reshape(4, 5))
    assert np.allclose(c, want.reshape(-1), atol=1e-13)


def test_u1_contract_matches_brute_force_loops():
    rng = _rng(3)
    la = _rand_u1_legs(rng, [1, 1, -1])
    lb = [la[1].dual(), la[2].dual(), u1.Leg([-1, 0, 1], [1, 2, 1], -1)]
    a = rng.standard_normal(u1.layout(la, 0)[2])
    b = rng.standard_normal(u1.layout(lb, 0)[2])
    lc, Qc, c, _ = oc.contract("u1", (la, 0, a), (lb, 0, b), [1, 2], [0, 1])
    Ad, Bd = u1.embed(la, 0, a), u1.embed(lb, 0, b)
    Cd = np.zeros((la[0].dim, lb[2].dim))
    for i in range(la[0].dim):
        for l in range(lb[2].dim):
            s = 0.0
            for j in range(la[1].dim):
                for k in range(la[2].dim):
                    s += Ad[i, j, k] * Bd[j, k, l]
            Cd[i, l] = s
    assert np.allclose(u1.embed(lc, Qc, c), Cd, atol=1e-12)


def test_u1_block_order_is_lexicographic():
    legs = [u1.Leg([-1, 0, 1], [1, 2, 3], 1), u1.Leg([-1, 0, 1], [2, 1, 1], -1)]
    secs, offs, n = u1.layout(legs, 0)
    assert secs == [(0, 0), (1, 1), (2, 2)]
    assert offs == [0, 2, 4] and n == 7
    secs, _, _ = u1.layout(legs, 1)
    assert secs == [(1, 0), (2, 1)]


def test_u1_fuse_is_a_permutation_of_the_product_basis():
    rng = _rng(4)
    legs = _rand_u1_legs(rng, [1, 1, -1])
    d, X = u1.fusion_matrix(legs[0], legs[1])
    M = X.reshape(-1, X.shape[2])
    assert np.allclose(M.T @ M, np.eye(M.shape[1]))
    assert d.dim == legs[0].dim * legs[1].dim
    x = rng.standard_normal(u1.layout(legs, 0)[2])
    _, _, f, resid = oc.fuse("u1", (legs, 0, x), 0)
    assert resid == 0.0 and np.isclose(np.linalg.norm(f), np.linalg.norm(x))


# ---------------------------------------------------------------- SU(2) ----------

TREES4 = [su2.left_comb(4), [(1, 2), (0, 4), (5, 3)], [(0, 1), (2, 3), (4, 5)],
          [(2, 3), (1, 4), (0, 5)]]


@pytest.mark.parametrize("dirs", [(1, 1, 1, 1), (1, -1, 1, -1), (-1, -1, 1, 1)])
@pytest.mark.parametrize("tree", range(len(TREES4)))
def test_su2_embedding_is_invariant(dirs, tree):
    # Ch. 5, Eq. Tinv: the generators annihilate the embedded tensor
    rng = _rng(10 + tree)
    legs = _rand_su2_legs(rng, dirs, spins=(0, 1, 2, 3))
    nodes = TREES4[tree]
    x = rng.standard_normal(su2.layout(legs, nodes)[2])
    d = su2.embed(legs, nodes, x)
    assert su2.invariance_residual(legs, d) < 1e-12 * max(1.0, np.linalg.norm(d))
    y, resid = su2.extract(legs, nodes, d)
    assert resid < 1e-12 and np.allclose(x, y, atol=1e-13)
    # embedding is an isometry: the tree basis is orthonormal
    assert np.isclose(np.linalg.norm(d), np.linalg.norm(x))
    # a generic dense tensor is not invariant
    g = rng.standard_normal(d.shape)
    assert su2.invariance_residual(legs, g) > 0.1
    assert su2.extract(legs, nodes, g)[1] > 0.1


def test_su2_all_spin_zero_is_dense():
    rng = _rng(20)
    la = [su2.Leg([0], [3], 1), su2.Leg([0], [2], -1), su2.Leg([0], [4], 1)]
    lb = [la[2].dual(), su2.Leg([0], [5], 1)]
    a = rng.standard_normal(24)
    b = rng.standard_normal(20)
    assert np.allclose(su2.embed(la, su2.left_comb(3), a), a.reshape(3, 2, 4))
    _, _, c, _ = oc.contract("su2", (la, su2.left_comb(3), a), (lb, su2.left_comb(2), b), [2], [0])
    want = np.einsum("ijk,kl->ijl", a.reshape(3, 2, 4), b.reshape(4, 5))
    assert np.allclose(c, want.reshape(-1), atol=1e-13)


def test_su2_rank3_is_wigner_eckart():
    # Ch. 5, Eq. three22: T_abc = P_{ja jb jc} C_{a,b->c}; with legs (in, in, out)
    # the tree decomposition gives P (x) Q with Q proportional to the CG tensor
    rng = _rng(21)
    legs = [su2.Leg([1, 2], [2, 1], 1), su2.Leg([0, 1], [1, 2], 1), su2.Leg([1, 2, 3], [1, 1, 2], 1)]
    nodes = su2.left_comb(3)
    for s in su2.sectors(legs, nodes):
        ja, jb, jc = (l.labels[p] for l, p in zip(legs, s[0]))
        Q = su2.structure_tensor(legs, nodes, s)
        C = cgm.cg_tensor(ja, jb, jc)  # (a, b, c)
        # all-out rank 3: Q[ma, mb, mc] = sum_e C_{a,b->e}(ma,mb,me) C_{e,c->0}(me, mc, 0)
        # = C_{a,b->c}(ma, mb, -mc) (-1)^(jc+mc)/sqrt(2jc+1)  (singlet formula)
        Cflip = C[:, :, ::-1]
        ph = np.array([(-1) ** ((jc - (-jc + 2 * i)) // 2) for i in range(jc + 1)])[::-1]
        want = Cflip * ph / sqrt(jc + 1)
        assert np.allclose(Q, want, atol=1e-14)


def test_su2_rank2_contraction_is_blockwise_matmul():
    # Ch. 5, Eq. blockmult: for matrices the contraction is blockwise.  With the
    # cup on the incoming index, the (in, out) canonical block reads
    # P_j (x) cup_j omega_j = P_j (x) (-1)^(2j) I/sqrt(2j+1) (Ch. 5, Ex. 12), so
    # the product block is (-1)^(2j) M_j N_j / sqrt(2j+1).
    rng = _rng(22)
    spins, deg = [0, 1, 2, 3], [2, 3, 1, 2]
    lm = [su2.Leg(spins, deg, -1), su2.Leg(spins, deg, 1)]
    ln = [su2.Leg(spins, deg, -1), su2.Leg(spins, deg, 1)]
    t = su2.left_comb(2)
    m = rng.standard_normal(su2.layout(lm, t)[2])
    n = rng.standard_normal(su2.layout(ln, t)[2])
    _, _, c, resid = oc.contract("su2", (lm, t, m), (ln, t, n), [1], [0])
    assert resid < 1e-12
    off = 0
    for j2, d in zip(spins, deg):
        M = m[off:off + d * d].reshape(d, d)
        N = n[off:off + d * d].reshape(d, d)
        want = (-1) ** j2 * (M @ N) / sqrt(j2 + 1)
        assert np.allclose(c[off:off + d * d].reshape(d, d), want, atol=1e-13)
        off += d * d


def test_su2_contraction_result_is_invariant():
    rng = _rng(23)
    la = _rand_su2_legs(rng, [1, -1, 1, 1], spins=(0, 1, 2))
    lb = [la[2].dual(), la[3].dual()] + _rand_su2_legs(rng, [-1, 1], spins=(0, 1, 2))
    ta, tb = TREES4[1], TREES4[2]
    a = rng.standard_normal(su2.layout(la, ta)[2])
    b = rng.standard_normal(su2.layout(lb, tb)[2])
    lc, tc, c, resid = oc.contract("su2", (la, ta, a), (lb, tb, b), [2, 3], [0, 1])
    assert resid < 1e-12
    assert su2.invariance_residual(lc, su2.embed(lc, tc, c)) < 1e-11


def test_su2_recoupling_is_product_of_F():
    # Ch. 5, Eq. fmove and the S = F F example: for single degeneracies the
    # overlap between the bases of (((A,B)E,C)F,D)J and ((A,B)E,(C,D)H)J is one F,
    # and to (A,(B,(C,D)H)G)J a product of two F's.  A fifth leg X (spin J) closes
    # the tree to spin 0.
    rng = _rng(24)
    J = 2
    legs = [su2.Leg([1], [1], 1), su2.Leg([1], [1], 1), su2.Leg([2], [1], 1),
            su2.Leg([1], [1], 1), su2.Leg([J], [1], 1)]
    t1 = [(0, 1), (5, 2), (6, 3), (7, 4)]
    t2 = [(0, 1), (2, 3), (5, 6), (7, 4)]
    t3 = [(2, 3), (1, 5), (0, 6), (7, 4)]
    s1, _, _ = su2.layout(legs, t1)
    s2, _, _ = su2.layout(legs, t2)
    s3, _, _ = su2.layout(legs, t3)
    A, B, C, D = 1, 1, 2, 1
    for x in s1:
        E, F, _J = x[1]
        q1 = su2.structure_tensor(legs, t1, x)
        for y in s2:
            E2, H, _ = y[1]
            ov = float(np.sum(q1 * su2.structure_tensor(legs, t2, y)))
            want = cgm.recoupling_F(F, H, E, C, D, J) if E2 == E else 0.0
            assert ov == pytest.approx(want, abs=1e-13)
        for z in s3:
            H, G, _ = z[1]
            ov = float(np.sum(q1 * su2.structure_tensor(legs, t3, z)))
            want = cgm.recoupling_F(F, H, E, C, D, J) * cgm.recoupling_F(E, G, A, B, H, J)
            assert ov == pytest.approx(want, abs=1e-13)


def test_su2_swap_factor_in_permute():
    # Ch. 5, Eq. perm11: swapping the two legs of one node multiplies by R
    rng = _rng(25)
    legs = _rand_su2_legs(rng, [1, 1, 1], spins=(0, 1, 2, 3))
    t = su2.left_comb(3)
    secs, offs, n = su2.layout(legs, t)
    x = rng.standard_normal(n)
    l2, t2, y, resid = oc.permute("su2", (legs, t, x), [1, 0, 2], t)
    assert resid < 1e-12
    secs2, offs2, _ = su2.layout(l2, t2)
    for s, o in zip(secs, offs):
        ja, jb = legs[0].labels[s[0][0]], legs[1].labels[s[0][1]]
        e = s[1][0]
        i2 = secs2.index(((s[0][1], s[0][0], s[0][2]), s[1]))
        shp = su2.block_shape(legs, s)
        P = x[o:o + int(np.prod(shp))].reshape(shp)
        P2 = y[offs2[i2]:offs2[i2] + P.size].reshape(shp[1], shp[0], shp[2])
        r = (-1) ** ((ja + jb - e) // 2)
        assert np.allclose(P2, r * P.transpose(1, 0, 2), atol=1e-13)


def test_su2_fused_leg_example8():
    # Ch. 5, Example 8 (read with V^(A) = V_1, V^(B) = 2V_0 + V_1: the printed example is inconsistent)
    a = su2.Leg([2], [1], 1)
    b = su2.Leg([0, 2], [2, 1], 1)
    d, pairs = su2.fused_leg(a, b)
    assert d.labels == [0, 2, 4] and d.degens == [1, 3, 1]


def test_su2_fusing_tensor_is_isometric_and_fuse_is_invariant():
    rng = _rng(26)
    for dirs in [(1, 1, -1), (-1, -1, 1)]:
        legs = _rand_su2_legs(rng, dirs, spins=(0, 1, 2))
        d, U = su2.fusing_tensor(legs[0].dual() if dirs[0] < 0 else legs[0],
                                 legs[1].dual() if dirs[1] < 0 else legs[1])
        M = U.reshape(-1, U.shape[2])
        assert np.allclose(M.T @ M, np.eye(M.shape[1]), atol=1e-13)
        x = rng.standard_normal(su2.layout(legs, su2.left_comb(3))[2])
        l2, t2, f, resid = oc.fuse("su2", (legs, su2.left_comb(3), x), 0)
        assert resid < 1e-12
        assert np.isclose(np.linalg.norm(f), np.linalg.norm(x))
        assert su2.invariance_residual(l2, su2.embed(l2, t2, f)) < 1e-11


def test_storage_counts():
    # Ch. 5, Examples 10 and 11 (V = V0 + 3V1 + V2 on each leg)
    rows = [[int(v) for v in r.split()] for r in read_golden("storage_counts.txt")]
    for rank, dense, nblk, ncoef in rows:
        legs = [su2.Leg([0, 2, 4], [1, 3, 1], 1) for _ in range(rank)]
        assert int(np.prod([l.dim for l in legs])) == dense
        if rank == 2:
            secs, _, n = su2.layout(legs, su2.left_comb(2))
        else:
            # rank 3 canonical form: blocks per compatible (ja, jb, jc)
            secs = [s for s in itertools.product(range(3), repeat=3)
                    if cgm.triangle(*[legs[0].labels[i] for i in s])]
            n = sum(int(np.prod([legs[l].degens[i] for l, i in enumerate(s)])) for s in secs)
        assert len(secs) == nblk and n == ncoef


def test_degdist_bond_dimensions():
    # Table degdist: chi = sum_j (2j+1) d_j
    for row in read_golden("degdist.txt"):
        chi, js, ds = (x.split() for x in row.split(";"))
        leg = su2.Leg([2 * int(j) for j in js], [int(d) for d in ds], 1)
        assert leg.dim == int(chi[0])


# ------------------------------------------------------------ gradients ----------

@pytest.mark.parametrize("group", ["u1", "su2"])
def test_contract_grad_matches_finite_differences(group):
    rng = _rng(30)
    if group == "u1":
        la = _rand_u1_legs(rng, [1, -1, 1])
        lb = [la[2].dual()] + _rand_u1_legs(rng, [1])
        ta, tb = 0, 1
        lay = u1.layout
    else:
        la = _rand_su2_legs(rng, [1, -1, 1], spins=(0, 1, 2))
        lb = [la[2].dual()] + _rand_su2_legs(rng, [1], spins=(0, 1, 2))
        ta, tb = su2.left_comb(3), su2.left_comb(2)
        lay = su2.layout
    a = rng.standard_normal(lay(la, ta)[2])
    b = rng.standard_normal(lay(lb, tb)[2])
    lc, tc, c, _ = oc.contract(group, (la, ta, a), (lb, tb, b), [2], [0])
    g = rng.standard_normal(c.size)
    dA, dB, resid = oc.contract_grad(group, (la, ta, a), (lb, tb, b), [2], [0], g)
    assert resid < 1e-12

    def f(a_, b_):
        return float(g @ oc.contract(group, (la, ta, a_), (lb, tb, b_), [2], [0])[2])

    h = 1e-6
    for _ in range(3):
        va, vb = rng.standard_normal(a.size), rng.standard_normal(b.size)
        fd = (f(a + h * va, b + h * vb) - f(a - h * va, b - h * vb)) / (2 * h)
        assert fd == pytest.approx(float(dA @ va + dB @ vb), rel=1e-7, abs=1e-8)


# ------------------------------------------------------- sampled dense elements ---

@pytest.mark.parametrize("tree", [None, [(1, 2), (0, 4), (5, 3)], [(0, 1), (2, 3), (4, 5)]])
def test_su2_embed_slice_is_the_slice_of_the_embedding(tree):
    # embed_slice only visits the sectors whose spins match the fixed legs: every
    # pattern of fixed legs must reproduce the same slice of the full embedding
    rng = _rng(11)
    legs = [su2.Leg([0, 1, 2], [2, 1, 2], 1), su2.Leg([1, 3], [1, 2], -1),
            su2.Leg([0, 2], [2, 1], 1), su2.Leg([1, 2, 3], [1, 1, 2], 1)]
    nodes = tree or su2.left_comb(4)
    n = su2.layout(legs, nodes)[2]
    x = rng.standard_normal(n)
    dense = su2.embed(legs, nodes, x)
    for fixed in ({0: 3}, {1: 2, 3: 5}, {0: 1, 1: 0, 2: 3, 3: 4}, {2: 0}, {}):
        idx = tuple(fixed.get(l, slice(None)) for l in range(4))
        assert np.array_equal(su2.embed_slice(legs, nodes, x, fixed), dense[idx])


def test_su2_sampled_contraction_element_matches_dense_contraction():
    # one element of C = contract(A, B) from two embedded slices equals the
    # element of the dense brute-force contraction
    rng = _rng(12)
    la = [su2.Leg([0, 1, 2], [1, 2, 1], 1) for _ in range(4)]
    lb = [la[1].dual(), la[3].dual(), su2.Leg([0, 2], [2, 1], 1), su2.Leg([1, 3], [1, 1], 1)]
    na, nb = su2.layout(la, su2.left_comb(4))[2], su2.layout(lb, su2.left_comb(4))[2]
    xa, xb = rng.standard_normal(na), rng.standard_normal(nb)
    Ad, Bd = su2.embed(la, su2.left_comb(4), xa), su2.embed(lb, su2.left_comb(4), xb)
    Cd = oc.contract_dense(Ad, Bd, [1, 3], [0, 1])
    for _ in range(12):
        i0, i2 = (int(rng.integers(l.dim)) for l in (la[0], la[2]))
        i4, i5 = (int(rng.integers(l.dim)) for l in (lb[2], lb[3]))
        sa = su2.embed_slice(la, su2.left_comb(4), xa, {0: i0, 2: i2})
        sb = su2.embed_slice(lb, su2.left_comb(4), xb, {2: i4, 3: i5})
        assert abs(float(np.sum(sa * sb)) - Cd[i0, i2, i4, i5]) <= 1e-12 * max(1.0, abs(Cd[i0, i2, i4, i5]))
