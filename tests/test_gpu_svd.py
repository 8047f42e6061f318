"""GPU parity of the blockwise SVD (include/symtensor.h, sym_svd_*) against the
FP64 oracle (oracle/svd.py).

What is unique is compared element by element: the singular values, the
truncation counts (integer decisions taken on each side's own FP64 values),
and the truncated product U diag(S) V.  The singular vectors are unique up
to signs (and rotations inside degenerate values), so for them the test
checks what makes them valid: orthonormal columns of U and rows of V.
Tolerance: 1e-12 relative to the largest singular value (FP64 on both sides).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import su2 as osu2  # noqa: E402
from oracle import svd as osvd  # noqa: E402
from oracle import u1 as ou1  # noqa: E402
from oracle import z2f as oz2f  # noqa: E402

TOL = 1e-12


def _P():
    import paper_1203_2222_gb300 as P
    return P


def _mods(group):
    P = _P()
    return {"u1": (P.U1, ou1), "z2f": (P.Z2F, oz2f), "su2": (P.SU2, osu2)}[group]


def _otot(group, total):
    return osu2.left_comb(2) if group == "su2" else total


def _tensor(group, legs, total, values):
    P = _P()
    g, m = _mods(group)
    S = P.Structure(g, legs, total=total)
    T = P.SymTensor(S, torch.as_tensor(values, dtype=torch.float64).cuda())
    return S, T, ([m.Leg(*l) for l in legs], _otot(group, total), np.asarray(values, dtype=np.float64))


def _dense_bond(group, X, first_is_bond):
    """Dense matrix of a factor: (rows, bond) for U, (bond, cols) for V."""
    _, m = _mods(group)
    legs = [m.Leg(*l) for l in X.structure.legs]
    d = m.embed(legs, _otot(group, X.structure.total), X.data.cpu().numpy())
    return d.reshape(d.shape[0], -1) if first_is_bond else d.reshape(-1, d.shape[-1])


def _check(group, legs, total, nrow, values, chi=None, cutoff=0.0):
    P = _P()
    S, T, To = _tensor(group, legs, total, values)
    plan = P.svd_plan(S, nrow)
    Sg = plan.execute(T.data).cpu().numpy()
    fac, bd = osvd.svd(group, To, nrow)
    Smax = max(float(np.max(fac[x][1])) for x in fac)
    So = np.concatenate([fac[x][1] for x in sorted(fac)])
    assert np.max(np.abs(Sg - So)) <= TOL * Smax
    sweeps, _ = plan.stats()
    sweeps32, _ = plan.stats(fp32=True)
    assert max(sweeps) < 64 and max(sweeps32) <= 40
    keep = plan.truncation(Sg, chi, cutoff)
    ko = osvd.truncation({x: fac[x][1] for x in fac}, chi, cutoff, group=group)
    assert keep == [ko[x] for x in plan.labels]
    M = osvd.matrix(group, To, nrow)
    Uo, kept, Vo = osvd.factors(group, To, nrow, ko, absorb=1, fac=fac)
    _, m = _mods(group)
    Ud, Vd = m.embed(*Uo), m.embed(*Vo)
    ref = Ud.reshape(-1, Ud.shape[-1]) @ Vd.reshape(Vd.shape[0], -1)
    for absorb in (0, 1, 2):
        U, Sk, V = P.svd(T, nrow, chi=chi, cutoff=cutoff, absorb=absorb)
        Sk = Sk.cpu().numpy()
        assert np.max(np.abs(Sk - np.concatenate([kept[x] for x in sorted(kept)]))) <= TOL * Smax
        Um, Vm = _dense_bond(group, U, False), _dense_bond(group, V, True)
        Sd = osvd.dense_values(group, {x: Sk[o:o + k] for x, k, o in zip(
            [x for x, k in zip(plan.labels, keep) if k], [k for k in keep if k],
            np.cumsum([0] + [k for k in keep if k])[:-1])})
        prod = Um @ (np.diag(Sd) if absorb == 0 else np.eye(len(Sd))) @ Vm
        assert np.max(np.abs(prod - ref)) <= TOL * Smax
        # orthonormal vectors (a vector of a numerically zero singular value
        # is only defined up to the rest, and is written as zeros when exactly 0)
        live = np.where(Sd > 1e-10 * Smax)[0]
        if absorb != 1:
            Ul = Um[:, live]
            assert np.max(np.abs(Ul.T @ Ul - np.eye(len(live)))) <= TOL
        if absorb != 2:
            Vl = Vm[live, :]
            assert np.max(np.abs(Vl @ Vl.T - np.eye(len(live)))) <= TOL
        # U and V carry nothing outside their blocks (their layouts are the library's own)
        for X in (U, V):
            legsX = [m.Leg(*l) for l in X.structure.legs]
            assert X.structure.numel == m.layout(legsX, _otot(group, X.structure.total))[2]
    if chi is None and not cutoff:
        assert np.max(np.abs(ref - M)) <= TOL * Smax
    P.device_status()
    return plan


def _rand(group, legs, total, seed):
    _, m = _mods(group)
    n = m.layout([m.Leg(*l) for l in legs], _otot(group, total))[2]
    return np.random.default_rng(seed).standard_normal(n)


U1_SMALL = [([-1, 0, 1], [2, 3, 1], 1), ([0, 1], [2, 2], 1), ([-1, 0, 2], [1, 2, 2], -1), ([0, 1], [1, 3], -1)]
Z2F_SMALL = [([0, 1], [3, 2], 1), ([0, 1], [1, 2], -1), ([0, 1], [2, 3], 1)]


@pytest.mark.parametrize("group,legs,total,nrow", [
    ("u1", U1_SMALL, 0, 2), ("u1", U1_SMALL, 1, 1), ("u1", U1_SMALL, -1, 3),
    ("z2f", Z2F_SMALL, 0, 1), ("z2f", Z2F_SMALL, 1, 2)])
def test_small_tensors(group, legs, total, nrow):
    _check(group, legs, total, nrow, _rand(group, legs, total, 21))


def test_ragged_blocks_tall_wide_odd():
    # blocks from 1 x 1 to ~120 x 60 and ~60 x 120: odd and even column
    # counts (the round-robin's bye), tall and wide (A = M^T), several warps
    legs = [([-2, -1, 0, 1, 2], [3, 17, 40, 9, 1], -1), ([0, 1], [1, 1], -1), ([-3, -2, -1, 0, 1, 2, 3],
                                                                               [2, 5, 33, 61, 20, 7, 1], 1)]
    vals = _rand("u1", legs, 0, 22)
    _check("u1", legs, 0, 2, vals)
    _check("u1", legs, 0, 1, vals)
    _check("u1", legs, 0, 2, vals, chi=40)
    _check("u1", legs, 0, 1, vals, cutoff=0.2)


def test_rank_deficient_block():
    # every block has rank 1 (outer products): most singular values are 0,
    # the product is still exact and nothing fails to converge
    legs = [([-1, 0, 1], [4, 6, 3], 1), ([-1, 0, 1], [5, 2, 7], -1)]
    P = _P()
    S = P.Structure(P.U1, legs)
    rng = np.random.default_rng(23)
    vals = []
    for d1, d2 in ((4, 5), (6, 2), (3, 7)):
        vals.append(np.outer(rng.standard_normal(d1), rng.standard_normal(d2)).reshape(-1))
    vals = np.concatenate(vals)
    assert vals.size == S.numel
    _check("u1", legs, 0, 1, vals, chi=3)
    _check("u1", legs, 0, 1, vals)


def test_two_site_theta_full_size():
    # the two-site tensor theta[a, s1, s2, b] of the MPS workload (bond 2048
    # over charges -20..20), truncated back to chi = 2048
    P = _P()
    from paper_1203_2222_gb300 import synthetic
    w = synthetic.u1_two_site_svd()
    legs, total = w["theta"], 0
    S = P.Structure(P.U1, legs)
    vals = synthetic.normal(w["seed"], S.numel)
    _check("u1", legs, total, w["nrow"], vals, chi=w["chi"])


def test_large_blocks_every_sweep_order():
    # blocks of 320 x 320 (FP32 sweeps by column blocks, FP64 by pairs: the
    # FP64 block pair would exceed the shared memory), 450 x 330 and
    # 200 x 500 (more than 384 rows: every sweep by pairs, columns streamed),
    # 272 x 272 (both by column blocks) and 40 x 20 (by pairs: too few columns)
    legs = [([-2, -1, 0, 1], [40, 272, 320, 450], 1), ([-2, -1, 0, 1], [20, 272, 320, 330], -1)]
    vals = _rand("u1", legs, 0, 24)
    _check("u1", legs, 0, 1, vals)
    legs = [([0], [200], 1), ([0], [500], -1)]
    _check("u1", legs, 0, 1, _rand("u1", legs, 0, 25), chi=150)


def test_su2_rank4_through_fuse_and_split():
    # SU(2) above rank 2: fuse the row legs and the column legs (equal
    # directions within each group), decompose the rank-2 form, split the
    # factors' fused legs back.  The fusions are isometries, so the singular
    # values are those of T's dense matrix (rows = legs 0, 1), and U S V
    # rebuilds T.
    P = _P()
    sp = [0, 1, 2]
    legs = [(sp, [2, 3, 1], 1), (sp, [1, 2, 2], 1), (sp, [2, 1, 2], -1), ([0, 1, 2, 3], [1, 2, 1, 1], -1)]
    ol = [osu2.Leg(*l) for l in legs]
    vals = np.random.default_rng(43).standard_normal(osu2.layout(ol, osu2.left_comb(4))[2])
    S = P.Structure(P.SU2, legs)
    assert S.numel == vals.size
    T = P.SymTensor(S, torch.as_tensor(vals, dtype=torch.float64).cuda())
    F = P.fuse(P.fuse(T, 0), 1)
    plan = P.svd_plan(F.structure, 1)
    Sg = plan.execute(F.data).cpu().numpy()
    ks = [min(a, b) for a, b in zip(plan.m, plan.n)]
    offs = np.cumsum([0] + ks)
    Sd = np.sort(osvd.dense_values("su2", {x: Sg[o:o + k] for x, k, o in zip(plan.labels, ks, offs)}))[::-1]
    dense = osu2.embed(ol, osu2.left_comb(4), vals)
    sv = np.linalg.svd(dense.reshape(dense.shape[0] * dense.shape[1], -1), compute_uv=False)
    assert np.max(np.abs(sv[:len(Sd)] - Sd)) <= TOL * sv[0]
    assert np.all(sv[len(Sd):] <= TOL * sv[0])
    U, Sk, V = P.svd(F, 1, absorb=1)
    U4 = P.split(U, 0, [legs[0], legs[1]])
    V4 = P.split(V, 1, [legs[2], legs[3]])
    R = P.contract(U4, V4, [2], [0])
    torch.cuda.synchronize()
    Rl = [osu2.Leg(*l) for l in R.structure.legs]
    Rd = osu2.embed(Rl, R.structure.tree, R.data.detach().cpu().numpy())
    assert np.max(np.abs(Rd - dense)) <= TOL * sv[0]
    P.device_status()


@pytest.mark.parametrize("dirs", [(1, -1), (1, 1), (-1, -1), (-1, 1)])
def test_su2_rank2(dirs):
    # the block-diagonal form of Eq. svd0: integer and half-integer spins,
    # blocks 1 x 1 to 40 x 33 (tall and wide), every direction pattern
    legs = [([0, 1, 2, 3, 4], [3, 40, 7, 1, 12], dirs[0]), ([0, 1, 2, 3, 4], [5, 33, 7, 2, 1], dirs[1])]
    vals = _rand("su2", legs, 0, 41)
    _check("su2", legs, 0, 1, vals)
    _check("su2", legs, 0, 1, vals, chi=30)
