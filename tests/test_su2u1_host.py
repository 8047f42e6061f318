"""SU(2) x U(1) structure on the host (include/symtensor.h, SYM_SU2U1): the
sector tables equal the oracle's (oracle/su2u1.py) bit for bit, and the
contraction, permute, fuse and split plans build and bounds-check their work
lists with SYM_PLAN_DRYRUN=1 (no GPU), their result structures equal the
oracle's."""
import os
import subprocess
import sys

from tests.conftest import ROOT

SCRIPT = r'''
import numpy as np
import paper_1203_2222_gb300 as P
from oracle import contract as oc, su2, su2u1 as m

CQ = [(-1, 1), (0, 0), (0, 2), (1, 1), (2, 0)]
legs = [(CQ, [2, 1, 2, 1, 1], 1), (CQ, [1, 2, 1, 2, 1], -1), (CQ, [2, 2, 1, 1, 2], 1), (CQ, [1, 1, 2, 1, 1], -1)]
for Q in (-2, 0, 2):
    for tree in (None, [(1, 2), (0, 4), (5, 3)], [(0, 1), (2, 3), (4, 5)]):
        S = P.Structure(P.SU2U1, legs, total=Q, tree=tree)
        t = su2.left_comb(4) if tree is None else tree
        secs, offs, n = m.layout([m.Leg(*l) for l in legs], (t, Q))
        lab, off = S.sectors()
        assert S.numel == n and S.nsec == len(secs)
        for i, (pos, inner) in enumerate(secs):
            assert tuple(lab[i][:4]) == pos and tuple(lab[i][4:]) == tuple(inner)
            assert off[i] == offs[i]
        assert [tuple(l[0]) for l in S.legs] == [tuple(CQ)] * 4

lb = [(CQ, [2, 2, 1, 1, 2], -1), (CQ, [1, 1, 2, 1, 1], 1), (CQ, [2, 1, 1, 2, 1], 1)]
for QA, QB, ta, tc in ((2, -2, None, None), (0, 0, [(1, 2), (0, 4), (5, 3)], None), (2, 0, None, [(1, 2), (0, 3)])):
    for prec in (P.FP64, P.BF16X3):
        SA = P.Structure(P.SU2U1, legs, total=QA, tree=ta)
        SB = P.Structure(P.SU2U1, lb, total=QB)
        plan = P.contract_plan(SA, SB, [2, 3], [0, 1], prec, tc)
        A = ([m.Leg(*l) for l in legs], (SA.tree, QA), np.zeros(SA.numel))
        B = ([m.Leg(*l) for l in lb], (SB.tree, QB), np.zeros(SB.numel))
        lc, tcc, c, _ = oc.contract("su2u1", A, B, [2, 3], [0, 1], tree_c=plan.out.tree)
        assert plan.out.numel == c.size and plan.out.total == tcc[1] == QA + QB
        assert [tuple(l.labels) for l in lc] == [tuple(l[0]) for l in plan.out.legs]

S = P.Structure(P.SU2U1, legs, total=2)
assert P.permute_plan(S, [2, 0, 3, 1], None, P.FP64).out.numel > 0
for l3 in ([(CQ, [2, 1, 1, 1, 1], 1), (CQ, [1, 2, 1, 1, 2], 1), (CQ, [1, 1, 2, 1, 1], -1)],
           [(CQ, [2, 1, 1, 1, 1], -1), (CQ, [1, 2, 1, 1, 2], -1), (CQ, [1, 1, 2, 1, 1], 1)]):
    for total in (0, 2):
        S = P.Structure(P.SU2U1, l3, total=total)
        fp = P.fuse_plan(S, 0, P.FP64)
        T = ([m.Leg(*l) for l in l3], (su2.left_comb(3), total), np.zeros(S.numel))
        lo, to, ref, _ = oc.fuse("su2u1", T, 0)
        assert [tuple(l.labels) for l in lo] == [tuple(l[0]) for l in fp.out.legs]
        assert [tuple(l.degens) for l in lo] == [tuple(l[1]) for l in fp.out.legs]
        assert fp.out.numel == ref.size
        assert P.split_plan(fp.out, 0, [l3[0], l3[1]], P.FP64).out.numel == S.numel

# a batch of composite contractions is one plan; each problem's result
# structure equals its single plan's
As = [P.Structure(P.SU2U1, legs, total=q) for q in (0, 2, -2)]
Bs = [P.Structure(P.SU2U1, lb, total=q) for q in (0, -2, 2)]
bp = P.contract_batch_plan(As, Bs, [2, 3], [0, 1], P.BF16X3)
for a, b, o in zip(As, Bs, bp.outs):
    single = P.contract_plan(a, b, [2, 3], [0, 1], P.BF16X3).out
    assert o.numel == single.numel and o.total == single.total and o.legs == single.legs

# the bench's composite MPS chain: every plan builds, results have the oracle's legs
from paper_1203_2222_gb300 import synthetic
ms = synthetic.su2u1_mps_heff()
Sm = {n: P.Structure(P.SU2U1, ms[n]) for n in ("L", "A", "W", "R")}
cur_s, cur_o = Sm["L"], ([m.Leg(*l) for l in ms["L"]], (su2.left_comb(3), 0), None)
for bn, pa, pb in (("A", [2], [0]), ("W", [1, 2], [0, 2]), ("R", [1, 3], [2, 1])):
    plan = P.contract_plan(cur_s, Sm[bn], pa, pb, P.BF16X3)
    lc = oc.result_legs(cur_o[0], [m.Leg(*l) for l in ms[bn]], pa, pb)
    assert [tuple(l.labels) for l in lc] == [tuple(l[0]) for l in plan.out.legs]
    assert plan.stats()["flops_fwd"] > 0
    cur_s, cur_o = plan.out, (lc, None, None)
assert cur_s.numel == Sm["A"].numel  # Y has A's legs

try:
    P.SVDPlan(P.Structure(P.SU2U1, legs[:2] + [(CQ, [1] * 5, 1)], total=0), 1)
    raise SystemExit("SVD of a composite tensor accepted")
except P.SymError as e:
    assert e.code == -7
print("SU2U1 HOST OK")
'''


def test_su2u1_structure_and_plans_match_the_oracle():
    env = dict(os.environ, SYM_PLAN_DRYRUN="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "SU2U1 HOST OK" in r.stdout
