"""Host side of the blockwise SVD (include/symtensor.h, sym_svd_*): the
diagonal blocks the planner finds, the truncation rule and the structures of
U and V, each against the oracle (oracle/svd.py), planned with
SYM_PLAN_DRYRUN=1 (no GPU); and the argument errors."""
import os
import subprocess
import sys

from tests.conftest import ROOT

SCRIPT = r'''
import numpy as np
import paper_1203_2222_gb300 as P
from oracle import svd as osvd, u1, z2f

def legs_u1():
    return [([-1, 0, 1], [2, 3, 1], 1), ([0, 1], [2, 2], 1), ([-1, 0, 2], [1, 2, 2], -1), ([0, 1], [1, 3], -1)]

def legs_z2f():
    return [([0, 1], [3, 2], 1), ([0, 1], [1, 2], -1), ([0, 1], [2, 3], 1)]

def oracle_tensor(group, legs, total):
    m = u1 if group == "u1" else z2f
    L = [m.Leg(*l) for l in legs]
    return (L, total, np.random.default_rng(1).standard_normal(m.layout(L, total)[2]))

cases = [("u1", P.U1, legs_u1(), 0, 2), ("u1", P.U1, legs_u1(), 1, 1), ("u1", P.U1, legs_u1(), -1, 3),
         ("z2f", P.Z2F, legs_z2f(), 0, 1), ("z2f", P.Z2F, legs_z2f(), 1, 2)]
for gname, g, legs, total, nrow in cases:
    S = P.Structure(g, legs, total=total)
    plan = P.SVDPlan(S, nrow)
    T = oracle_tensor(gname, legs, total)
    fac, bd = osvd.svd(gname, T, nrow)
    assert plan.labels == sorted(bd), (plan.labels, sorted(bd))
    assert plan.m == [bd[x][0].shape[0] for x in plan.labels]
    assert plan.n == [bd[x][0].shape[1] for x in plan.labels]
    assert plan.nsv == sum(min(a, b) for a, b in zip(plan.m, plan.n))
    # truncation: the library's rule on the oracle's singular values
    Sx = {x: fac[x][1] for x in plan.labels}
    flat = np.concatenate([Sx[x] for x in plan.labels])
    for chi, cut in ((None, 0.0), (1, 0.0), (5, 0.0), (plan.nsv // 2, 0.0), (None, 0.3), (4, 0.1), (0, 0.0)):
        keep = plan.truncation(flat, chi, cut)
        ko = osvd.truncation(Sx, chi, cut)
        assert keep == [ko[x] for x in plan.labels], (chi, cut, keep, ko)
    # U and V structures against the oracle's recast factors
    keep = plan.truncation(flat, max(plan.nsv // 2, 1))
    Us, Vs = plan.bond(keep)
    U, kept, V = osvd.factors(gname, T, nrow, {x: k for x, k in zip(plan.labels, keep)})
    for st, (lg, tot, d) in ((Us, U), (Vs, V)):
        assert st.total == tot and st.numel == d.size
        assert [tuple(l[0]) for l in st.legs] == [tuple(l.labels) for l in lg]
        assert [tuple(l[1]) for l in st.legs] == [tuple(l.degens) for l in lg]
        assert [l[2] for l in st.legs] == [l.dir for l in lg]

# ties between blocks: smaller label first; within a block, its own order
S = P.Structure(P.U1, [([-1, 0, 1], [2, 2, 2], 1), ([-1, 0, 1], [2, 2, 2], -1)])
plan = P.SVDPlan(S, 1)
vals = np.array([3.0, 1.0, 3.0, 2.0, 3.0, 1.0])
assert plan.truncation(vals, 2) == [1, 1, 0]
assert plan.truncation(vals, 3) == [1, 1, 1]
assert plan.truncation(vals, 4) == [1, 2, 1]
assert plan.truncation(vals, 5) == [2, 2, 1]
assert plan.truncation(vals, None, 0.5) == [1, 2, 1]

def rejects(code, f):
    try:
        f()
    except P.SymError as e:
        assert e.code == code, (e.code, code)
        return
    raise SystemExit("accepted")

from paper_1203_2222_gb300 import _lib as L
rejects(L.SYM_ERR_UNSUPPORTED, lambda: P.SVDPlan(P.Structure(P.SU2, [([0, 2], [1, 1], 1)] * 3), 1))

# SU(2) rank 2: blocks per spin, truncation by dense count (2j+1 per value)
from oracle import su2
legs2 = [([0, 1, 2, 3], [3, 2, 4, 2], 1), ([0, 1, 2, 3], [2, 3, 3, 1], -1)]
S2 = P.Structure(P.SU2, legs2)
plan2 = P.SVDPlan(S2, 1)
L2 = [su2.Leg(*l) for l in legs2]
T2 = (L2, su2.left_comb(2), np.random.default_rng(3).standard_normal(su2.layout(L2, su2.left_comb(2))[2]))
fac2, bd2 = osvd.svd("su2", T2, 1)
assert plan2.labels == sorted(bd2) and plan2.m == [3, 2, 4, 2] and plan2.n == [2, 3, 3, 1]
Sx2 = {x: fac2[x][1] for x in plan2.labels}
flat2 = np.concatenate([Sx2[x] for x in plan2.labels])
for chi in (None, 1, 2, 5, 9, 13, 20):
    keep = plan2.truncation(flat2, chi)
    ko = osvd.truncation(Sx2, chi, group="su2")
    assert keep == [ko[x] for x in plan2.labels], (chi, keep, ko)
Us2, Vs2 = plan2.bond(plan2.truncation(flat2, 9))
assert [l[2] for l in Us2.legs] == [1, -1] and [l[2] for l in Vs2.legs] == [1, -1]
rejects(L.SYM_ERR_ARG, lambda: P.SVDPlan(S, 0))
rejects(L.SYM_ERR_ARG, lambda: P.SVDPlan(S, 2))
rejects(L.SYM_ERR_ARG, lambda: plan.bond([0, 0, 0]))
rejects(L.SYM_ERR_ARG, lambda: plan.bond([1, 3, 0]))
rejects(L.SYM_ERR_NUMERIC, lambda: plan.truncation(np.array([1.0, np.nan, 1, 1, 1, 1])))
rejects(L.SYM_ERR_UNSUPPORTED, lambda: L.check(L.lib.sym_svd_execute(plan._h, 1, 1, None)))
print("SVD HOST OK")
'''


def test_svd_host_planning_matches_the_oracle():
    env = dict(os.environ, SYM_PLAN_DRYRUN="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "SVD HOST OK" in r.stdout
