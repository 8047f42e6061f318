"""Plans of every GPU test case and workload, built and bounds-checked on the host.

Runs the planner in a subprocess with SYM_PLAN_DRYRUN=1: every work item's
largest source/destination offset is checked against its buffer before any
GPU sees the plan (no GPU needed)."""
import os
import subprocess
import sys

from tests.conftest import ROOT

SCRIPT = r'''
import numpy as np
import paper_1203_2222_gb300 as P
from paper_1203_2222_gb300 import synthetic
import tests.test_gpu_parity as T

def plan(group, la, lb, pa, pb, ta=None, tb=None, tree_c=None, QA=0, QB=0):
    g = P.U1 if group == "u1" else P.SU2
    A = P.Structure(g, la, total=QA, tree=ta); B = P.Structure(g, lb, total=QB, tree=tb)
    for prec in (P.FP64, P.BF16X3):
        p = P.contract_plan(A, B, pa, pb, prec, tree_c)
        st = p.stats()
        assert st["flops_fwd"] >= 0
    return st

c = synthetic.u1_pairwise(); plan("u1", c["A"], c["B"], c["pairsA"], c["pairsB"])
qs = [-1, 0, 1]
plan("u1", [(qs, [70, 150, 33], -1), (qs, [5, 9, 2], 1), (qs, [90, 140, 61], 1)],
     [(qs, [90, 140, 61], -1), (qs, [100, 131, 7], 1)], [2], [0])
s = synthetic.su2_recouple(dmax=3, jmax2=4)
for ti in T.SU2_TREES:
    plan("su2", s["A"], s["B"], s["pairsA"], s["pairsB"], ta=ti)
sp = [0, 1, 2, 3]
la = [(sp, [2, 1, 2, 1], -1), (sp, [1, 2, 1, 1], 1), (sp, [2, 2, 1, 1], -1), (sp, [1, 1, 2, 1], 1)]
lb = [(sp, [1, 2, 1, 1], -1), (sp, [2, 2, 1, 1], 1), (sp, [1, 1, 1, 2], 1)]
plan("su2", la, lb, [1, 2], [0, 1], ta=[(1, 2), (0, 4), (5, 3)])
plan("su2", la, lb, [1, 2], [0, 1], tree_c=[(1, 2), (0, 3)])
a = [(sp, [2, 1, 1, 1], 1), (sp, [1, 2, 1, 1], 1)]; b = [(sp, [2, 1, 1, 1], -1), (sp, [1, 2, 1, 1], -1)]
plan("su2", a, b, [0, 1], [0, 1])
m = synthetic.u1_mps_heff()
Ls = [P.Structure(P.U1, m[n]) for n in ("L", "A", "W", "R")]
t1 = P.contract_plan(Ls[0], Ls[1], [2], [0], P.BF16X3)
t2 = P.contract_plan(t1.out, Ls[2], [1, 2], [0, 2], P.BF16X3)
t3 = P.contract_plan(t2.out, Ls[3], [1, 3], [2, 1], P.BF16X3)
print("MPS flops", t1.stats()["flops_fwd"] + t2.stats()["flops_fwd"] + t3.stats()["flops_fwd"])
# the MPO step: every sector has B's matrix at most 4 x 4 and is contracted
# directly on the blocks, unless SYM_DIRECT_MAX=0 sends it through the GEMMs
import os
direct = os.environ.get("SYM_DIRECT_MAX") != "0"
assert (len(t2.gemm_shapes()) == 0) == direct, len(t2.gemm_shapes())
assert len(t1.gemm_shapes()) > 0 and len(t3.gemm_shapes()) > 0
bond_in, bond_out = (T.MPO[0], T.MPO[1], -1), (T.MPO[0], T.MPO[1], 1)
qs5 = [-2, -1, 0, 1, 2]
plan("u1", [(qs5, [7, 19, 33, 21, 5], -1), (*T.MPO, -1), (*T.PHYS, -1), (qs5, [6, 17, 40, 23, 9], 1)],
     [(*T.MPO, 1), (*T.PHYS, -1), (*T.PHYS, 1), (*T.MPO, -1)], [1, 2], [0, 2])
plan("u1", [(qs5, [4, 11, 20, 9, 3], -1), (*T.PHYS, -1), (qs5, [5, 13, 17, 12, 6], 1), (*T.PHYS, 1), (*T.MPO, 1)],
     [(*T.MPO, -1), (*T.PHYS, 1), (*T.PHYS, 1), (*T.MPO, 1)], [1, 4], [2, 0], QA=1)
plan("u1", [([-1, 0, 1, 2], [37, 64, 129, 3], 1), ([-1, 0, 1], [1, 2, 1], -1)],
     [([-1, 0, 1], [1, 2, 1], 1), ([0, 2], [1, 2], 1)], [1], [0], QB=1)
# fermion parity: permutation swap signs on the gathers
def zplan(la, lb, pa, pb, QA=0, QB=0):
    A = P.Structure(P.Z2F, la, total=QA); B = P.Structure(P.Z2F, lb, total=QB)
    for prec in (P.FP64, P.BF16X3):
        P.contract_plan(A, B, pa, pb, prec)
zplan([([0, 1], [23, 17], 1), ([0, 1], [9, 14], -1), ([0, 1], [30, 11], 1), ([0, 1], [12, 19], 1)],
      [([0, 1], [12, 19], -1), ([0, 1], [40, 25], 1), ([0, 1], [9, 14], 1)], [3, 1], [0, 2], QA=1)
Z = P.Structure(P.Z2F, [([0, 1], [2, 3], 1), ([0, 1], [3, 1], 1), ([0, 1], [1, 2], -1)], total=1)
P.permute_plan(Z, [2, 0, 1]); P.fuse_plan(Z, 0)
try:
    P.Structure(P.Z2F, [([0, 2], [1, 1], 1)])
    raise SystemExit("accepted a parity label 2")
except P.SymError:
    pass
b5 = synthetic.u1_two_site_batch(n=6, seed=7, dmin=40, dmax=90, qmax=4)
pr = b5["problems"]
S5 = {n: [P.Structure(P.U1, q[n]) for q in pr] for n in ("L", "theta", "W", "R")}
cur = S5["L"]
for an, bn, pa, pb in b5["steps"]:
    bp = P.contract_batch_plan(cur if an is None else S5[an], S5[bn], pa, pb, P.BF16X3)
    cur = bp.outs
# transforms
U = P.Structure(P.U1, [(qs, [2, 3, 1], 1), (qs, [1, 2, 2], 1), (qs, [3, 1, 2], -1)])
P.permute_plan(U, [2, 0, 1]); f = P.fuse_plan(U, 0); P.split_plan(f.out, 0, [U.legs[0], U.legs[1]])
S = P.Structure(P.SU2, [([0, 1, 2], [2, 1, 1], 1), ([0, 1, 2], [1, 2, 1], 1), ([0, 1, 2, 3, 4], [1, 1, 2, 1, 1], 1)])
P.permute_plan(S, [2, 0, 1]); f = P.fuse_plan(S, 0); P.split_plan(f.out, 0, [S.legs[0], S.legs[1]])
# SU(2) transforms with fused recoupling items: blocks of many positions, the
# permute into the matrix tree, inner-leg fuses (the destination's fused-leg
# dimension as its row stride) and the splits back
sp3 = [0, 1, 2]
for legs in ([(sp3, [12, 9, 7], 1), (sp3, [9, 7, 12], -1), (sp3, [7, 12, 9], -1), (sp3, [12, 7, 9], -1)],
             [([3, 4], [6, 5], 1), ([2, 3, 4], [3, 6, 4], 1), ([3, 4], [5, 6], 1), ([2, 4], [6, 5], 1)]):
    S4 = P.Structure(P.SU2, legs)
    P.permute_plan(S4, [0, 2, 1, 3], [(0, 1), (2, 3), (4, 5)])
    P.permute_plan(S4, [3, 1, 0, 2])
    for f in (1, 2):
        fp = P.fuse_plan(S4, f)
        P.split_plan(fp.out, f, [legs[f], legs[f + 1]])
# a large recoupling permute (items of up to 2048 positions) and the
# contraction whose gather recouples the same tensor
c3 = synthetic.su2_recouple(dmax=12, jmax2=8)
A3, B3 = P.Structure(P.SU2, c3["A"]), P.Structure(P.SU2, c3["B"])
P.permute_plan(A3, [0, 2, 1, 3], [(0, 1), (2, 3), (4, 5)])
for prec in (P.FP64, P.BF16X3):
    P.contract_plan(A3, B3, c3["pairsA"], c3["pairsB"], prec)
try:
    P.contract(None, None, [], [])
except Exception:
    pass
print("DRYRUN OK")
'''


import pytest  # noqa: E402


@pytest.mark.parametrize("direct", ["default", "off"])
def test_all_plans_bounds_check_on_host(direct):
    env = dict(os.environ, SYM_PLAN_DRYRUN="1", PYTHONPATH=ROOT)
    env.pop("SYM_DIRECT_MAX", None)
    if direct == "off":
        env["SYM_DIRECT_MAX"] = "0"
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "DRYRUN OK" in r.stdout
