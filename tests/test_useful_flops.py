"""The bench's useful flops (the numerator of its TFLOP/s) equal an
independent count: for a U(1) or fermion-parity contraction, sum over the
matrix-form sectors x of 2 m_x n_x k_x, with m_x, k_x and n_x counted from
the legs alone (the free-leg and contracted-leg label tuples of A and B whose
fused label is x).  Planned with SYM_PLAN_DRYRUN=1 (no GPU)."""
import os
import subprocess
import sys

from tests.conftest import ROOT

SCRIPT = r'''
import itertools
from collections import defaultdict
import paper_1203_2222_gb300 as P
from paper_1203_2222_gb300 import synthetic

def extents(group, legs, idxs, sign):
    """{fused label x: sum over label tuples of these legs of prod d}."""
    out = defaultdict(int)
    for t in itertools.product(*[range(len(legs[i][0])) for i in idxs]):
        x, d = 0, 1
        for i, p in zip(idxs, t):
            lab, deg, dr = legs[i]
            x = (x ^ lab[p]) if group == "z2f" else x + sign * dr * lab[p]
            d *= deg[p]
        out[x] += d
    return out

def useful(group, la, QA, lb, QB, pa, pb):
    fa = [i for i in range(len(la)) if i not in pa]
    fb = [i for i in range(len(lb)) if i not in pb]
    # key x: charge of A's contracted legs as A sees them (= minus B's, by the opposite directions)
    kA = extents(group, la, pa, 1)
    # rows of A: free tuples whose complement charge lands on x
    rows = defaultdict(int)
    for t in itertools.product(*[range(len(la[i][0])) for i in fa]):
        y, d = 0, 1
        for i, p in zip(fa, t):
            lab, deg, dr = la[i]
            y = (y ^ lab[p]) if group == "z2f" else y + dr * lab[p]
            d *= deg[p]
        x = (QA ^ y) if group == "z2f" else QA - y
        rows[x] += d
    cols = defaultdict(int)
    for t in itertools.product(*[range(len(lb[i][0])) for i in fb]):
        y, d = 0, 1
        for i, p in zip(fb, t):
            lab, deg, dr = lb[i]
            y = (y ^ lab[p]) if group == "z2f" else y + dr * lab[p]
            d *= deg[p]
        x = (QB ^ y) if group == "z2f" else -(QB - y)
        cols[x] += d
    return sum(2.0 * rows[x] * kA[x] * cols[x] for x in kA if x in rows and x in cols)

for group, spec in (("u1", synthetic.u1_mps_heff()), ("z2f", synthetic.z2f_mps_heff())):
    g = P.U1 if group == "u1" else P.Z2F
    S = {n: P.Structure(g, spec[n]) for n in ("L", "A", "W", "R")}
    p1 = P.contract_plan(S["L"], S["A"], [2], [0], P.BF16X3)
    p2 = P.contract_plan(p1.out, S["W"], [1, 2], [0, 2], P.BF16X3)
    p3 = P.contract_plan(p2.out, S["R"], [1, 3], [2, 1], P.BF16X3)
    t1 = [tuple(l) for l in p1.out.legs]
    t2 = [tuple(l) for l in p2.out.legs]
    want = [useful(group, spec["L"], 0, spec["A"], 0, [2], [0]),
            useful(group, t1, 0, spec["W"], 0, [1, 2], [0, 2]),
            useful(group, t2, 0, spec["R"], 0, [1, 3], [2, 1])]
    got = [p.stats()["flops_fwd"] for p in (p1, p2, p3)]
    assert got == want, (group, got, want)
    print(group, [round(x / 1e9, 4) for x in got])
print("FLOPS OK")
'''


def test_useful_flops_match_an_independent_count():
    env = dict(os.environ, SYM_PLAN_DRYRUN="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "FLOPS OK" in r.stdout
