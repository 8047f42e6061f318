"""Planning parameters (include/symtensor.h, sym_tune): the C-ABI round trip,
range checks, the epoch, and that plans built afterwards follow them (host
planning with SYM_PLAN_DRYRUN=1, no GPU)."""
import os
import subprocess
import sys

from tests.conftest import ROOT

SCRIPT = r'''
import paper_1203_2222_gb300 as P
from paper_1203_2222_gb300 import synthetic
d = P.tune_get()
assert d == {"tc_min_mn": 64, "tc_min_k": 48, "tc_max_k": 16384, "direct_max": 4, "direct_chunk": 1024,
             "rows_spans": 8, "splitk_ctas": 2, "thin_slice": 4096, "tc_order": 0, "tc_group": 8,
             "direct_mixed": 1, "tc_all": 0}, d
e0 = P.tune_epoch()
for bad in ({"direct_max": 5}, {"direct_chunk": 100}, {"tc_max_k": 10}, {"thin_slice": 100}, {"tc_order": 2},
            {"rows_spans": 0}, {"tc_group": -1}, {"direct_mixed": 2}, {"tc_all": 3}):
    try:
        P.tune_set(**bad)
        raise SystemExit(f"accepted {bad}")
    except P.SymError:
        pass
assert P.tune_get() == d and P.tune_epoch() == e0
try:
    P.tune_set(no_such_parameter=1)
    raise SystemExit("accepted an unknown name")
except KeyError:
    pass
m = synthetic.u1_mps_heff()
S = {n: P.Structure(P.U1, m[n]) for n in ("L", "A", "W", "R")}
def kinds():
    t1 = P.contract_plan(S["L"], S["A"], [2], [0], P.BF16X3)
    t2 = P.contract_plan(t1.out, S["W"], [1, 2], [0, 2], P.BF16X3)
    k1 = [x[3] for x in t1.gemm_shapes()]
    return k1.count(0), len(k1), len(t2.gemm_shapes())
tc0, n0, w0 = kinds()
assert w0 == 0  # the MPO step is direct
P.tune_set(tc_min_mn=16, tc_min_k=16)
assert P.tune_epoch() == e0 + 1
tc1, n1, w1 = kinds()
assert n1 == n0 and tc1 > tc0, (tc0, tc1)  # narrower sectors moved onto the tensor cores
P.tune_set(direct_max=0)
assert kinds()[2] > 0  # the MPO step back on the GEMMs
P.tune_set(direct_max=4, direct_mixed=0)
k2 = kinds()
assert k2[2] == 0 and k2[1] >= n0  # the all-direct MPO step stays direct; mixed plans keep every sector on GEMMs
P.tune_set(direct_max=0, tc_all=1)
k3 = kinds()
assert k3[0] == k3[1] > 0  # every GEMM of L.A on the tensor cores
P.tune_set(**d)
assert kinds() == (tc0, n0, w0)
print("TUNE OK")
'''


def test_tune_parameters_round_trip_and_drive_planning():
    env = dict(os.environ, SYM_PLAN_DRYRUN="1", PYTHONPATH=ROOT)
    for k in ("SYM_TUNE", "SYM_DIRECT_MAX", "SYM_TC_MIN_MN", "SYM_TC_MIN_K", "SYM_TC_MAX_K"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "TUNE OK" in r.stdout


def test_tune_environment_seeds_the_parameters():
    env = dict(os.environ, SYM_PLAN_DRYRUN="1", PYTHONPATH=ROOT, SYM_TUNE="direct_chunk=256,tc_order=1",
               SYM_TC_MIN_MN="32")
    code = "import paper_1203_2222_gb300 as P; t = P.tune_get(); print(t['direct_chunk'], t['tc_order'], t['tc_min_mn'])"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == ["256", "1", "32"]


def test_autotune_table_round_trip(tmp_path):
    from paper_1203_2222_gb300 import autotune
    path = str(tmp_path / "tuned.json")
    assert autotune.load("w", path, device="dev") is None
    p = {"tc_min_mn": 32, "tc_order": 1}
    autotune.save("w", p, 1.5, 2.0, 7, path=path, device="dev")
    autotune.save("other", {"tc_min_mn": 64}, 1.0, 1.0, 1, path=path, device="dev")
    assert autotune.load("w", path, device="dev") == p
    assert autotune.load("w", path, device="another device") is None


CHECK_SCRIPT = r'''
import paper_1203_2222_gb300 as P
from paper_1203_2222_gb300 import autotune

# timing stand-in: tc_all = 1 would be the fastest point, a lower tc_min_mn next
def fake_time(step, reps, warmup, trials, graph=True):
    t = P.tune_get()
    return 1.0 - 0.5 * t["tc_all"] - 0.001 * (64 - t["tc_min_mn"])

autotune.time_step = fake_time
space = {"tc_all": [0, 1], "tc_min_mn": [16, 64]}
base = dict(P.tune_get(), tc_all=0, tc_min_mn=64)
# without a check the descent takes tc_all = 1
params, ms, hist = autotune.tune(lambda: None, space=space, start=base, starts=())
assert params["tc_all"] == 1, params
# a check that rejects tc_all = 1 (as an accuracy bar would) keeps it off
params, ms, hist = autotune.tune(lambda: None, space=space, start=base, starts=(),
                                 check=lambda: P.tune_get()["tc_all"] == 0)
assert params["tc_all"] == 0 and params["tc_min_mn"] == 16, params
assert any(h.get("accurate") is False for h in hist)
assert P.tune_get()["tc_all"] == 0
print("CHECK OK")
'''


def test_search_rejects_candidates_the_accuracy_check_refuses():
    env = dict(os.environ, SYM_PLAN_DRYRUN="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHECK_SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "CHECK OK" in r.stdout
