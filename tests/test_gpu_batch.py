"""Batched contraction: many independent two-site effective-Hamiltonian applies as one plan.

Problem i's tensors sit in packed buffers at the batch plan's offsets; every
phase of every problem runs in one launch per kernel.  Checks:
  * a small batch, each problem's whole chain Y = (((L.theta).W1).W2).R and
    the gradients of <G, Y> (chained through the oracle's contract_grad),
    against the FP64 oracle, in FP64 and split-BF16;
  * the full 512-problem batch: sampled problems' results equal the same
    contraction planned and run alone (FP64), and the smallest problems
    match the oracle.
"""
import numpy as np
import pytest

import graph_replay

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 2e-5}
STREAMS = {"L": 1, "theta": 2, "W": 3, "R": 4}  # random sub-stream of each tensor role


def _rel(x, y):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300))


def _batch(P, spec, dtype, names=("L", "theta", "W", "R")):
    """Structures, batch plans of the four steps and packed seeded inputs."""
    from paper_1203_2222_gb300 import synthetic
    pr = spec["problems"]
    S = {n: [P.Structure(P.U1, p[n]) for p in pr] for n in names}
    prec = P.FP64 if dtype == torch.float64 else P.BF16X3
    plans, cur = [], S["L"]
    for an, bn, pa, pb in spec["steps"]:
        bp = P.contract_batch_plan(cur if an is None else S[an], S[bn], pa, pb, prec)
        plans.append(bp)
        cur = bp.outs
    offs = {"L": plans[0].off_a, "theta": plans[0].off_b, "W": plans[1].off_b, "R": plans[3].off_b}
    data = {}
    for n in names:
        parts = [synthetic.normal(p["seed"], offs[n][i + 1] - offs[n][i], stream=STREAMS[n])
                 for i, p in enumerate(pr)]
        data[n] = torch.as_tensor(np.concatenate(parts)).to(dtype).cuda().requires_grad_(True)
    return S, plans, offs, data


def _chain(P, plans, data):
    t1 = P.contract_batch(plans[0], data["L"], data["theta"])
    t2 = P.contract_batch(plans[1], t1, data["W"])
    t3 = P.contract_batch(plans[2], t2, data["W"])
    return P.contract_batch(plans[3], t3, data["R"])


def _oracle_chain(spec, i, host):
    """Y and the gradients of <G, Y> of problem i with the FP64 oracle."""
    from oracle import contract as oc
    from oracle import u1
    p = spec["problems"][i]
    legs = {n: [u1.Leg(*l) for l in p[n]] for n in ("L", "theta", "W", "R")}
    ins, cur = [], (legs["L"], 0, host["L"])
    for an, bn, pa, pb in spec["steps"]:
        a = cur if an is None else (legs[an], 0, host[an])
        b = (legs[bn], 0, host[bn])
        lc, qc, c, _ = oc.contract("u1", a, b, pa, pb)
        ins.append((a, b, pa, pb))
        cur = (lc, qc, c)
    return ins, cur


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["float64", "float32"])
def test_small_batch_chain_and_gradients_against_oracle(dtype):
    import paper_1203_2222_gb300 as P
    from oracle import contract as oc
    from paper_1203_2222_gb300 import synthetic
    spec = synthetic.u1_two_site_batch(n=5, seed=7, dmin=40, dmax=90, qmax=4)
    S, plans, offs, data = _batch(P, spec, dtype)
    Y = _chain(P, plans, data)
    G = torch.as_tensor(np.random.default_rng(3).standard_normal(Y.numel())).to(dtype).cuda()
    grads = torch.autograd.grad(Y, [data[n] for n in ("L", "theta", "W", "R")], grad_outputs=G)
    torch.cuda.synchronize()
    yh, gh = Y.detach().double().cpu().numpy(), G.double().cpu().numpy()
    gr = {n: g.double().cpu().numpy() for n, g in zip(("L", "theta", "W", "R"), grads)}
    for i in range(len(spec["problems"])):
        sl = {n: slice(offs[n][i], offs[n][i + 1]) for n in offs}
        host = {n: data[n].detach().double().cpu().numpy()[sl[n]] for n in offs}
        ins, (_, _, y_ref) = _oracle_chain(spec, i, host)
        ys = slice(plans[3].off_c[i], plans[3].off_c[i + 1])
        assert _rel(yh[ys], y_ref) <= TOL[dtype]
        # backward through the chain with the oracle's adjoint of every step
        dc, ref = gh[ys], {"W": 0.0}
        for k in range(3, -1, -1):
            a, b, pa, pb = ins[k]
            da, db, _ = oc.contract_grad("u1", a, b, pa, pb, dc)
            name_b = spec["steps"][k][1]
            ref[name_b] = ref.get(name_b, 0.0) + db if name_b == "W" else db
            dc = da
        ref["L"] = dc
        for n in ("L", "theta", "W", "R"):
            assert _rel(gr[n][sl[n]], ref[n]) <= TOL[dtype], (i, n)
    P.device_status()


def test_full_batch_matches_single_plans_and_oracle():
    import paper_1203_2222_gb300 as P
    from oracle import contract as oc
    from oracle import u1
    from paper_1203_2222_gb300 import synthetic
    spec = synthetic.u1_two_site_batch()
    S, plans, offs, data = _batch(P, spec, torch.float64)
    with torch.no_grad():
        t1 = P.contract_batch(plans[0], data["L"], data["theta"])
    torch.cuda.synchronize()
    pr = spec["problems"]
    order = np.argsort([p["D"] for p in pr])
    sample = list(order[:3]) + list(order[-2:]) + [len(pr) // 2]
    for i in sample:
        la = slice(offs["L"][i], offs["L"][i + 1])
        th = slice(offs["theta"][i], offs["theta"][i + 1])
        single = P.contract(P.SymTensor(S["L"][i], data["L"].detach()[la]),
                            P.SymTensor(S["theta"][i], data["theta"].detach()[th]), [2], [0])
        got = t1[plans[0].off_c[i]:plans[0].off_c[i + 1]]
        assert torch.allclose(got, single.data, rtol=1e-12, atol=1e-12), i
    for i in order[:2]:  # the smallest problems against the oracle
        p = pr[i]
        la = slice(offs["L"][i], offs["L"][i + 1])
        th = slice(offs["theta"][i], offs["theta"][i + 1])
        a = ([u1.Leg(*l) for l in p["L"]], 0, data["L"].detach()[la].cpu().numpy())
        b = ([u1.Leg(*l) for l in p["theta"]], 0, data["theta"].detach()[th].cpu().numpy())
        _, _, c_ref, _ = oc.contract("u1", a, b, [2], [0])
        got = t1[plans[0].off_c[i]:plans[0].off_c[i + 1]].cpu().numpy()
        assert _rel(got, c_ref) <= 1e-12
    P.device_status()


def test_full_batch_bf16x3_chain_and_gradients_against_oracle():
    """The bench's batched step at full size (512 problems, split-BF16 x3):
    the whole four-contraction chain forward and the gradients of <G, Y>,
    replayed from a CUDA graph as the bench times it,
    with respect to L, theta, W (both uses) and R, for the three smallest
    problems, a stratified sample across the bond dimension (the problems
    at the 20/40/60/80% quantiles of D) and the largest, against the FP64
    oracle's dense chain and its adjoint step by step."""
    import paper_1203_2222_gb300 as P
    from oracle import contract as oc
    from paper_1203_2222_gb300 import synthetic
    spec = synthetic.u1_two_site_batch()
    S, plans, offs, data = _batch(P, spec, torch.float32)
    G = torch.as_tensor(synthetic.normal(4243, plans[3].off_c[-1])).to(torch.float32).cuda()
    names = ("L", "theta", "W", "R")

    def step():
        Y = _chain(P, plans, data)
        return (Y,) + tuple(torch.autograd.grad(Y, [data[n] for n in names], grad_outputs=G))

    # the bench's launch configuration: the autograd step replayed from a CUDA graph
    (Y, *grads), graph = graph_replay.replay(step)
    P.device_status()
    yh, gh = Y.detach().double().cpu().numpy(), G.double().cpu().numpy()
    gr = {n: g.double().cpu().numpy() for n, g in zip(names, grads)}
    dh = {n: data[n].detach().double().cpu().numpy() for n in names}
    pr = spec["problems"]
    order = list(np.argsort([p["D"] for p in pr], kind="stable"))
    n = len(order)
    sample = order[:3] + [order[int(q * (n - 1))] for q in (0.2, 0.4, 0.6, 0.8)] + [order[-1]]
    for i in sample:
        sl = {k: slice(offs[k][i], offs[k][i + 1]) for k in offs}
        host = {k: dh[k][sl[k]] for k in offs}
        ins, (_, _, y_ref) = _oracle_chain(spec, i, host)
        ys = slice(plans[3].off_c[i], plans[3].off_c[i + 1])
        assert _rel(yh[ys], y_ref) <= 2e-5, (i, pr[i]["D"])
        dc, ref = gh[ys], {}
        for k in range(3, -1, -1):
            a, b, pa, pb = ins[k]
            da, db, _ = oc.contract_grad("u1", a, b, pa, pb, dc)
            nb = spec["steps"][k][1]
            ref[nb] = ref.get(nb, 0.0) + db
            dc = da
        ref["L"] = dc
        for k in names:
            assert _rel(gr[k][sl[k]], ref[k]) <= 2e-5, (i, pr[i]["D"], k)
