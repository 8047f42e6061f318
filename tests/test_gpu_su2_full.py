"""SU(2) recoupling contraction at full size: forward and backward checked
against the oracle on sampled dense elements.

The workload of the large-sector configuration: rank-4 SU(2) tensors whose
legs carry 2j = 0..8 with degeneracies drawn in 1..32, A in the comb tree,
its legs 1 and 3 contracted with the dual legs of B (the gather recouples A
into the matrix tree by 6j coefficients).  At this size (A: 7.5e8 block
entries, 1.3e13 useful flops per forward) the dense oracle cannot embed the
tensors, so the test draws dense elements of C = contract(A, B) and of the
gradients dA, dB of <G, C>, lets the oracle compute each one from slices of
the embedded inputs (oracle.sample), and embeds the GPU's result blocks at
the same indices.  The full-size split-BF16 step runs as the bench times
it: the autograd step captured in a CUDA graph and replayed.  Elements are
drawn with J_z conserved (so none is a
structural zero), at least 16 in every matrix-form sector of C (coupled spin
2e = 0..16) plus the largest block of each result, and at least 256 per
result.  The oracle's elements run in a pool of spawned host processes that
read the tensors from memory-mapped files.

Inputs are N(0,1) draws of a seeded torch generator on the device.
"""
import os
import shutil
import tempfile

import numpy as np
import pytest

import graph_replay
import oracle_pool

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

def _tasks(c, dmax, per_e, per_tensor, seed):
    """Sampled indices: C stratified by its matrix-form sector (coupled spin
    e), dA and dB uniform over their sectors, plus the largest block of each."""
    from oracle import contract as oc
    from oracle import sample, su2
    la = [su2.Leg(*l) for l in c["A"]]
    lb = [su2.Leg(*l) for l in c["B"]]
    lc = oc.result_legs(la, lb, c["pairsA"], c["pairsB"])
    comb, nodes_c = su2.left_comb(4), oc.comb_pair_tree(2, 2)
    rng = np.random.default_rng(seed)
    tasks = []
    secs_c = su2.layout(lc, nodes_c)[0]
    by_e = {}
    for s in secs_c:
        by_e.setdefault(s[1][0], []).append(s)  # the node spin of legs (0, 1) = that of (2, 3)
    assert sorted(by_e) == list(range(0, 17)), sorted(by_e)
    for e, secs in sorted(by_e.items()):
        tasks += [("C", i) for i in sample.draw_indices(su2, lc, nodes_c, rng, per_e, sectors=secs)]
    for name, legs, nodes in (("C", lc, nodes_c), ("dA", la, comb), ("dB", lb, comb)):
        secs = su2.layout(legs, nodes)[0]
        big = max(secs, key=lambda s: int(np.prod(su2.block_shape(legs, s))))
        tasks += [(name, i) for i in sample.draw_indices(su2, legs, nodes, rng, 8, sectors=[big])]
        if name != "C":
            tasks += [(name, i) for i in sample.draw_indices(su2, legs, nodes, rng, per_tensor)]
    return tasks


def _check(dmax, dtype, per_e, per_tensor, tol, graph=False):
    import paper_1203_2222_gb300 as P
    from paper_1203_2222_gb300 import synthetic
    c = synthetic.su2_recouple(dmax=dmax, jmax2=8)
    tasks = _tasks(c, dmax, per_e, per_tensor, seed=dmax)
    SA, SB = P.Structure(P.SU2, c["A"]), P.Structure(P.SU2, c["B"])
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1236)
    a = torch.randn(SA.numel, device="cuda", dtype=dtype, generator=gen).requires_grad_(True)
    b = torch.randn(SB.numel, device="cuda", dtype=dtype, generator=gen).requires_grad_(True)
    prec = P.FP64 if dtype == torch.float64 else P.BF16X3
    nc = P.contract_plan(SA, SB, c["pairsA"], c["pairsB"], prec).out.numel
    G = torch.randn(nc, device="cuda", dtype=dtype, generator=gen)

    def step():
        C = P.contract(P.SymTensor(SA, a), P.SymTensor(SB, b), c["pairsA"], c["pairsB"])
        return (C.data,) + tuple(torch.autograd.grad(C.data, [a, b], grad_outputs=G))

    if graph:  # the bench's launch configuration: the autograd step replayed from a CUDA graph
        (cdata, da, db), g = graph_replay.replay(step)
    else:
        cdata, da, db = step()
    torch.cuda.synchronize()
    P.device_status()
    # the six tensors (about 18 GB at full size) go to a memory-backed
    # directory when it has room, else to the default temporary directory
    need = sum(t.numel() * t.element_size() for t in (a, b, G, cdata, da, db))
    where = "/dev/shm" if os.path.isdir("/dev/shm") and shutil.disk_usage("/dev/shm").free > 2 * need else None
    d = tempfile.mkdtemp(prefix="su2full_", dir=where)
    try:
        for n, t in (("A", a), ("B", b), ("G", G), ("C", cdata), ("dA", da), ("dB", db)):
            np.save(os.path.join(d, n + ".npy"), t.detach().cpu().numpy())
        del a, b, G, cdata, da, db
        if graph:
            del g
        torch.cuda.empty_cache()
        res = oracle_pool.su2_elements(d, c, tasks)
    finally:
        shutil.rmtree(d, ignore_errors=True)
    for kind in ("C", "dA", "dB"):
        ref = np.array([r for k, r, _ in res if k == kind])
        got = np.array([g for k, _, g in res if k == kind])
        assert len(ref) >= (256 if per_tensor >= 256 else per_tensor)
        assert np.count_nonzero(np.abs(ref) > 0) >= 0.9 * len(ref), kind  # not zero against zero
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= tol, (kind, rel)


def test_su2_recouple_full_size_bf16x3_forward_and_backward_against_oracle():
    _check(32, torch.float32, per_e=16, per_tensor=256, tol=2e-5, graph=True)


def test_su2_recouple_half_size_fp64_forward_and_backward_against_oracle():
    _check(16, torch.float64, per_e=4, per_tensor=64, tol=1e-12)
