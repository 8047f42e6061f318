"""SU(2) recoupling contraction at full size, checked on sampled dense elements.

The workload of the large-sector configuration: rank-4 SU(2) tensors whose
legs carry 2j = 0..8 with degeneracies drawn in 1..32, A in the comb tree,
its legs 1 and 3 contracted with the dual legs of B (the gather recouples A
into the matrix tree by 6j coefficients).  At this size (A: 7.5e8 block
entries, 1.3e13 useful flops per forward) the dense oracle cannot embed the
tensors, so the test draws elements of the dense result and lets the oracle
compute each one from two embedded slices (oracle.su2.embed_slice), and it
embeds the GPU's result blocks at the same indices.  The backward pass is
checked through the identity <dA, X> = <G, contract(X, B)> (C is linear in
A), which holds at any size; the gradients are checked against the oracle
and finite differences at small sizes in test_gpu_parity.py.

Inputs are N(0,1) draws of a seeded torch generator on the device.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _sampled_elements(la, lb, lc, nodes_c, ah, bh, ch, nsamp, seed):
    from oracle import su2
    secs = su2.layout(lc, nodes_c)[0]
    loffs = [l.offsets() for l in lc]
    rng = np.random.default_rng(seed)
    ref, got = [], []
    for _ in range(nsamp):
        sec = secs[int(rng.integers(len(secs)))]
        idx = []
        for l, p in enumerate(sec[0]):
            j2, d = lc[l].labels[p], lc[l].degens[p]
            idx.append(loffs[l][p] + int(rng.integers((j2 + 1) * d)))
        sa = su2.embed_slice(la, su2.left_comb(4), ah, {0: idx[0], 2: idx[1]})
        sb = su2.embed_slice(lb, su2.left_comb(4), bh, {2: idx[2], 3: idx[3]})
        ref.append(float(np.sum(sa * sb)))
        got.append(float(su2.embed_slice(lc, nodes_c, ch, dict(enumerate(idx)))))
    return np.array(got), np.array(ref)


@pytest.mark.parametrize("dmax,dtype,tol", [(32, torch.float32, 2e-5), (16, torch.float64, 1e-12)],
                         ids=["full_bf16x3", "half_fp64"])
def test_su2_recouple_contraction_sampled_against_oracle(dmax, dtype, tol):
    import paper_1203_2222_gb300 as P
    from paper_1203_2222_gb300 import synthetic
    from oracle import contract as oc
    from oracle import su2
    c = synthetic.su2_recouple(dmax=dmax, jmax2=8)
    SA, SB = P.Structure(P.SU2, c["A"]), P.Structure(P.SU2, c["B"])
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1236)
    a = torch.randn(SA.numel, device="cuda", dtype=dtype, generator=gen)
    b = torch.randn(SB.numel, device="cuda", dtype=dtype, generator=gen)
    C = P.contract(P.SymTensor(SA, a), P.SymTensor(SB, b), c["pairsA"], c["pairsB"])
    nodes_c = oc.comb_pair_tree(2, 2)
    assert C.structure.tree == nodes_c
    la = [su2.Leg(*l) for l in c["A"]]
    lb = [su2.Leg(*l) for l in c["B"]]
    lc = oc.result_legs(la, lb, c["pairsA"], c["pairsB"])
    ah, bh, ch = a.cpu().numpy(), b.cpu().numpy(), C.data.cpu().numpy()
    got, ref = _sampled_elements(la, lb, lc, nodes_c, ah, bh, ch, nsamp=24, seed=dmax)
    assert np.linalg.norm(ref) > 0
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= tol, rel


def test_su2_recouple_backward_is_the_adjoint_at_full_size():
    import paper_1203_2222_gb300 as P
    from paper_1203_2222_gb300 import synthetic
    c = synthetic.su2_recouple(dmax=32, jmax2=8)
    SA, SB = P.Structure(P.SU2, c["A"]), P.Structure(P.SU2, c["B"])
    gen = torch.Generator(device="cuda")
    gen.manual_seed(77)
    a = torch.randn(SA.numel, device="cuda", generator=gen).requires_grad_(True)
    b = torch.randn(SB.numel, device="cuda", generator=gen).requires_grad_(True)
    C = P.contract(P.SymTensor(SA, a), P.SymTensor(SB, b), c["pairsA"], c["pairsB"])
    G = torch.randn(C.structure.numel, device="cuda", generator=gen)
    da, db = torch.autograd.grad(C.data, [a, b], grad_outputs=G)
    X = torch.randn(SA.numel, device="cuda", generator=gen)
    Y = torch.randn(SB.numel, device="cuda", generator=gen)
    with torch.no_grad():
        cx = P.contract(P.SymTensor(SA, X), P.SymTensor(SB, b.detach()), c["pairsA"], c["pairsB"]).data
        cy = P.contract(P.SymTensor(SA, a.detach()), P.SymTensor(SB, Y), c["pairsA"], c["pairsB"]).data
    for g, x, cxy in ((da, X, cx), (db, Y, cy)):
        lhs = float(torch.dot(g.double(), x.double()))
        rhs = float(torch.dot(G.double(), cxy.double()))
        # both sides are sums of ~1e9 products of N(0,1) numbers computed in
        # split-BF16 with FP32 accumulation: compare against the scale of the terms
        scale = float(G.double().norm() * cxy.double().norm())
        assert abs(lhs - rhs) <= 2e-5 * scale, (lhs, rhs, scale)
