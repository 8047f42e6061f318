"""Single dense elements of a contraction and of its gradients (oracle).

TEST INFRASTRUCTURE ONLY.  For tensors too large to embed densely (the
full-size SU(2) recoupling contraction holds 7.5e8 block entries, 66 GB
dense) the plain definition is evaluated one dense element at a time:

* ``contraction_element``: Ch. 5, Eq. tensormult at one index of C,
  C[f_A, f_B] = sum_c A[f_A, c] B[c, f_B], from the slice of A with its free
  legs held at f_A and the slice of B with its free legs held at f_B.
* ``grad_a_element``: the gradient of <G, C> with respect to A at one dense
  index (f_A, c): sum_{f_B} G[f_A, f_B] B[c, f_B].
* ``grad_b_element``: the gradient with respect to B at (c, f_B):
  sum_{f_A} A[f_A, c] G[f_A, f_B].
* ``element``: the dense embedding of a block vector at one index.

The dense gradient of <G, C> is invariant (a contraction of invariant
tensors), and the embedding has orthonormal columns on the invariant
subspace, so the block gradient embedded at an index equals the dense
gradient there (the statement ``contract.contract_grad`` rests on).

Tensors are (legs, tree, data) with ``data`` any flat array indexable by
block offsets; ``m`` is the oracle module providing ``embed_slice``
(oracle.su2).  Pinned against the full dense oracle in
tests/test_oracle_sample.py.
"""
import numpy as np


def _free(rank, pairs):
    return [l for l in range(rank) if l not in pairs]


def contraction_element(m, A, B, pairsA, pairsB, idx):
    """C[idx], idx over C's legs (A's free legs, then B's free legs)."""
    legsA, tA, a = A
    legsB, tB, b = B
    freeA, freeB = _free(len(legsA), pairsA), _free(len(legsB), pairsB)
    sa = m.embed_slice(legsA, tA, a, {l: idx[i] for i, l in enumerate(freeA)})
    sb = m.embed_slice(legsB, tB, b, {l: idx[len(freeA) + i] for i, l in enumerate(freeB)})
    # slice axes run over the contracted legs in each tensor's own leg order;
    # bring both into pair order before summing the product
    ca, cb = sorted(pairsA), sorted(pairsB)
    sa = np.transpose(sa, [ca.index(p) for p in pairsA])
    sb = np.transpose(sb, [cb.index(p) for p in pairsB])
    return float(np.sum(sa * sb))


def grad_a_element(m, A, B, pairsA, pairsB, Cg, idx):
    """d<G, C>/dA at the dense index idx over A's legs; Cg = (legsC, treeC, G)."""
    legsA = A[0]
    legsB, tB, b = B
    legsC, tC, g = Cg
    freeA, freeB = _free(len(legsA), pairsA), _free(len(legsB), pairsB)
    sg = m.embed_slice(legsC, tC, g, {i: idx[l] for i, l in enumerate(freeA)})  # over C's B-side legs
    sb = m.embed_slice(legsB, tB, b, {pb: idx[pa] for pa, pb in zip(pairsA, pairsB)})  # over B's free legs
    assert sg.shape == sb.shape
    return float(np.sum(sg * sb))


def grad_b_element(m, A, B, pairsA, pairsB, Cg, idx):
    """d<G, C>/dB at the dense index idx over B's legs; Cg = (legsC, treeC, G)."""
    legsA, tA, a = A
    legsB = B[0]
    legsC, tC, g = Cg
    freeA, freeB = _free(len(legsA), pairsA), _free(len(legsB), pairsB)
    sa = m.embed_slice(legsA, tA, a, {pa: idx[pb] for pa, pb in zip(pairsA, pairsB)})  # over A's free legs
    sg = m.embed_slice(legsC, tC, g, {len(freeA) + i: idx[l] for i, l in enumerate(freeB)})  # over C's A-side legs
    assert sa.shape == sg.shape
    return float(np.sum(sa * sg))


def element(m, T, idx):
    """embed(T)[idx] without forming the dense tensor."""
    legs, t, data = T
    return float(m.embed_slice(legs, t, data, dict(enumerate(idx))))


def draw_indices(m, legs, nodes, rng, k, sectors=None):
    """k dense indices of a tensor with the given legs and tree, each in a
    sector drawn uniformly (or from ``sectors``, a list of sector keys as
    ``m.layout`` lists them), with degeneracy indices uniform and the
    magnetic numbers conserving J_z: sum over legs of dir * m = 0 (a cup
    turns an incoming leg's m into -m), so that the element is not a
    structural zero of the invariant tensor.  Where no conserving choice
    exists for the last leg after a few tries, the last draw is kept."""
    secs = sectors if sectors is not None else m.layout(legs, nodes)[0]
    loffs = [l.offsets() for l in legs]
    out = []
    for _ in range(k):
        sec = secs[int(rng.integers(len(secs)))]
        pos = sec[0]
        j2 = [legs[l].labels[p] for l, p in enumerate(pos)]
        for _try in range(32):
            m2 = [int(rng.integers(j + 1)) * 2 - j for j in j2[:-1]]
            last = -legs[-1].dir * sum(legs[l].dir * x for l, x in enumerate(m2))
            if abs(last) <= j2[-1]:
                break
        else:
            last = int(rng.integers(j2[-1] + 1)) * 2 - j2[-1]
        m2.append(last)
        idx = []
        for l, p in enumerate(pos):
            t = int(rng.integers(legs[l].degens[p]))
            idx.append(loffs[l][p] + t * (j2[l] + 1) + (m2[l] + j2[l]) // 2)
        out.append(idx)
    return out
