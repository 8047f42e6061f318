"""U(1)-symmetric tensors, plain FP64 definition (oracle; test infrastructure only).

Ch. 4 of the thesis (the U(1) implementation) is not in the available text;
what is used here is its general statement (Ch. 1 and Ch. 7: blocks labelled
by charges, charges conserved) read through the direction rule of Ch. 5
(an incoming index carries the dual space, so it contributes -q):

* a leg is (charges, degeneracies, direction), charges listed in the order of
  the leg's dense basis; direction +1 = 'out', -1 = 'in';
* a block (sector) is a tuple of charge positions, one per leg; it is allowed
  iff  sum_out q - sum_in q == Q  (the tensor's total charge);
* blocks are dense arrays d_1 x ... x d_k in row-major order (last leg
  fastest), concatenated in lexicographic sector order (leg 0 slowest);
* the dense index of leg l runs over its charges in listed order and, inside
  a charge, over the degeneracy index t.

``embed`` writes the blocks into the dense tensor (zeros elsewhere) and
``extract`` reads them back, reporting the norm of what lies outside the
allowed sectors.  Dense leg fusion follows the same enumeration rule: fused
charge q = q_a + q_b for legs of equal direction, fused pairs ordered
lexicographically (q_a slowest), and (t_a, t_b) row-major inside a pair.
"""
import itertools

import numpy as np


class Leg:
    def __init__(self, charges, degens, direction):
        assert len(charges) == len(degens)
        assert direction in (1, -1)
        self.labels = [int(q) for q in charges]
        self.degens = [int(d) for d in degens]
        self.dir = int(direction)

    @property
    def dim(self):
        return sum(self.degens)

    def offsets(self):
        out, acc = [], 0
        for d in self.degens:
            out.append(acc)
            acc += d
        return out

    def dual(self):
        return Leg(self.labels, self.degens, -self.dir)

    def __repr__(self):
        return f"U1Leg({self.labels}, {self.degens}, {self.dir})"


def sectors(legs, Q):
    """All allowed charge-position tuples, lexicographic (leg 0 slowest)."""
    out = []
    for idx in itertools.product(*[range(len(l.labels)) for l in legs]):
        tot = sum(l.dir * l.labels[i] for l, i in zip(legs, idx))
        if tot == Q:
            out.append(idx)
    return out


def block_shape(legs, sec):
    return tuple(l.degens[i] for l, i in zip(legs, sec))


def layout(legs, Q):
    """(sectors, block offsets, numel): blocks concatenated in sector order."""
    secs = sectors(legs, Q)
    offs, acc = [], 0
    for s in secs:
        offs.append(acc)
        acc += int(np.prod(block_shape(legs, s), dtype=np.int64))
    return secs, offs, acc


def embed(legs, Q, data):
    """Dense tensor whose allowed blocks are the given data, zero elsewhere."""
    data = np.asarray(data, dtype=np.float64)
    secs, offs, n = layout(legs, Q)
    assert data.size == n, (data.size, n)
    dense = np.zeros([l.dim for l in legs])
    loffs = [l.offsets() for l in legs]
    for s, o in zip(secs, offs):
        shp = block_shape(legs, s)
        sl = tuple(slice(loffs[l][i], loffs[l][i] + shp[l]) for l, i in enumerate(s))
        dense[sl] = data[o:o + int(np.prod(shp, dtype=np.int64))].reshape(shp)
    return dense


def extract(legs, Q, dense):
    """(blocks, residual): blocks read back; residual = norm outside the sectors."""
    secs, offs, n = layout(legs, Q)
    out = np.zeros(n)
    mask = np.zeros(dense.shape, dtype=bool)
    loffs = [l.offsets() for l in legs]
    for s, o in zip(secs, offs):
        shp = block_shape(legs, s)
        sl = tuple(slice(loffs[l][i], loffs[l][i] + shp[l]) for l, i in enumerate(s))
        out[o:o + int(np.prod(shp, dtype=np.int64))] = dense[sl].reshape(-1)
        mask[sl] = True
    resid = float(np.linalg.norm(dense[~mask])) if dense.size else 0.0
    return out, resid


def fused_leg(a, b):
    """Leg d = a x b of two legs with equal direction (enumeration rule above).

    Returns (leg, pairs) where pairs[qd_index] lists, in fused order, the
    (ia, ib, row0) charge-position pairs with their first fused row.
    """
    assert a.dir == b.dir
    qs = sorted({qa + qb for qa in a.labels for qb in b.labels})
    pairs, degens = [], []
    for q in qs:
        lst, acc = [], 0
        for ia, qa in enumerate(a.labels):
            for ib, qb in enumerate(b.labels):
                if qa + qb == q:
                    lst.append((ia, ib, acc))
                    acc += a.degens[ia] * b.degens[ib]
        pairs.append(lst)
        degens.append(acc)
    return Leg(qs, degens, a.dir), pairs


def fusion_matrix(a, b):
    """Dense 0/1 map X[(a),(b),(d)] of the fusion a x b -> d (a permutation)."""
    d, pairs = fused_leg(a, b)
    X = np.zeros((a.dim, b.dim, d.dim))
    aoff, boff, doff = a.offsets(), b.offsets(), d.offsets()
    for iq, lst in enumerate(pairs):
        for ia, ib, row0 in lst:
            for ta in range(a.degens[ia]):
                for tb in range(b.degens[ib]):
                    X[aoff[ia] + ta, boff[ib] + tb,
                      doff[iq] + row0 + ta * b.degens[ib] + tb] = 1.0
    return d, X
