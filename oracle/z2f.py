"""Fermion-parity (Z2-graded) tensors, plain FP64 definition (oracle; test infrastructure only).

The thesis's conclusion sketches how the framework carries over to
fermionic charges: the charge is the parity p of the fermion number (p = 0
even, p = 1 odd); two parities fuse by addition mod 2 (the Z2 fusion
rules); every recoupling coefficient F equals 1; and the swap tensor R,
which encodes exchanging two charges, is 1 unless both charges are odd,
where it is -1.  Read into the block layout of the U(1) oracle:

* a leg is (parities, degeneracies, direction), parities 0/1 listed in the
  order of the leg's dense basis; the direction does not change a parity;
* a block (p_1, ..., p_k) is allowed iff p_1 + ... + p_k = P (mod 2), P the
  tensor's total parity; blocks are dense, row-major, concatenated in
  lexicographic sector order (leg 0 slowest);
* ``permute``: T'[i_perm(0), ..] = s(i) T[i_0, ..], where s(i) applies R
  once to every pair of legs whose order the permutation reverses (any
  decomposition into exchanges of neighbours crosses such a pair an odd
  number of times, every other pair an even number), i.e. s(i) = -1 to the
  number of reversed pairs whose parities at i are both odd;
* ``contract``: the thesis's recipe for a contraction -- permute A so that
  its free legs come first and its contracted legs last (in pair order),
  permute B so that its contracted legs come first (in pair order), and sum
  over the contracted index; no sign beyond those of the two permutations;
* ``fuse``: adjacent legs of equal direction, fused parity p_a + p_b mod 2,
  pairs ordered with p_a slowest and (t_a, t_b) row-major; fusing
  neighbours exchanges nothing, so it carries no sign.
"""
import itertools

import numpy as np


class Leg:
    def __init__(self, parities, degens, direction):
        assert len(parities) == len(degens)
        assert direction in (1, -1)
        assert all(p in (0, 1) for p in parities)
        self.labels = [int(p) for p in parities]
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

    def parity_of_index(self):
        """Parity of every dense index of the leg."""
        return np.concatenate([np.full(d, p, dtype=np.int64) for p, d in zip(self.labels, self.degens)])

    def dual(self):
        return Leg(self.labels, self.degens, -self.dir)


def swap(p, q):
    """The swap tensor R for charges p, q (thesis conclusion, fermionic charges)."""
    return -1.0 if (p == 1 and q == 1) else 1.0


def sectors(legs, P):
    out = []
    for idx in itertools.product(*[range(len(l.labels)) for l in legs]):
        if sum(l.labels[i] for l, i in zip(legs, idx)) % 2 == P:
            out.append(idx)
    return out


def block_shape(legs, sec):
    return tuple(l.degens[i] for l, i in zip(legs, sec))


def layout(legs, P):
    secs = sectors(legs, P)
    offs, acc = [], 0
    for s in secs:
        offs.append(acc)
        acc += int(np.prod(block_shape(legs, s), dtype=np.int64))
    return secs, offs, acc


def embed(legs, P, data):
    """Dense tensor whose allowed blocks are the given data, zero elsewhere."""
    data = np.asarray(data, dtype=np.float64)
    secs, offs, n = layout(legs, P)
    assert data.size == n, (data.size, n)
    dense = np.zeros([l.dim for l in legs])
    loffs = [l.offsets() for l in legs]
    for s, o in zip(secs, offs):
        shp = block_shape(legs, s)
        sl = tuple(slice(loffs[l][i], loffs[l][i] + shp[l]) for l, i in enumerate(s))
        dense[sl] = data[o:o + int(np.prod(shp, dtype=np.int64))].reshape(shp)
    return dense


def extract(legs, P, dense):
    """(blocks, residual): blocks read back; residual = norm outside the sectors."""
    secs, offs, n = layout(legs, P)
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


def sign_field(legs, perm):
    """s(i) over the dense index space of `legs` for the permutation `perm`
    (output leg n = input leg perm[n]): R applied to every reversed pair."""
    k = len(legs)
    par = [l.parity_of_index() for l in legs]
    s = np.ones([l.dim for l in legs])
    for a in range(k):
        for b in range(a + 1, k):
            # legs a < b end up in the order b, a when perm places b first
            if list(perm).index(a) > list(perm).index(b):
                shape = [1] * k
                shape[a] = legs[a].dim
                pa = par[a].reshape(shape)
                shape = [1] * k
                shape[b] = legs[b].dim
                pb = par[b].reshape(shape)
                s = s * np.where((pa == 1) & (pb == 1), -1.0, 1.0)
    return s


def permute_dense(legs, dense, perm):
    return np.transpose(sign_field(legs, perm) * dense, list(perm))


def permute(T, perm):
    """T = (legs, parity, data) -> (legs', parity, data', residual)."""
    legs, P, data = T
    legs2 = [legs[p] for p in perm]
    out, resid = extract(legs2, P, permute_dense(legs, embed(legs, P, data), perm))
    return legs2, P, out, resid


def _orders(rank, pairs, contracted_last):
    free = [i for i in range(rank) if i not in pairs]
    return free + list(pairs) if contracted_last else list(pairs) + free


def contract_dense(legsA, Ad, legsB, Bd, pairsA, pairsB):
    """C[freeA..., freeB...]: A and B permuted into matrix order with their
    swap signs, then summed over the contracted legs."""
    pa = _orders(len(legsA), pairsA, True)
    pb = _orders(len(legsB), pairsB, False)
    Ap = permute_dense(legsA, Ad, pa)
    Bp = permute_dense(legsB, Bd, pb)
    nc = len(pairsA)
    return np.tensordot(Ap, Bp, axes=(list(range(Ap.ndim - nc, Ap.ndim)), list(range(nc))))


def result_legs(legsA, legsB, pairsA, pairsB):
    for a, b in zip(pairsA, pairsB):
        la, lb = legsA[a], legsB[b]
        assert la.labels == lb.labels and la.degens == lb.degens and la.dir == -lb.dir, \
            "contracted legs must have equal content and opposite directions"
    return ([legsA[i] for i in range(len(legsA)) if i not in pairsA]
            + [legsB[i] for i in range(len(legsB)) if i not in pairsB])


def contract(A, B, pairsA, pairsB):
    """A, B = (legs, parity, data).  Returns (legsC, parityC, data, residual)."""
    legsA, PA, a = A
    legsB, PB, b = B
    legsC = result_legs(legsA, legsB, pairsA, pairsB)
    Cd = contract_dense(legsA, embed(legsA, PA, a), legsB, embed(legsB, PB, b), pairsA, pairsB)
    PC = (PA + PB) % 2
    c, resid = extract(legsC, PC, Cd)
    return legsC, PC, c, resid


def contract_grad(A, B, pairsA, pairsB, dC):
    """(dA, dB, residual): gradient of <dC, contract(A, B)> with respect to the
    blocks.  C is linear in each operand, so each gradient is the adjoint of
    its map: the matrix-form gradient permuted back by the inverse
    permutation, which reverses the same pairs and so carries the same signs."""
    legsA, PA, a = A
    legsB, PB, b = B
    legsC = result_legs(legsA, legsB, pairsA, pairsB)
    PC = (PA + PB) % 2
    nc = len(pairsA)
    pa = _orders(len(legsA), pairsA, True)
    pb = _orders(len(legsB), pairsB, False)
    Ap = permute_dense(legsA, embed(legsA, PA, a), pa)
    Bp = permute_dense(legsB, embed(legsB, PB, b), pb)
    G = embed(legsC, PC, dC)
    na = len(legsA) - nc
    nb = len(legsB) - nc
    # matrix-order gradients: dA'[freeA, c] = sum G[freeA, freeB] B'[c, freeB]
    dAp = np.tensordot(G, Bp, axes=(list(range(na, na + nb)), list(range(nc, nc + nb))))
    # dB'[c, freeB] = sum A'[freeA, c] G[freeA, freeB]
    dBp = np.tensordot(Ap, G, axes=(list(range(na)), list(range(na))))
    inv_a = list(np.argsort(pa))
    inv_b = list(np.argsort(pb))
    legsAp = [legsA[i] for i in pa]
    legsBp = [legsB[i] for i in pb]
    dA, ra = extract(legsA, PA, permute_dense(legsAp, dAp, inv_a))
    dB, rb = extract(legsB, PB, permute_dense(legsBp, dBp, inv_b))
    return dA, dB, max(ra, rb)


def fused_leg(a, b):
    """Leg d = a x b of two legs with equal direction and its fused pairs."""
    assert a.dir == b.dir
    qs = sorted({(pa + pb) % 2 for pa in a.labels for pb in b.labels})
    pairs, degens = [], []
    for q in qs:
        lst, acc = [], 0
        for ia, pa in enumerate(a.labels):
            for ib, pb in enumerate(b.labels):
                if (pa + pb) % 2 == q:
                    lst.append((ia, ib, acc))
                    acc += a.degens[ia] * b.degens[ib]
        pairs.append(lst)
        degens.append(acc)
    return Leg(qs, degens, a.dir), pairs


def fuse(T, first):
    """Fuse adjacent legs (first, first + 1) with the 0/1 fusion map (no sign)."""
    legs, P, data = T
    la, lb = legs[first], legs[first + 1]
    ld, pairs = fused_leg(la, lb)
    X = np.zeros((la.dim, lb.dim, ld.dim))
    aoff, boff, doff = la.offsets(), lb.offsets(), ld.offsets()
    for iq, lst in enumerate(pairs):
        for ia, ib, row0 in lst:
            for ta in range(la.degens[ia]):
                for tb in range(lb.degens[ib]):
                    X[aoff[ia] + ta, boff[ib] + tb, doff[iq] + row0 + ta * lb.degens[ib] + tb] = 1.0
    d = np.tensordot(embed(legs, P, data), X, axes=([first, first + 1], [0, 1]))
    d = np.moveaxis(d, -1, first)
    legs2 = legs[:first] + [ld] + legs[first + 2:]
    out, resid = extract(legs2, P, d)
    return legs2, P, out, resid
