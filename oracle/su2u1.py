"""SU(2) x U(1)-invariant tensors, plain FP64 definition (oracle; test infrastructure only).

The thesis's conclusion notes that the framework extends to a symmetry made
of several groups, which then act component by component.  For SU(2) x U(1)
a label is a pair (q, 2j): a U(1) charge and an SU(2) spin.  Read into the
two single-group oracles (u1.py, su2.py):

* a leg is (labels, degeneracies, direction) with labels (q, 2j) strictly
  increasing (charge slowest).  Its dense basis runs over the labels in
  order and, inside a label, over t (degeneracy, slowest) and m (the spin
  projection, fastest), as for an SU(2) leg;
* a sector is one label per leg whose charges obey the U(1) rule
  (sum of dir * q = Q, the tensor's total charge) together with node spins
  of the fusion tree that obey the SU(2) rules for the spin parts (root
  spin 0).  Node charges are not labels: a node's charge is fixed by the
  legs below it;
* the structural part of a sector is the SU(2) one of its spins (CG tree
  with the root on m = 0, cups on incoming legs), since the U(1) factor of
  a charge-conserving block is 1;
* fusing two legs of equal direction adds the charges and couples the spins
  (pairs of labels ordered with the first leg slowest, (t_a, t_b) row-major,
  fused labels ascending), with the CG tensor of the spins as its map.

A tensor is (legs, (tree nodes, Q), data).  ``embed`` sums block (x)
structure over sectors; ``extract`` projects back and reports the residual;
``invariance_residual`` applies the SU(2) generators and the charge operator.
"""
import itertools

import numpy as np

from . import cg as cgm
from . import su2 as su2m


class Leg:
    def __init__(self, labels, degens, direction):
        labels = [(int(q), int(j2)) for q, j2 in labels]
        assert len(labels) == len(degens)
        assert labels == sorted(set(labels)), "labels (q, 2j) must increase strictly"
        assert all(j2 >= 0 for _, j2 in labels)
        assert direction in (1, -1)
        self.labels = labels
        self.degens = [int(d) for d in degens]
        self.dir = int(direction)

    @property
    def dim(self):
        return sum((j2 + 1) * d for (_, j2), d in zip(self.labels, self.degens))

    def offsets(self):
        out, acc = [], 0
        for (_, j2), d in zip(self.labels, self.degens):
            out.append(acc)
            acc += (j2 + 1) * d
        return out

    def spin_leg(self, i):
        """The SU(2) leg of label i alone (its spin, degeneracy and direction)."""
        return su2m.Leg([self.labels[i][1]], [self.degens[i]], self.dir)

    def dual(self):
        return Leg(self.labels, self.degens, -self.dir)


def _fake(legs, idx):
    return [l.spin_leg(i) for l, i in zip(legs, idx)]


def sectors(legs, tot):
    """(label positions, node spins) of every allowed block, lexicographic."""
    nodes, Q = tot
    out = []
    for idx in itertools.product(*[range(len(l.labels)) for l in legs]):
        if sum(l.dir * l.labels[i][0] for l, i in zip(legs, idx)) != Q:
            continue
        for _, inner in su2m.sectors(_fake(legs, idx), nodes):
            out.append((idx, inner))
    return out


def block_shape(legs, sec):
    return tuple(l.degens[i] for l, i in zip(legs, sec[0]))


def layout(legs, tot):
    secs = sectors(legs, tot)
    offs, acc = [], 0
    for s in secs:
        offs.append(acc)
        acc += int(np.prod(block_shape(legs, s), dtype=np.int64))
    return secs, offs, acc


def structure_tensor(legs, tot, sec):
    nodes, _ = tot
    k = len(legs)
    return su2m.structure_tensor(_fake(legs, sec[0]), nodes, ((0,) * k, sec[1]))


def _slices(legs, sec):
    sl = []
    for l, p in zip(legs, sec[0]):
        off = l.offsets()[p]
        sl.append(slice(off, off + (l.labels[p][1] + 1) * l.degens[p]))
    return tuple(sl)


def embed(legs, tot, data):
    data = np.asarray(data, dtype=np.float64)
    secs, offs, n = layout(legs, tot)
    assert data.size == n, (data.size, n)
    dense = np.zeros([l.dim for l in legs])
    for s, o in zip(secs, offs):
        shp = block_shape(legs, s)
        P = data[o:o + int(np.prod(shp, dtype=np.int64))].reshape(shp)
        dense[_slices(legs, s)] += su2m._interleave(P, structure_tensor(legs, tot, s))
    return dense


def extract(legs, tot, dense):
    """(blocks, residual): P = <Q, T>/<Q, Q> per sector; residual = |T - embed(P)|."""
    secs, offs, n = layout(legs, tot)
    out = np.zeros(n)
    k = len(legs)
    for s, o in zip(secs, offs):
        shp = block_shape(legs, s)
        Q = structure_tensor(legs, tot, s)
        sub = dense[_slices(legs, s)].reshape([a for i in range(k) for a in (shp[i], Q.shape[i])])
        P = np.tensordot(sub, Q, axes=(list(range(1, 2 * k, 2)), list(range(k))))
        out[o:o + P.size] = P.reshape(-1) / float(np.sum(Q * Q))
    resid = float(np.linalg.norm(dense - embed(legs, tot, out))) if dense.size else 0.0
    return out, resid


def leg_generators(leg):
    """(Jz, J+, J-, N) on the dense space of a leg: SU(2) generators on the
    spin parts, N the charge."""
    n = leg.dim
    mats = [np.zeros((n, n)) for _ in range(4)]
    for off, (q, j2), d in zip(leg.offsets(), leg.labels, leg.degens):
        sl = slice(off, off + d * (j2 + 1))
        for g, M in zip(cgm.generators(j2), mats):
            M[sl, sl] = np.kron(np.eye(d), g)
        mats[3][sl, sl] = q * np.eye(d * (j2 + 1))
    return mats


def invariance_residual(legs, tot, dense):
    """max of |sum_l G_l T| for Jz, J+, J- (conjugate on 'in' legs) and of
    |sum_l dir_l N_l T - Q T| (charge conservation)."""
    _, Q = tot
    gens = [leg_generators(l) for l in legs]
    res = 0.0
    for a in range(3):
        acc = np.zeros(dense.shape)
        for i, l in enumerate(legs):
            jz, jp, jm, _ = gens[i]
            G = (jz, jp, jm)[a] if l.dir == 1 else (-jz, -jm, -jp)[a]
            acc += np.moveaxis(np.tensordot(G, dense, axes=([1], [i])), 0, i)
        res = max(res, float(np.linalg.norm(acc)))
    acc = -Q * dense
    for i, l in enumerate(legs):
        acc = acc + l.dir * np.moveaxis(np.tensordot(gens[i][3], dense, axes=([1], [i])), 0, i)
    return max(res, float(np.linalg.norm(acc)))


def fused_leg(a, b):
    """Leg d = a x b (equal directions) and, per fused label, its (ia, ib, row0) pairs."""
    assert a.dir == b.dir
    labs = sorted({(qa + qb, jc) for (qa, ja) in a.labels for (qb, jb) in b.labels
                   for jc in range(abs(ja - jb), ja + jb + 1, 2)})
    pairs, degens = [], []
    for (q, jd) in labs:
        lst, acc = [], 0
        for ia, (qa, ja) in enumerate(a.labels):
            for ib, (qb, jb) in enumerate(b.labels):
                if qa + qb == q and cgm.triangle(ja, jb, jd):
                    lst.append((ia, ib, acc))
                    acc += a.degens[ia] * b.degens[ib]
        pairs.append(lst)
        degens.append(acc)
    return Leg(labs, degens, a.dir), pairs


def fusing_tensor(a, b):
    """Dense map [(a), (b), (d)]: the degeneracy pairing times the spins' CG tensor."""
    d, pairs = fused_leg(a, b)
    U = np.zeros((a.dim, b.dim, d.dim))
    aoff, boff, doff = a.offsets(), b.offsets(), d.offsets()
    for iq, lst in enumerate(pairs):
        jd = d.labels[iq][1]
        for ia, ib, row0 in lst:
            ja, jb = a.labels[ia][1], b.labels[ib][1]
            c = cgm.cg_tensor(ja, jb, jd)
            for ta in range(a.degens[ia]):
                for tb in range(b.degens[ib]):
                    td = row0 + ta * b.degens[ib] + tb
                    U[aoff[ia] + ta * (ja + 1): aoff[ia] + (ta + 1) * (ja + 1),
                      boff[ib] + tb * (jb + 1): boff[ib] + (tb + 1) * (jb + 1),
                      doff[iq] + td * (jd + 1): doff[iq] + (td + 1) * (jd + 1)] = c
    return d, U


def _leg_block_map(leg, f):
    M = np.zeros((leg.dim, leg.dim))
    for off, (_, j2), d in zip(leg.offsets(), leg.labels, leg.degens):
        M[off:off + d * (j2 + 1), off:off + d * (j2 + 1)] = np.kron(np.eye(d), f(j2))
    return M


def leg_cup(leg):
    return _leg_block_map(leg, cgm.cup)


def leg_cap(leg):
    return _leg_block_map(leg, cgm.cap)
