"""SU(2)-invariant tensors in a tree decomposition, plain FP64 definition.

Oracle; test infrastructure only.  Follows Ch. 6, "Tree decompositions of
SU(2)-invariant tensors": a tensor T with legs i_1..i_k is stored as
(legs, directions, fusion tree tau, vector v), where v is the SU(2)-invariant
vector obtained by fusing all legs along tau; T is recovered by applying the
splitting tensors of tau to v and a cup to every incoming leg.

Conventions fixed here (the thesis leaves them open or prints them garbled):

* A leg is (doubled spins 2j in ascending order, degeneracies d_j, direction);
  its dense basis runs over spins in listed order, inside a spin over t
  (slow) and m = -j..j (fast) -- the order of Ch. 5, Examples 4-5.
* A tree over k legs is a list of k-1 nodes (left, right); ids 0..k-1 are the
  legs, node n has id k+n, the last node is the root, and each node joins
  two adjacent leg ranges (left range first).  Default: the left comb
  ((0,1),2),...  The root link carries spin 0 (v is invariant).
* The components of v are grouped into degeneracy blocks P, one per sector
  = (spin position on every leg, spin on every non-root node).  Sectors are
  ordered lexicographically by leg spin positions (leg 0 slowest), then by
  node spins (node 0 slowest).  A block is d_{j_1} x ... x d_{j_k},
  row-major, blocks concatenated in sector order.  This is the X-map of
  Ch. 5, Example 7 taken row-major (the printed list and the text of that
  example disagree on which index runs fastest; any bijection is valid).
* The structural part of a sector is the tree of CG tensors
  C_{a,b->c}(m_a, m_b, m_c) (Ch. 5, Eq. cg; a splitting tensor has the same
  values, Eq. splitcg) with the root projected on m = 0, and on every
  incoming leg the cup of Ch. 5, Eq. cupj applied as
  T[.., m, ..] = sum_m' cup_j[m, m'] T'[.., m', ..]  (the reversal of
  Ch. 5, Example 12; Ch. 6 stores the cup as part of the decomposition).

``embed`` sums P (x) Q over sectors into the dense tensor; ``extract``
projects a dense tensor back, P = <Q, T>/<Q, Q>, and reports the residual
T - embed(P) (zero iff T lies in the span of the tree basis).
``invariance_residual`` measures sum_l J^(l) T for Jz, J+ and J- with the
conjugate representation on incoming legs (Ch. 5, Eq. Tinv).
"""
import itertools
from math import sqrt

import numpy as np

from . import cg as cgm


class Leg:
    def __init__(self, spins2, degens, direction):
        assert len(spins2) == len(degens)
        assert list(spins2) == sorted(set(spins2))
        assert direction in (1, -1)
        self.labels = [int(s) for s in spins2]
        self.degens = [int(d) for d in degens]
        self.dir = int(direction)

    @property
    def dim(self):
        return sum((j2 + 1) * d for j2, d in zip(self.labels, self.degens))

    def offsets(self):
        out, acc = [], 0
        for j2, d in zip(self.labels, self.degens):
            out.append(acc)
            acc += (j2 + 1) * d
        return out

    def dual(self):
        return Leg(self.labels, self.degens, -self.dir)

    def __repr__(self):
        return f"SU2Leg({self.labels}, {self.degens}, {self.dir})"


def left_comb(k):
    """((0,1),2),... as a node list."""
    if k < 2:
        return []
    nodes = [(0, 1)]
    for i in range(2, k):
        nodes.append((k + i - 2, i))
    return nodes


def check_tree(k, nodes):
    """Validate a planar binary tree over k legs; return each id's leg range."""
    assert len(nodes) == max(k - 1, 0)
    rng = {i: (i, i + 1) for i in range(k)}
    used = set()
    for n, (a, b) in enumerate(nodes):
        assert a in rng and b in rng and a not in used and b not in used, nodes
        assert rng[a][1] == rng[b][0], "children must be adjacent, left first"
        rng[k + n] = (rng[a][0], rng[b][1])
        used.update((a, b))
    if k >= 2:
        assert rng[k + len(nodes) - 1] == (0, k)
    return rng


def sectors(legs, nodes):
    """Allowed sectors: (leg spin positions, node spins excluding the root)."""
    k = len(legs)
    nodes = list(nodes)
    check_tree(k, nodes)
    out = []
    for idx in itertools.product(*[range(len(l.labels)) for l in legs]):
        spin = {i: legs[i].labels[p] for i, p in enumerate(idx)}
        if k == 1:
            if spin[0] == 0:
                out.append((idx, ()))
            continue
        if k == 0:
            out.append(((), ()))
            continue

        def rec(n, spin):
            a, b = nodes[n]
            ja, jb = spin[a], spin[b]
            last = n == len(nodes) - 1
            cands = [0] if last else range(abs(ja - jb), ja + jb + 1, 2)
            for jc in cands:
                if not cgm.triangle(ja, jb, jc):
                    continue
                spin2 = dict(spin)
                spin2[k + n] = jc
                if last:
                    yield tuple(spin2[k + i] for i in range(len(nodes) - 1))
                else:
                    yield from rec(n + 1, spin2)

        for inner in rec(0, spin):
            out.append((idx, inner))
    return out


def block_shape(legs, sec):
    return tuple(l.degens[i] for l, i in zip(legs, sec[0]))


def layout(legs, nodes):
    secs = sectors(legs, nodes)
    offs, acc = [], 0
    for s in secs:
        offs.append(acc)
        acc += int(np.prod(block_shape(legs, s), dtype=np.int64))
    return secs, offs, acc


def structure_tensor(legs, nodes, sec):
    """Q[m_1..m_k] of one sector: CG tree, root on m=0, cups on 'in' legs."""
    k = len(legs)
    spin = {i: legs[i].labels[p] for i, p in enumerate(sec[0])}
    for n in range(len(nodes) - 1):
        spin[k + n] = sec[1][n]
    if k >= 2:
        spin[k + len(nodes) - 1] = 0
    if k == 0:
        return np.ones(())
    if k == 1:
        q = np.ones((1,))
    else:
        sub = {i: np.eye(spin[i] + 1) for i in range(k)}  # axes: (legs..., top m)
        for n, (a, b) in enumerate(nodes):
            c = cgm.cg_tensor(spin[a], spin[b], spin[k + n])
            ta, tb = sub.pop(a), sub.pop(b)
            x = np.tensordot(ta, c, axes=([ta.ndim - 1], [0]))   # (..a, b, c)
            x = np.tensordot(x, tb, axes=([ta.ndim - 1], [tb.ndim - 1]))  # (..a, c, ..b)
            x = np.moveaxis(x, ta.ndim - 1, -1)                   # (..a, ..b, c)
            sub[k + n] = x
        q = sub[k + len(nodes) - 1][..., 0]
    for i, l in enumerate(legs):
        if l.dir == -1:
            q = np.moveaxis(np.tensordot(cgm.cup(spin[i]), q, axes=([1], [i])), 0, i)
    return q


def _slices(legs, sec, loffs):
    sl = []
    for l, (leg, p) in enumerate(zip(legs, sec[0])):
        n = (leg.labels[p] + 1) * leg.degens[p]
        sl.append(slice(loffs[l][p], loffs[l][p] + n))
    return tuple(sl)


def _interleave(P, Q):
    """(d_1..d_k) x (n_1..n_k) -> dense sub-block with index t*n + m per leg."""
    k = P.ndim
    x = np.multiply.outer(P, Q)  # (d..., n...)
    order = [a for i in range(k) for a in (i, k + i)]
    x = np.transpose(x, order)
    return x.reshape([P.shape[i] * Q.shape[i] for i in range(k)])


def embed(legs, nodes, data):
    data = np.asarray(data, dtype=np.float64)
    secs, offs, n = layout(legs, nodes)
    assert data.size == n, (data.size, n)
    dense = np.zeros([l.dim for l in legs])
    loffs = [l.offsets() for l in legs]
    for s, o in zip(secs, offs):
        shp = block_shape(legs, s)
        P = data[o:o + int(np.prod(shp, dtype=np.int64))].reshape(shp)
        Q = structure_tensor(legs, nodes, s)
        dense[_slices(legs, s, loffs)] += _interleave(P, Q)
    return dense


def embed_slice(legs, nodes, data, fixed):
    """Sub-tensor of embed(legs, nodes, data) with some legs held at one index.

    ``fixed`` maps leg -> dense index on that leg; the result runs over the
    other legs in order (a scalar when every leg is fixed).  Only the sectors
    whose spins on the fixed legs match contribute, so one slice of a large
    tensor costs a fraction of the full embedding.  ``data`` may be any flat
    array indexable by the layout's block offsets (read in FP64).
    """
    secs, offs, _ = layout(legs, nodes)
    loffs = [l.offsets() for l in legs]
    k = len(legs)
    dec = {}
    for l, i in fixed.items():
        leg = legs[l]
        for p, (o, j2, d) in enumerate(zip(loffs[l], leg.labels, leg.degens)):
            if o <= i < o + (j2 + 1) * d:
                r = i - o
                dec[l] = (p, r // (j2 + 1), r % (j2 + 1))  # spin position, t, m
                break
        else:
            raise IndexError(f"index {i} outside leg {l}")
    free = [l for l in range(k) if l not in fixed]
    out = np.zeros([legs[l].dim for l in free])
    for s, o in zip(secs, offs):
        if any(s[0][l] != dec[l][0] for l in fixed):
            continue
        shp = block_shape(legs, s)
        P = np.asarray(data[o:o + int(np.prod(shp, dtype=np.int64))], dtype=np.float64).reshape(shp)
        Q = structure_tensor(legs, nodes, s)
        ip = tuple(dec[l][1] if l in fixed else slice(None) for l in range(k))
        iq = tuple(dec[l][2] if l in fixed else slice(None) for l in range(k))
        sl = []
        for l in free:
            p = s[0][l]
            n = (legs[l].labels[p] + 1) * legs[l].degens[p]
            sl.append(slice(loffs[l][p], loffs[l][p] + n))
        out[tuple(sl)] += _interleave(np.asarray(P[ip]), np.asarray(Q[iq]))
    return out


def extract(legs, nodes, dense):
    """(blocks, residual): P = <Q,T>/<Q,Q> per sector; residual = |T - embed(P)|."""
    secs, offs, n = layout(legs, nodes)
    out = np.zeros(n)
    loffs = [l.offsets() for l in legs]
    k = len(legs)
    for s, o in zip(secs, offs):
        shp = block_shape(legs, s)
        Q = structure_tensor(legs, nodes, s)
        sub = dense[_slices(legs, s, loffs)]
        # split every dense leg index into (t, m)
        sub = sub.reshape([a for i in range(k) for a in (shp[i], Q.shape[i])])
        P = np.tensordot(sub, Q, axes=(list(range(1, 2 * k, 2)), list(range(k))))
        out[o:o + P.size] = P.reshape(-1) / float(np.sum(Q * Q))
    resid = float(np.linalg.norm(dense - embed(legs, nodes, out))) if dense.size else 0.0
    return out, resid


def leg_generators(leg):
    """(Jz, J+, J-) on the dense space of a leg: (+)_j I_{d_j} (x) J_j."""
    n = leg.dim
    mats = [np.zeros((n, n)) for _ in range(3)]
    for off, j2, d in zip(leg.offsets(), leg.labels, leg.degens):
        gens = cgm.generators(j2)
        for g, M in zip(gens, mats):
            M[off:off + d * (j2 + 1), off:off + d * (j2 + 1)] = np.kron(np.eye(d), g)
    return mats


def invariance_residual(legs, dense):
    """max over Jz, J+, J- of |sum_l G_l T|, G = J on 'out', -J^* on 'in' legs.

    For the real ladder matrices, -J^* of (Jz, J+, J-) is (-Jz, -J-, -J+).
    """
    res = 0.0
    gens = [leg_generators(l) for l in legs]
    for a in range(3):
        acc = np.zeros(dense.shape)
        for i, l in enumerate(legs):
            jz, jp, jm = gens[i]
            if l.dir == 1:
                G = (jz, jp, jm)[a]
            else:
                G = (-jz, -jm, -jp)[a]
            acc += np.moveaxis(np.tensordot(G, dense, axes=([1], [i])), 0, i)
        res = max(res, float(np.linalg.norm(acc)))
    return res


def fused_leg(a, b):
    """Leg d = a x b (equal directions): spins jd of every compatible (ja, jb).

    Degeneracy d_jd = sum over compatible (ja, jb) of d_ja d_jb, the pairs
    ordered lexicographically (ja slowest) and (t_a, t_b) row-major inside a
    pair (Ch. 5, Eq. decoVAB and Example 8).  Returns (leg, pairs) with
    pairs[jd_index] = [(ia, ib, row0), ...].
    """
    assert a.dir == b.dir
    js = sorted({jc for ja in a.labels for jb in b.labels
                 for jc in range(abs(ja - jb), ja + jb + 1, 2)})
    pairs, degens = [], []
    for jd in js:
        lst, acc = [], 0
        for ia, ja in enumerate(a.labels):
            for ib, jb in enumerate(b.labels):
                if cgm.triangle(ja, jb, jd):
                    lst.append((ia, ib, acc))
                    acc += a.degens[ia] * b.degens[ib]
        pairs.append(lst)
        degens.append(acc)
    return Leg(js, degens, a.dir), pairs


def fusing_tensor(a, b):
    """Dense Upsilon[(a),(b),(d)] = X (degeneracy map) x C (Ch. 5, Eq. basischange1)."""
    d, pairs = fused_leg(a, b)
    U = np.zeros((a.dim, b.dim, d.dim))
    aoff, boff, doff = a.offsets(), b.offsets(), d.offsets()
    for iq, lst in enumerate(pairs):
        jd = d.labels[iq]
        for ia, ib, row0 in lst:
            ja, jb = a.labels[ia], b.labels[ib]
            c = cgm.cg_tensor(ja, jb, jd)
            for ta in range(a.degens[ia]):
                for tb in range(b.degens[ib]):
                    td = row0 + ta * b.degens[ib] + tb
                    U[aoff[ia] + ta * (ja + 1): aoff[ia] + (ta + 1) * (ja + 1),
                      boff[ib] + tb * (jb + 1): boff[ib] + (tb + 1) * (jb + 1),
                      doff[iq] + td * (jd + 1): doff[iq] + (td + 1) * (jd + 1)] = c
    return d, U


def leg_cup(leg):
    """(+)_j I_{d_j} (x) cup_j on the dense space of a leg (Ch. 5, Eq. cup)."""
    M = np.zeros((leg.dim, leg.dim))
    for off, j2, d in zip(leg.offsets(), leg.labels, leg.degens):
        M[off:off + d * (j2 + 1), off:off + d * (j2 + 1)] = np.kron(np.eye(d), cgm.cup(j2))
    return M


def leg_cap(leg):
    M = np.zeros((leg.dim, leg.dim))
    for off, j2, d in zip(leg.offsets(), leg.labels, leg.degens):
        M[off:off + d * (j2 + 1), off:off + d * (j2 + 1)] = np.kron(np.eye(d), cgm.cap(j2))
    return M
