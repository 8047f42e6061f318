"""Blockwise singular value decomposition, plain FP64 (oracle; test infrastructure only).

Ch. 5, "Factorization of a matrix" (Eq. svd0, svd1) and Ch. 6, "Matrix
multiplication and factorizations": a symmetric matrix is block diagonal in
the label it carries between its row and column spaces, so its SVD is the
SVD of every block, taken independently, and the factors are recast into
tensors with the same block structure.  The steps, in that order:

1. block-diagonal form: T with rows = legs 0..nrow-1 and columns = the other
   legs.  A block of T (one label position per leg) lies in the diagonal
   block M_x of the fused row label x (U(1): x = sum of dir * q over the row
   legs; fermion parity: x = sum of the row parities mod 2).  Inside M_x the
   row label tuples are listed lexicographically (leg 0 slowest), each
   taking prod d rows, and likewise the column tuples; the tensor block,
   row-major with the row legs leading, is the (prod d_rows) x (prod d_cols)
   sub-matrix at its tuples' first row and column.  SU(2): rank-2 tensors
   (the block-diagonal form of Eq. svd0), x = the spin 2j both legs carry;
2. M_x = U_x diag(S_x) V_x (numpy's SVD of the block, thin, descending).
   SU(2): the stored block is not the thesis's canonical T_j.  With the
   normalisation of reading 5 the dense matrix is the direct sum of
   M_x / sqrt(2j+1) times a (2j+1)-dimensional orthogonal map, so its
   singular values are S_x / sqrt(2j+1), each 2j+1 times (pinned against the
   dense SVD), and the factors whose contraction rebuilds T are
   sqrt(2j+1) U_x and sqrt(2j+1) V_x with those values between them;
3. truncation (reading 17): all singular values sorted in descending order
   (ties: smaller x first, then the block's own order); keep the leading
   ones while their dense count (SU(2): 2j+1 each, else 1) stays <= chi,
   and only those above cutoff times the largest; keep[x] = how many of
   block x were kept;
4. recast: U with legs (row legs..., bond) and V with legs (bond, column
   legs...).  The bond leg lists the labels x with keep[x] > 0, degeneracy
   keep[x]; it is incoming on U (U carries total label 0) and outgoing on V
   (V carries T's total), so contracting U's bond with V's rebuilds T's
   labels.  U's block (row tuple, x) = rows of U_x[:, :keep]; V's block
   (x, column tuple) = columns of V_x[:keep, :].  absorb = 1 multiplies U's
   columns by S, absorb = 2 V's rows.
"""
import itertools
from math import sqrt

import numpy as np

from . import su2 as su2m
from . import u1 as u1m
from . import z2f as z2fm


def _mod(group):
    return {"u1": u1m, "z2f": z2fm, "su2": su2m}[group]


def _key(group, legs, idx):
    """Fused label of `legs` at label positions `idx` (step 1)."""
    if group == "u1":
        return sum(l.dir * l.labels[i] for l, i in zip(legs, idx))
    if group == "su2":
        (l,), (i,) = legs, idx  # rank 2: the spin of the one row leg
        return l.labels[i]
    return sum(l.labels[i] for l, i in zip(legs, idx)) % 2


def _col_partner(group, total, y):
    """Row label x of the diagonal block that column label y belongs to."""
    if group == "su2":
        return y
    return total - y if group == "u1" else (total + y) % 2


def _weight(group, x):
    """Dense singular values one value of block x stands for."""
    return x + 1 if group == "su2" else 1


def _scale(group, x):
    return sqrt(x + 1) if group == "su2" else 1.0


def _positions(group, s):
    return tuple(s[0]) if group == "su2" else tuple(s)


def _enumerate(group, legs, partner):
    """{x: [(label tuple, first index, extent)]} over all tuples of `legs`."""
    groups = {}
    for idx in itertools.product(*[range(len(l.labels)) for l in legs]):
        x = partner(_key(group, legs, idx))
        ext = int(np.prod([l.degens[i] for l, i in zip(legs, idx)], dtype=np.int64))
        lst = groups.setdefault(x, [])
        first = lst[-1][1] + lst[-1][2] if lst else 0
        lst.append((idx, first, ext))
    return groups


def block_diagonal(group, T, nrow):
    """{x: (M_x, rows, cols)} for the x that have rows and columns (step 1)."""
    legs, total, data = T
    m = _mod(group)
    if group == "su2" and (len(legs) != 2 or nrow != 1):
        raise ValueError("SU(2): rank-2 tensors (the block-diagonal form)")
    data = np.asarray(data, dtype=np.float64)
    rl, cl = legs[:nrow], legs[nrow:]
    rows = _enumerate(group, rl, lambda k: k)
    cols = _enumerate(group, cl, lambda k: _col_partner(group, total, k))
    out = {}
    for x in sorted(set(rows) & set(cols)):
        mx = rows[x][-1][1] + rows[x][-1][2]
        nx = cols[x][-1][1] + cols[x][-1][2]
        out[x] = (np.zeros((mx, nx)), rows[x], cols[x])
    secs, offs, _ = m.layout(legs, total)
    for s, o in zip(secs, offs):
        s = _positions(group, s)
        rt, ct = tuple(s[:nrow]), tuple(s[nrow:])
        x = _key(group, rl, rt)
        M, rws, cls = out[x]
        r0, h = next((f, e) for t, f, e in rws if t == rt)
        c0, w = next((f, e) for t, f, e in cls if t == ct)
        M[r0:r0 + h, c0:c0 + w] = data[o:o + h * w].reshape(h, w)
    return out


def svd(group, T, nrow):
    """{x: (U_x, S_x, V_x)} (step 2; SU(2): the tensor-level factors and the
    dense singular values) and the block-diagonal form."""
    bd = block_diagonal(group, T, nrow)
    fac = {}
    for x, (M, _, _) in bd.items():
        U, S, V = np.linalg.svd(M, full_matrices=False)
        c = _scale(group, x)
        fac[x] = (U * c, S / c, V * c)
    return fac, bd


def truncation(S_by_x, chi=None, cutoff=0.0, group="u1"):
    """keep[x] (step 3)."""
    vals = [(-s, x, i) for x in sorted(S_by_x) for i, s in enumerate(S_by_x[x])]
    vals.sort()
    smax = -vals[0][0] if vals else 0.0
    keep = {x: 0 for x in S_by_x}
    n = 0
    for neg, x, i in vals:
        w = _weight(group, x)
        if chi is not None and n + w > chi:
            break
        if cutoff > 0.0 and -neg <= cutoff * smax:
            break
        keep[x] += 1
        n += w
    return keep


def bond_leg(group, keep, direction):
    m = _mod(group)
    xs = [x for x in sorted(keep) if keep[x] > 0]
    return m.Leg(xs, [keep[x] for x in xs], direction)


def factors(group, T, nrow, keep, absorb=0, fac=None):
    """(U, S_kept, V) as (legs, total, data) tensors and {x: kept values} (step 4)."""
    legs, total, data = T
    m = _mod(group)
    if fac is None:
        fac, bd = svd(group, T, nrow)
    else:
        bd = block_diagonal(group, T, nrow)
    rl, cl = legs[:nrow], legs[nrow:]
    bu, bv = bond_leg(group, keep, -1), bond_leg(group, keep, 1)
    legsU, legsV = list(rl) + [bu], [bv] + list(cl)
    totU = su2m.left_comb(2) if group == "su2" else 0
    totV = su2m.left_comb(2) if group == "su2" else total
    secsU, offsU, nU = m.layout(legsU, totU)
    secsV, offsV, nV = m.layout(legsV, totV)
    Ud, Vd = np.zeros(nU), np.zeros(nV)
    for s, o in zip(secsU, offsU):
        s = _positions(group, s)
        x = bu.labels[s[-1]]
        k = keep[x]
        U, S, _ = fac[x]
        r0, h = next((f, e) for t, f, e in bd[x][1] if t == tuple(s[:-1]))
        blk = U[r0:r0 + h, :k] * (S[:k] if absorb == 1 else 1.0)
        Ud[o:o + h * k] = blk.reshape(-1)
    for s, o in zip(secsV, offsV):
        s = _positions(group, s)
        x = bv.labels[s[0]]
        k = keep[x]
        _, S, V = fac[x]
        c0, w = next((f, e) for t, f, e in bd[x][2] if t == tuple(s[1:]))
        blk = V[:k, c0:c0 + w] * (S[:k, None] if absorb == 2 else 1.0)
        Vd[o:o + k * w] = blk.reshape(-1)
    kept = {x: fac[x][1][:keep[x]] for x in sorted(keep) if keep[x] > 0}
    return (legsU, totU, Ud), kept, (legsV, totV, Vd)


def matrix(group, T, nrow):
    """Dense matrix of T: the dense tensor with rows = legs 0..nrow-1 flattened."""
    legs, total, data = T
    d = _mod(group).embed(legs, total, data)
    r = int(np.prod([l.dim for l in legs[:nrow]], dtype=np.int64))
    return d.reshape(r, -1)


def dense_values(group, kept):
    """The kept singular values as the dense matrix has them, in the bond
    leg's dense order (SU(2): each value 2j+1 times, the m index fastest)."""
    return np.concatenate([np.repeat(kept[x], _weight(group, x)) for x in sorted(kept)])
