"""Dense brute-force operations on symmetric tensors (oracle; test infrastructure only).

Each operation is its plain dense definition applied to the embedded tensors
(``u1.embed`` / ``su2.embed``), followed by extraction into the result's
block layout.  No symmetry is used in the arithmetic.

* ``contract``: Ch. 5, Eq. tensormult -- sum over paired dense indices; a
  paired index must be outgoing in one tensor and incoming in the other with
  the same charge/spin content.  Result legs: free legs of A (in order) then
  free legs of B (in order), directions kept.  U(1) total charge QA + QB;
  SU(2) result in the caller's tree (default: the comb over A's free legs
  and the comb over B's free legs joined at the root).
* ``contract_grad``: the gradient of <dC, C> with respect to the blocks of A
  and B.  Embedding has orthonormal columns on the invariant subspace, so the
  block gradient is the extraction of the dense gradient.
* ``permute``: Ch. 5, Eq. permute, T'[i_{p(0)}, ..] = T[i_0, ..], then
  extraction in the requested tree (PERMUTE of Ch. 6).
* ``fuse``: Ch. 5, Eq. fuse with the fusing tensor of Eq. basischange1 (U(1):
  the 0/1 map alone); incoming legs lose their cups first and the fused leg
  gets one (Ch. 6, reshape of indices carrying cups).
* SU(2) x U(1) ("su2u1", oracle/su2u1.py) runs the SU(2) branches with
  composite legs; a tensor's second member is (tree, total charge).
"""
import numpy as np

from . import su2 as su2m
from . import su2u1 as su2u1m
from . import u1 as u1m
from . import z2f as z2fm


def _mod(group):
    return {"u1": u1m, "su2": su2m, "su2u1": su2u1m}[group]


def _with_total(group, tree, total):
    """The second member of a tensor: U(1) total, SU(2) tree, SU(2) x U(1) (tree, Q)."""
    return (tree, total) if group == "su2u1" else tree


def _charge(group, t):
    return t[1] if group == "su2u1" else 0


def comb_pair_tree(na, nb):
    """Comb over legs 0..na-1 and comb over na..na+nb-1 joined at the root."""
    k = na + nb
    nodes = []
    top_a = 0 if na >= 1 else None
    for i in range(1, na):
        nodes.append((top_a, i))
        top_a = k + len(nodes) - 1
    top_b = na if nb >= 1 else None
    for i in range(na + 1, na + nb):
        nodes.append((top_b, i))
        top_b = k + len(nodes) - 1
    if na >= 1 and nb >= 1:
        nodes.append((top_a, top_b))
    return nodes


def _free(rank, pairs):
    return [i for i in range(rank) if i not in pairs]


def contract_dense(Ad, Bd, pairsA, pairsB):
    """C[freeA..., freeB...] = sum_c A[.., c, ..] B[.., c, ..] (library tensordot)."""
    return np.tensordot(Ad, Bd, axes=(list(pairsA), list(pairsB)))


def result_legs(legsA, legsB, pairsA, pairsB):
    for a, b in zip(pairsA, pairsB):
        la, lb = legsA[a], legsB[b]
        assert la.labels == lb.labels and la.degens == lb.degens and la.dir == -lb.dir, \
            "contracted legs must have equal content and opposite directions"
    return ([legsA[i] for i in _free(len(legsA), pairsA)]
            + [legsB[i] for i in _free(len(legsB), pairsB)])


def contract(group, A, B, pairsA, pairsB, tree_c=None):
    """A, B = (legs, total_or_tree, data).  Returns (legsC, total_or_tree, data, resid).
    Fermion parity ("z2f"): oracle/z2f.py, the contraction with its swap signs."""
    if group == "z2f":
        return z2fm.contract(A, B, pairsA, pairsB)
    m = _mod(group)
    legsA, tA, a = A
    legsB, tB, b = B
    legsC = result_legs(legsA, legsB, pairsA, pairsB)
    Cd = contract_dense(m.embed(legsA, tA, a), m.embed(legsB, tB, b), pairsA, pairsB)
    if group == "u1":
        tC = tA + tB
    else:
        na = len(legsA) - len(pairsA)
        tC = _with_total(group, tree_c if tree_c is not None else comb_pair_tree(na, len(legsC) - na),
                         _charge(group, tA) + _charge(group, tB))
    c, resid = m.extract(legsC, tC, Cd)
    return legsC, tC, c, resid


def contract_grad(group, A, B, pairsA, pairsB, dC, tree_c=None):
    """(dA, dB) blocks of the gradient of <dC, contract(A, B)>."""
    if group == "z2f":
        return z2fm.contract_grad(A, B, pairsA, pairsB, dC)
    m = _mod(group)
    legsA, tA, a = A
    legsB, tB, b = B
    legsC = result_legs(legsA, legsB, pairsA, pairsB)
    na = len(legsA) - len(pairsA)
    nb = len(legsB) - len(pairsB)
    if group == "u1":
        tC = tA + tB
    else:
        tC = _with_total(group, tree_c if tree_c is not None else comb_pair_tree(na, nb),
                         _charge(group, tA) + _charge(group, tB))
    Ad, Bd, dCd = m.embed(legsA, tA, a), m.embed(legsB, tB, b), m.embed(legsC, tC, dC)
    freeA, freeB = _free(len(legsA), pairsA), _free(len(legsB), pairsB)
    # dA[freeA, c] = sum_{freeB} dC[freeA, freeB] B[c, freeB]
    g = np.tensordot(dCd, Bd, axes=(list(range(na, na + nb)), freeB))
    # g axes: freeA (A order) then B's contracted axes in ascending B order
    bc = sorted(pairsB)
    pos = {}
    for i, ax in enumerate(freeA):
        pos[ax] = i
    for a_ax, b_ax in zip(pairsA, pairsB):
        pos[a_ax] = na + bc.index(b_ax)
    dAd = np.transpose(g, [pos[i] for i in range(len(legsA))])
    # dB[c, freeB] = sum_{freeA} A[freeA, c] dC[freeA, freeB]
    h = np.tensordot(Ad, dCd, axes=(freeA, list(range(na))))
    ac = sorted(pairsA)
    pos = {}
    for a_ax, b_ax in zip(pairsA, pairsB):
        pos[b_ax] = ac.index(a_ax)
    for i, ax in enumerate(freeB):
        pos[ax] = len(pairsA) + i
    dBd = np.transpose(h, [pos[i] for i in range(len(legsB))])
    dA, ra = m.extract(legsA, tA, dAd)
    dB, rb = m.extract(legsB, tB, dBd)
    return dA, dB, max(ra, rb)


def permute(group, T, perm, tree_out=None):
    """Output leg n is input leg perm[n]; SU(2) result in tree_out (default comb)."""
    if group == "z2f":
        return z2fm.permute(T, perm)
    m = _mod(group)
    legs, t, data = T
    legs2 = [legs[p] for p in perm]
    d = np.transpose(m.embed(legs, t, data), list(perm))
    if group == "u1":
        t2 = t
    else:
        t2 = _with_total(group, tree_out if tree_out is not None else su2m.left_comb(len(legs2)), _charge(group, t))
    out, resid = m.extract(legs2, t2, d)
    return legs2, t2, out, resid


def fuse(group, T, first, tree_out=None):
    """Fuse adjacent legs (first, first+1) of equal direction into one leg."""
    if group == "z2f":
        return z2fm.fuse(T, first)
    m = _mod(group)
    legs, t, data = T
    la, lb = legs[first], legs[first + 1]
    assert la.dir == lb.dir, "fused legs must have equal directions"
    d = m.embed(legs, t, data)
    if group == "u1":
        ld, X = u1m.fused_leg(la, lb)[0], u1m.fusion_matrix(la, lb)[1]
        out_d = np.tensordot(d, X, axes=([first, first + 1], [0, 1]))
        out_d = np.moveaxis(out_d, -1, first)
        legs2 = legs[:first] + [ld] + legs[first + 2:]
        res, resid = u1m.extract(legs2, t, out_d)
        return legs2, t, res, resid
    if la.dir == -1:
        # detach the cups (cap inverts cup), fuse as outgoing, re-attach
        d = np.moveaxis(np.tensordot(m.leg_cap(la), d, axes=([1], [first])), 0, first)
        d = np.moveaxis(np.tensordot(m.leg_cap(lb), d, axes=([1], [first + 1])), 0, first + 1)
    ld, U = m.fusing_tensor(la.dual() if la.dir == -1 else la,
                            lb.dual() if lb.dir == -1 else lb)
    out_d = np.tensordot(d, U, axes=([first, first + 1], [0, 1]))
    out_d = np.moveaxis(out_d, -1, first)
    if la.dir == -1:
        ld = ld.dual()
        out_d = np.moveaxis(np.tensordot(m.leg_cup(ld), out_d, axes=([1], [first])), 0, first)
    legs2 = legs[:first] + [ld] + legs[first + 2:]
    t2 = _with_total(group, tree_out if tree_out is not None else su2m.left_comb(len(legs2)), _charge(group, t))
    res, resid = m.extract(legs2, t2, out_d)
    return legs2, t2, res, resid
