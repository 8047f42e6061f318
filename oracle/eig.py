"""Blockwise symmetric eigendecomposition, plain FP64 (oracle; test infrastructure only).

Ch. 5, "Factorization of a matrix" (Eq. spectral; and, for symmetric
tensors, the statement after Eq. svd1 that a spectral decomposition is
obtained by the analogous factorization of the blocks): a symmetric tensor
seen as a square matrix is block diagonal in the label it carries, so its
eigendecomposition is that of every diagonal block, taken independently.
The steps, in that order:

1. block-diagonal form, as for the SVD (oracle.svd step 1).  The matrix is
   square: the column legs are the row legs reversed (same labels and
   degeneracies, opposite directions, same order) and the total label is 0,
   so that M_x's row and column tuples are the same list;
2. M_x is taken as symmetric: its eigendecomposition is that of the
   symmetric part (M_x + M_x^T) / 2 (numpy's eigh), M_x = Q diag(lam) Q^T,
   the eigenpairs ordered by |lam| descending (ties: the larger lam first,
   then numpy's order).  SU(2) (rank 2, one incoming and one outgoing leg):
   with the block normalisation of reading 5 the dense matrix is the direct
   sum of sgn_j M_x / sqrt(2j+1) (x) 1_{2j+1}, sgn_j = (-1)^{2j} when the row
   leg is incoming and +1 otherwise (pinned against the dense matrix), so its
   eigenvalues are sgn_j lam / sqrt(2j+1), each 2j+1 times; the factors whose
   contraction rebuilds T are U = sqrt(2j+1) Q and V = sgn_j sqrt(2j+1) Q^T
   with those values between them;
3. truncation: the SVD's rule (oracle.svd.truncation) on |lam|, which for a
   symmetric matrix are its singular values, so that a truncation to chi
   keeps the best rank-chi approximation (Eckart-Young);
4. recast: oracle.svd.factors with these (U_x, lam_x, V_x).
"""
from math import sqrt

import numpy as np

from . import svd as svdm


def check_square(group, T, nrow):
    """The column legs are the row legs reversed and the total label is 0."""
    legs, total, _ = T
    if len(legs) != 2 * nrow:
        raise ValueError("eigendecomposition needs rank = 2 nrow")
    for a, b in zip(legs[:nrow], legs[nrow:]):
        if a.labels != b.labels or a.degens != b.degens or a.dir != -b.dir:
            raise ValueError("column legs must be the row legs reversed")
    if group != "su2" and total != 0:
        raise ValueError("eigendecomposition needs total label 0")


def sign(group, legs, x):
    """sgn_x of step 2 (1 outside SU(2))."""
    if group != "su2":
        return 1.0
    return -1.0 if (legs[0].dir == -1 and x % 2) else 1.0


def eig(group, T, nrow):
    """{x: (U_x, lam_x, V_x)} (step 2; SU(2): the tensor-level factors and
    the dense eigenvalues) and the block-diagonal form."""
    check_square(group, T, nrow)
    bd = svdm.block_diagonal(group, T, nrow)
    fac = {}
    for x, (M, _, _) in bd.items():
        assert M.shape[0] == M.shape[1]
        lam, Q = np.linalg.eigh(0.5 * (M + M.T))
        order = sorted(range(len(lam)), key=lambda i: (-abs(lam[i]), -lam[i], i))
        lam, Q = lam[order], Q[:, order]
        c = sqrt(x + 1) if group == "su2" else 1.0
        s = sign(group, T[0], x)
        fac[x] = (Q * c, s * lam / c, s * c * Q.T)
    return fac, bd


def truncation(L_by_x, chi=None, cutoff=0.0, group="u1"):
    """keep[x] (step 3)."""
    return svdm.truncation({x: np.abs(v) for x, v in L_by_x.items()}, chi, cutoff, group=group)


def factors(group, T, nrow, keep, absorb=0, fac=None):
    """(U, lam_kept, V) as (legs, total, data) tensors and {x: kept values} (step 4)."""
    if fac is None:
        fac, _ = eig(group, T, nrow)
    return svdm.factors(group, T, nrow, keep, absorb=absorb, fac=fac)
