"""Energy of a ternary-MERA patch, plain FP64 definition (dense).

Oracle; test infrastructure only.  The thesis's MERA chapter works with
symmetric disentanglers and isometries (Ch. 7: a MERA built from U(1)- or
SU(2)-invariant tensors) but prints no closed network.  The patch used here:

    psi = (1 x 1 x u x 1 x 1) (w x w) t
    E   = <psi| h |psi> / <psi|psi>,   h acting on the two sites u outputs

with t[T, S] the top, w[T, a1, a2, a3] the isometry (upper leg T), u[c, d,
a, b] the disentangler on (a3 of the first w, a1 of the second) and
h[c, d, c', d'] = <c d| h |c' d'>.  All tensors are real, so a conjugate is
the same array.

``energy`` contracts through reduced density matrices (never forming psi; each step
is a two-operand einsum evaluated with BLAS):
    rho_top = t (x) t,  W1 = w w over (a1, a2),  W2 = w w over (b2, b3),
    rho     = rho_top W1 W2  on (a3, b1),   rho' = u rho u^T,
    E       = sum(rho' h) / trace(rho').
``energy_brute`` forms psi explicitly (tiny bond dimensions only); the two
must agree, which pins the contraction order and every index of ``energy``.
"""
import numpy as np


def energy(t, w, u, h):
    rho_top = np.einsum("TS,UV->TSUV", t, t, optimize=True)
    W1 = np.einsum("Tabc,Uabd->TcUd", w, w, optimize=True)  # (T, a3, T', a3')
    W2 = np.einsum("Sabc,Vdbc->SaVd", w, w, optimize=True)  # (S, b1, S', b1')
    X = np.einsum("TSUV,TcUd->SVcd", rho_top, W1, optimize=True)  # (S, S', a3, a3')
    rho = np.einsum("SVcd,SaVb->cadb", X, W2, optimize=True)  # (a3, b1, a3', b1')
    Y = np.einsum("cdab,abef->cdef", u, rho, optimize=True)  # (c, d, a3', b1')
    rhop = np.einsum("cdef,ghef->cdgh", Y, u, optimize=True)  # (c, d, c', d')
    num = float(np.einsum("cdgh,cdgh->", rhop, h))
    den = float(np.einsum("cdcd->", rhop))
    return num / den


def energy_brute(t, w, u, h):
    psi0 = np.einsum("TS,Tabc,Sdef->abcdef", t, w, w)
    psi = np.einsum("xycd,abcdef->abxyef", u, psi0)
    hpsi = np.einsum("xyzw,abzwef->abxyef", h, psi)
    return float(np.sum(psi * hpsi) / np.sum(psi * psi))


def h_dense(legs, entry):
    """Dense h[c, d, c', d'] on the dense spaces of four U(1) legs from an
    entry function entry(qc, tc, qd, td, qc', tc', qd', td')."""
    def basis(leg):
        return [(q, t) for q, d in zip(leg.labels, leg.degens) for t in range(d)]
    b = [basis(l) for l in legs]
    H = np.zeros([len(x) for x in b])
    for i, (qc, tc) in enumerate(b[0]):
        for j, (qd, td) in enumerate(b[1]):
            for k, (qc2, tc2) in enumerate(b[2]):
                qd2 = qc + qd - qc2
                for l, (q4, td2) in enumerate(b[3]):
                    if q4 == qd2:
                        H[i, j, k, l] = entry(qc, tc, qd, td, qc2, tc2, qd2, td2)
    return H
