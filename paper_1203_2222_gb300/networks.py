"""Network-level compositions of the contraction: the ternary-MERA patch energy.

psi = (1 x 1 x u x 1 x 1)(w x w) t and E = <psi|h|psi> / <psi|psi> with h on
the two sites u outputs (a MERA patch of Ch. 7, built from U(1)-invariant
tensors), contracted through reduced density matrices so that psi is never
formed:

    rho_top = t (x) t*,   W1 = w w* over (a1, a2),   W2 = w w* over (b2, b3),
    rho     = (rho_top W1) W2  on the bond (a3, b1),
    rho'    = (u rho) u*,      E = <rho', h> / <rho', 1>.

A conjugate is the same (real) block data under the structure with every
leg's direction reversed, so autograd sums the contributions of u and u*,
w and w* into one gradient.  With ``checkpoint`` the environment rho is
recomputed in the backward pass instead of keeping rho_top, W1, W2 and the
intermediate in memory (torch.utils.checkpoint around its contractions).
"""
import numpy as np
import torch

from . import symtensor as st


def reversed_legs(legs):
    return [(l, d, -dr) for (l, d, dr) in legs]


def mera_structures(spec):
    """Structures of t, w, u, h, their conjugates (t*, w*, u*, h*) and the identity operator 1*."""
    S = {}
    for n in ("t", "w", "u", "h"):
        S[n] = st.Structure(st.U1, spec[n])
        S[n + "*"] = st.Structure(st.U1, reversed_legs(spec[n]))
    S["1*"] = S["h*"]
    return S


def operator_blocks(S, entry):
    """Block data of a two-site operator op[c, d, c', d'] with structure S from entry(qc, tc, qd, td, qc', tc', qd', td')."""
    pos, offs = S.sectors()  # label positions of every leg per sector
    out = np.zeros(S.numel)
    for s in range(S.nsec):
        q = [S.legs[i][0][pos[s][i]] for i in range(4)]
        dims = [S.legs[i][1][pos[s][i]] for i in range(4)]
        blk = np.zeros(dims)
        for idx in np.ndindex(*dims):
            blk[idx] = entry(q[0], idx[0], q[1], idx[1], q[2], idx[2], q[3], idx[3])
        out[offs[s]:offs[s + 1]] = blk.reshape(-1)
    return out


def mera_h_and_identity(S, spec):
    from .synthetic import mera_h_entry
    h = operator_blocks(S["h*"], lambda *a: mera_h_entry(spec["delta"], *a))
    one = operator_blocks(S["1*"], lambda qc, tc, qd, td, qc2, tc2, qd2, td2:
                          1.0 if (qc, tc, qd, td) == (qc2, tc2, qd2, td2) else 0.0)
    return h, one


def _contract(SA, a, SB, b, pa, pb):
    plan = st.contract_plan(SA, SB, pa, pb, st._precision(a.dtype))
    return st._Contract.apply(plan, a, b), plan.out


def mera_environment(S, t, w):
    """rho[a3, a3', b1, b1'] of the bond under u (block data) and its structure."""
    rho_top, Sr = _contract(S["t"], t, S["t*"], t, [], [])
    W1, S1 = _contract(S["w"], w, S["w*"], w, [1, 2], [1, 2])
    W2, S2 = _contract(S["w"], w, S["w*"], w, [2, 3], [2, 3])
    X, Sx = _contract(Sr, rho_top, S1, W1, [0, 2], [0, 2])  # (S, S', a3, a3')
    return _contract(Sx, X, S2, W2, [0, 1], [0, 2])        # (a3, a3', b1, b1')


def mera_energy(S, t, w, u, h, one, checkpoint=False):
    """E = <psi|h|psi> / <psi|psi> (autograd-aware in t, w and u)."""
    if checkpoint:
        Srho = mera_environment_structure(S, t.dtype)
        # the environment draws no random numbers: no RNG state to save, which
        # also keeps the step capturable in a CUDA graph
        rho = torch.utils.checkpoint.checkpoint(lambda tt, ww: mera_environment(S, tt, ww)[0], t, w,
                                                use_reentrant=False, preserve_rng_state=False)
    else:
        rho, Srho = mera_environment(S, t, w)
    Y, Sy = _contract(S["u"], u, Srho, rho, [2, 3], [0, 2])       # (c, d, a3', b1')
    rhop, Sp = _contract(Sy, Y, S["u*"], u, [2, 3], [2, 3])       # (c, d, c', d')
    num, _ = _contract(Sp, rhop, S["h*"], h, [0, 1, 2, 3], [0, 1, 2, 3])
    den, _ = _contract(Sp, rhop, S["1*"], one, [0, 1, 2, 3], [0, 1, 2, 3])
    return num[0] / den[0]


def mera_environment_structure(S, dtype):
    """Structure of the environment rho (from the cached plans, no data)."""
    prec = st._precision(dtype)
    Sr = st.contract_plan(S["t"], S["t*"], [], [], prec).out
    S1 = st.contract_plan(S["w"], S["w*"], [1, 2], [1, 2], prec).out
    S2 = st.contract_plan(S["w"], S["w*"], [2, 3], [2, 3], prec).out
    Sx = st.contract_plan(Sr, S1, [0, 2], [0, 2], prec).out
    return st.contract_plan(Sx, S2, [0, 1], [0, 2], prec).out
