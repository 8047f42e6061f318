"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module holds leg structures (charges or doubled spins, degeneracies,
directions) and seeded N(0,1) draws only -- none of the method's arithmetic.
Each side builds its own tensors from these plain tuples and asks for as many
random values as its own sector enumeration says the tensor holds.

A leg spec is ``(labels, degens, dir)`` with ``dir = +1`` ('out') or ``-1``
('in'); U(1) labels are charges, SU(2) labels are doubled spins 2j.

Workload shapes (all seeds are ``1234 + index``):

* ``u1_pairwise``   two rank-4 U(1) tensors, charges -2..2, degeneracies
  uniform in 1..4 per leg, total charge 0; contract A's legs 2,3 with B's
  legs 0,1 (B's first two legs are A's last two, reversed).
* ``u1_mps_heff``   MPS effective-Hamiltonian apply (L.A).W.R with bond
  D = 2048 over charges -20..20 (Gaussian degeneracy profile, sigma 6),
  physical leg {0:1, 1:1}, MPO leg {-1:1, 0:3, +1:1}.
* ``u1_two_site_batch``  n independent two-site effective-Hamiltonian
  applies Y = (((L.theta).W1).W2).R, problem i seeded by seed * 1000 + i:
  bond D_i = round(exp(U(ln 64, ln 1024))) over charges -12..12 with the
  Gaussian profile above (sigma_i ~ U(2, 6)), physical legs {0:1, 1:1},
  MPO legs {-1:1, 0:3, +1:1}.
* ``u1_mera``  a patch of a ternary U(1) MERA: bond chi = 48 over charges
  -4..4 (degeneracy 5, plus 1 on q = -1, 0, 1), a charge-0 top t (out, out),
  two copies of the isometry w (upper leg in, three lower legs out) and a
  disentangler u (two lower legs in, two upper legs out) on the middle bond;
  h is the XXZ-like two-site term given entry by entry (``mera_h_entry``).
* ``u1_two_site_svd``  the two-site tensor theta[a, s1, s2, b] of that chain
  (D = 2048, total charge 0) as the matrix (a, s1) x (s2, b), truncated to
  chi = 2048 singular values.
* ``u1_two_site_eig``  the reduced density matrix theta theta* of that
  tensor over (a, s1), eigendecomposed and truncated to chi = 2048.
* ``su2u1_mps_heff``  the MPS chain with SU(2) x U(1) legs (labels (q, 2j)):
  a Hubbard-like site {(0,0), (1,1), (2,0)}, MPO {(-1,1):2, (0,0):3, (1,1):2},
  about 1024 bond multiplets over q = -8..8, 2j = 0..4 (2j = q mod 2).
* ``z2f_mps_heff``  the MPS chain above with fermion-parity legs: bond
  D = 2048 as {0: 1024, 1: 1024}, physical {0:1, 1:1}, MPO {0:3, 1:2}.
* ``su2_recouple``  rank-4 SU(2) tensors, every leg with 2j = 0..8 and
  degeneracies uniform in 1..dmax (32 at full size); A has all legs out in
  the comb tree, is permuted (0,2,1,3) into the matrix tree and its legs 1,3
  are contracted with a tensor B whose first two legs are their duals.
"""
import math

import numpy as np


def normal(seed, n, stream=0):
    """n draws of N(0,1) in float64 from PCG64(seed), sub-stream ``stream``."""
    ss = np.random.SeedSequence([int(seed), int(stream)])
    return np.random.Generator(np.random.PCG64(ss)).standard_normal(int(n))


def uniform_int(seed, lo, hi, n, stream=0):
    ss = np.random.SeedSequence([int(seed), int(stream), 7])
    return np.random.Generator(np.random.PCG64(ss)).integers(lo, hi + 1, size=n).tolist()


def gaussian_degeneracies(D, qmin, qmax, sigma):
    """Degeneracies over charges qmin..qmax summing to D, profile exp(-q^2/(2 sigma^2)).

    d_q = max(1, round-half-even(D g_q / sum g)); the remainder is fixed by
    +-1 steps on charges in order of increasing |q|, negative first.
    """
    qs = list(range(qmin, qmax + 1))
    g = [math.exp(-q * q / (2.0 * sigma * sigma)) for q in qs]
    sg = sum(g)
    d = [max(1, int(round(D * gi / sg))) for gi in g]
    order = sorted(range(len(qs)), key=lambda i: (abs(qs[i]), qs[i]))
    rem = D - sum(d)
    i = 0
    while rem != 0:
        j = order[i % len(order)]
        step = 1 if rem > 0 else -1
        if d[j] + step >= 1:
            d[j] += step
            rem -= step
        i += 1
    return qs, d


def u1_pairwise(seed=1234):
    """Two rank-4 U(1) tensors and the contracted pairs (dense dim per leg <= 20)."""
    qs = [-2, -1, 0, 1, 2]
    dl = [uniform_int(seed, 1, 4, 5, stream=l) for l in range(6)]
    A = [(qs, dl[0], 1), (qs, dl[1], 1), (qs, dl[2], -1), (qs, dl[3], -1)]
    B = [(qs, dl[2], 1), (qs, dl[3], 1), (qs, dl[4], -1), (qs, dl[5], -1)]
    return {"group": "u1", "A": A, "QA": 0, "B": B, "QB": 0,
            "pairsA": [2, 3], "pairsB": [0, 1], "seedA": seed, "seedB": seed + 1}


def u1_mps_heff(D=2048, qmax=20, sigma=6.0, seed=1235):
    """Legs of L[a,w,a'], A[a',s',b'], W[w,s,s',w2], R[b,w2,b'] (all total charge 0).

    Directions: A (in, in, out); L (in, in, out); W (out, in, out, in);
    R (out, out, in).  Contraction order ((L.A).W).R:
      L.A    over L2 <-> A0            -> T1[a, w, s', b']   (in, in, in, out)
      T1.W   over T1(1,2) <-> W(0,2)   -> T2[a, b', s, w2]   (in, out, in, in)
      T2.R   over T2(1,3) <-> R(2,1)   -> Y[a, s, b]         (in, in, out)
    """
    qs, d = gaussian_degeneracies(D, -qmax, qmax, sigma)
    bond_in, bond_out = (qs, d, -1), (qs, d, 1)
    wq, wd = [-1, 0, 1], [1, 3, 1]
    phys_in, phys_out = ([0, 1], [1, 1], -1), ([0, 1], [1, 1], 1)
    L = [bond_in, (wq, wd, -1), bond_out]
    A = [bond_in, phys_in, bond_out]
    W = [(wq, wd, 1), phys_in, phys_out, (wq, wd, -1)]
    R = [bond_out, (wq, wd, 1), bond_in]
    return {"group": "u1", "L": L, "A": A, "W": W, "R": R,
            "steps": [((1, 2), (0, 2)), ((1, 3), (2, 1))],
            "seeds": {"L": seed, "A": seed + 100, "W": seed + 200, "R": seed + 300},
            "D": D}


def u1_two_site_svd(D=2048, qmax=20, sigma=6.0, seed=1240):
    """Legs of the two-site tensor theta[a, s1, s2, b] of the MPS chain above
    (bond D over charges -qmax..qmax, Gaussian profile; directions in, in,
    in, out; total charge 0), split as a matrix (a, s1) x (s2, b) and
    truncated back to chi = D singular values: the truncation step that
    follows an effective-Hamiltonian apply."""
    qs, d = gaussian_degeneracies(D, -qmax, qmax, sigma)
    phys_in = ([0, 1], [1, 1], -1)
    theta = [(qs, d, -1), phys_in, phys_in, (qs, d, 1)]
    return {"group": "u1", "theta": theta, "nrow": 2, "chi": D, "seed": seed, "D": D}


def u1_two_site_eig(D=2048, qmax=20, sigma=6.0, seed=1240):
    """Legs of the two-site tensor theta of ``u1_two_site_svd``; the workload
    is the reduced density matrix rho[(a, s1), (a', s1')] = sum over (s2, b)
    of theta theta* (legs a, s1 incoming, a', s1' outgoing, total 0), whose
    eigendecomposition truncated to chi = D eigenvalues is the density-matrix
    form of the same truncation step."""
    w = u1_two_site_svd(D, qmax, sigma, seed)
    w["pairs"] = ([2, 3], [2, 3])
    return w


def su2u1_mps_heff(D=1024, qmax=8, sigma=3.0, seed=1241):
    """Legs of the MPS chain ((L.A).W).R with SU(2) x U(1) legs (labels (q, 2j)).

    A Hubbard-like chain: physical leg {(0,0):1, (1,1):1, (2,0):1} (empty,
    singly occupied with spin 1/2, doubly occupied), MPO leg
    {(-1,1):2, (0,0):3, (1,1):2} (hopping channels carrying charge -1 or +1
    and spin 1/2, and three scalar channels).  The bond carries labels
    (q, 2j) for q = -qmax..qmax and 2j = 0..4 with 2j = q mod 2, degeneracy
    max(1, round-half-even(D w / sum w)) with w = exp(-q^2 / (2 sigma^2)) s_j,
    s = (1, 1, 0.6, 0.5, 0.25) for 2j = 0..4 (about D multiplets in all).
    Directions and contraction order as ``u1_mps_heff``; totals 0.
    """
    sj = [1.0, 1.0, 0.6, 0.5, 0.25]
    labs = [(q, j2) for q in range(-qmax, qmax + 1) for j2 in range(5) if (j2 - q) % 2 == 0]
    w = [math.exp(-q * q / (2.0 * sigma * sigma)) * sj[j2] for q, j2 in labs]
    tot = sum(w)
    d = [max(1, int(round(D * x / tot))) for x in w]
    bond_in, bond_out = (labs, d, -1), (labs, d, 1)
    phys = [(0, 0), (1, 1), (2, 0)]
    phys_in, phys_out = (phys, [1, 1, 1], -1), (phys, [1, 1, 1], 1)
    wl, wd = [(-1, 1), (0, 0), (1, 1)], [2, 3, 2]
    L = [bond_in, (wl, wd, -1), bond_out]
    A = [bond_in, phys_in, bond_out]
    W = [(wl, wd, 1), phys_in, phys_out, (wl, wd, -1)]
    R = [bond_out, (wl, wd, 1), bond_in]
    return {"group": "su2u1", "L": L, "A": A, "W": W, "R": R,
            "steps": [((1, 2), (0, 2)), ((1, 3), (2, 1))],
            "seeds": {"L": seed, "A": seed + 100, "W": seed + 200, "R": seed + 300},
            "D": D}


def z2f_mps_heff(D=2048, seed=1239):
    """Legs of the fermionic MPS effective-Hamiltonian apply ((L.A).W).R.

    Fermion-parity legs (labels 0 even, 1 odd): bond D split evenly between
    the two parities, physical leg {0:1, 1:1} (an empty or occupied fermion
    site), MPO leg {0:3, 1:2} (three even channels -- identity, number,
    identity -- and two odd ones carrying a creation or annihilation
    operator, as in a hopping MPO).  Directions and contraction order as
    ``u1_mps_heff``; every tensor has total parity 0.
    """
    bond_in, bond_out = ([0, 1], [D // 2, D - D // 2], -1), ([0, 1], [D // 2, D - D // 2], 1)
    wq, wd = [0, 1], [3, 2]
    phys_in, phys_out = ([0, 1], [1, 1], -1), ([0, 1], [1, 1], 1)
    L = [bond_in, (wq, wd, -1), bond_out]
    A = [bond_in, phys_in, bond_out]
    W = [(wq, wd, 1), phys_in, phys_out, (wq, wd, -1)]
    R = [bond_out, (wq, wd, 1), bond_in]
    return {"group": "z2f", "L": L, "A": A, "W": W, "R": R,
            "steps": [((1, 2), (0, 2)), ((1, 3), (2, 1))],
            "seeds": {"L": seed, "A": seed + 100, "W": seed + 200, "R": seed + 300},
            "D": D}


def su2_recouple(dmax=32, jmax2=8, seed=1236):
    """Legs of the SU(2) recoupling contraction (A all out; B = duals + 2 out legs)."""
    spins = list(range(0, jmax2 + 1))
    dl = [uniform_int(seed, 1, dmax, len(spins), stream=l) for l in range(6)]
    A = [(spins, dl[l], 1) for l in range(4)]
    B = [(spins, dl[1], -1), (spins, dl[3], -1), (spins, dl[4], 1), (spins, dl[5], 1)]
    return {"group": "su2", "A": A, "B": B, "perm": [0, 2, 1, 3],
            "pairsA": [1, 3], "pairsB": [0, 1], "seedA": seed, "seedB": seed + 1}


def u1_two_site_batch(n=512, seed=1238, dmin=64, dmax=1024, qmax=12):
    """Legs of n two-site problems L[a,w,a'] theta[a',s1',s2',b'] W1 W2 R[b,w'',b'].

    Directions: L (in, in, out), theta (in, in, in, out), W (out, in, out, in),
    R (out, out, in).  Contraction chain per problem:
      T1 = L.theta   over L2 <-> theta0          -> [a, w, s1', s2', b']
      T2 = T1.W1     over T1(1,2) <-> W1(0,2)    -> [a, s2', b', s1, w']
      T3 = T2.W2     over T2(1,4) <-> W2(2,0)    -> [a, b', s1, s2, w'']
      Y  = T3.R      over T3(1,4) <-> R(2,1)     -> [a, s1, s2, b]
    """
    wq, wd = [-1, 0, 1], [1, 3, 1]
    phys_in, phys_out = ([0, 1], [1, 1], -1), ([0, 1], [1, 1], 1)
    probs = []
    for i in range(n):
        rng = np.random.default_rng(seed * 1000 + i)
        D = int(round(math.exp(rng.uniform(math.log(dmin), math.log(dmax)))))
        sigma = float(rng.uniform(2.0, 6.0))
        qs, d = gaussian_degeneracies(D, -qmax, qmax, sigma)
        bond_in, bond_out = (qs, d, -1), (qs, d, 1)
        probs.append({
            "D": D, "sigma": sigma,
            "L": [bond_in, (wq, wd, -1), bond_out],
            "theta": [bond_in, phys_in, phys_in, bond_out],
            "W": [(wq, wd, 1), phys_in, phys_out, (wq, wd, -1)],
            "R": [bond_out, (wq, wd, 1), bond_in],
            "seed": seed * 1000 + i,
        })
    steps = [("L", "theta", [2], [0]), (None, "W", [1, 2], [0, 2]), (None, "W", [1, 4], [2, 0]),
             (None, "R", [1, 4], [2, 1])]
    return {"group": "u1", "problems": probs, "steps": steps}


def u1_mera(chi_extra=1, qmax=4, deg=5, delta=0.8, seed=1237):
    """Legs of the MERA patch: t[T, S], w[T, a1, a2, a3], u[c, d, a, b], h[c, d, c', d'].

    chi = deg * (2 qmax + 1) + chi_extra * 3 (48 by default): degeneracy
    ``deg`` on every charge plus ``chi_extra`` on q = -1, 0, 1.  h acts on the
    two middle sites (w1's a3 and w2's a1 after u): upper legs c, d (out),
    lower legs c', d' (in).
    """
    qs = list(range(-qmax, qmax + 1))
    d = [deg + (chi_extra if abs(q) <= 1 else 0) for q in qs]
    out_, in_ = (qs, d, 1), (qs, d, -1)
    return {"group": "u1", "chi": sum(d), "delta": delta,
            "t": [out_, out_], "w": [in_, out_, out_, out_], "u": [out_, out_, in_, in_],
            "h": [out_, out_, in_, in_],
            "seeds": {"t": seed, "w": seed + 1, "u": seed + 2}}


def mera_h_entry(delta, qc, tc, qd, td, qc2, tc2, qd2, td2):
    """<c d| h |c' d'> for h = (S+ S- + S- S+) / 2 + delta Sz Sz on two sites.

    Sz = diag(q); S+ raises the charge by one and keeps the degeneracy index
    (zero where the target charge has fewer states, which the caller's index
    range already excludes).  Charges and indices of the upper legs c, d and
    of the lower legs c', d'.
    """
    v = 0.0
    if qc == qc2 and qd == qd2 and tc == tc2 and td == td2:
        v += delta * qc2 * qd2
    if tc == tc2 and td == td2 and ((qc == qc2 + 1 and qd == qd2 - 1) or (qc == qc2 - 1 and qd == qd2 + 1)):
        v += 0.5
    return v
