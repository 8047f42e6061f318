"""Pins of the oracle's MERA-patch energy against brute force and closed forms."""
import numpy as np

from oracle import mera, u1
from paper_1203_2222_gb300 import synthetic


def test_density_matrix_route_equals_brute_force():
    # psi formed explicitly (tiny bond dimension) against the reduced-density
    # contraction order the oracle uses at full size
    rng = np.random.default_rng(0)
    for chi in (2, 3):
        t = rng.standard_normal((chi, chi))
        w = rng.standard_normal((chi, chi, chi, chi))
        u = rng.standard_normal((chi, chi, chi, chi))
        h = rng.standard_normal((chi, chi, chi, chi))
        h = h + h.transpose(2, 3, 0, 1)  # real symmetric operator
        assert abs(mera.energy(t, w, u, h) - mera.energy_brute(t, w, u, h)) <= 1e-12 * max(1.0, abs(mera.energy_brute(t, w, u, h)))


def test_h_is_the_xxz_bond_operator():
    # one state per charge on charges {0, 1}: h = (S+S- + S-S+)/2 + delta Sz Sz
    # with Sz = diag(0, 1) has eigenvalues {0, -1/2, 1/2, delta}
    delta = 0.8
    leg_o, leg_i = u1.Leg([0, 1], [1, 1], 1), u1.Leg([0, 1], [1, 1], -1)
    H = mera.h_dense([leg_o, leg_o, leg_i, leg_i], lambda *a: synthetic.mera_h_entry(delta, *a))
    M = H.reshape(4, 4)
    assert np.array_equal(M, M.T)
    assert np.allclose(sorted(np.linalg.eigvalsh(M)), sorted([0.0, -0.5, 0.5, delta]), atol=1e-14)


def test_h_conserves_charge_and_is_symmetric_at_full_size():
    spec = synthetic.u1_mera()
    legs = [u1.Leg(*l) for l in spec["h"]]
    H = mera.h_dense(legs, lambda *a: synthetic.mera_h_entry(spec["delta"], *a))
    q = np.concatenate([[qq] * d for qq, d in zip(legs[0].labels, legs[0].degens)])
    chi = len(q)
    assert chi == spec["chi"] == 48
    M = H.reshape(chi * chi, chi * chi)
    assert np.array_equal(M, M.T)
    charge = (q[:, None] + q[None, :]).reshape(-1)
    nz = np.nonzero(M)
    assert np.all(charge[nz[0]] == charge[nz[1]])  # U(1): the total charge is conserved
