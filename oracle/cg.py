"""SU(2) coupling coefficients in FP64 (oracle; test infrastructure only).

All spins and projections are passed doubled (``j2 = 2j``, ``m2 = 2m``) so
that half-integers stay exact integers.

* ``cg``        Clebsch-Gordan coefficient <ja ma; jb mb | jc mc> of Ch. 5,
                Eq. cg (basis change from the product to the coupled basis),
                evaluated with Racah's closed single-sum formula in exact
                rational arithmetic (Condon-Shortley phase, which reproduces
                the spin-1/2 values printed in Ch. 5, Example 6).
* ``cg_tensor`` the same as an array C[ia, ib, ic] with m = -j + i, i.e. the
                projections in ascending order as in the spin basis of Ch. 5,
                Examples 2-3.
* ``recoupling_F``  the recoupling coefficient F^{jD jE}_{jA jB jC J} of Ch. 5,
                Eq. f, computed by explicit contraction of four CG tensors.
                Reading: the printed Eq. f repeats C_{D,C->ABC} in its second
                line; the fourth factor is taken to be C_{A,E->ABC}, the only
                choice that makes F the overlap of the two coupled bases of
                Eq. fmove (Q' of Eq. cob2 against Q of Eq. cob1).
* ``sixj_from_F``   F divided by the prefactor alpha of Eq. sixj, i.e. the
                Wigner 6j symbol as the paper relates it to F.
* ``omega``     the singlet matrix omega_j of Eq. singletomega.
* ``generators``  J_z, J_+, J_- of a spin-j irrep (Ch. 5, Eq. irrepladder).
"""
from fractions import Fraction
from functools import lru_cache
from math import factorial, sqrt

import numpy as np


def triangle(ja2, jb2, jc2):
    """Fusion rule of Ch. 5, Eq. fusionrules: |ja-jb| <= jc <= ja+jb, integer sum."""
    return (abs(ja2 - jb2) <= jc2 <= ja2 + jb2) and ((ja2 + jb2 + jc2) % 2 == 0)


@lru_cache(maxsize=None)
def cg(ja2, ma2, jb2, mb2, jc2, mc2):
    """<ja ma; jb mb | jc mc> by Racah's formula (doubled arguments)."""
    if not triangle(ja2, jb2, jc2):
        return 0.0
    if ma2 + mb2 != mc2:
        return 0.0
    for j2, m2 in ((ja2, ma2), (jb2, mb2), (jc2, mc2)):
        if abs(m2) > j2 or (j2 - m2) % 2:
            return 0.0
    # integer arguments of the factorials
    a_p_b_m_c = (ja2 + jb2 - jc2) // 2
    a_m_b_p_c = (ja2 - jb2 + jc2) // 2
    mb_pa_pc = (-ja2 + jb2 + jc2) // 2
    a_b_c_1 = (ja2 + jb2 + jc2) // 2 + 1
    ja_pm, ja_mm = (ja2 + ma2) // 2, (ja2 - ma2) // 2
    jb_pm, jb_mm = (jb2 + mb2) // 2, (jb2 - mb2) // 2
    jc_pm, jc_mm = (jc2 + mc2) // 2, (jc2 - mc2) // 2
    pref = Fraction((jc2 + 1) * factorial(a_p_b_m_c) * factorial(a_m_b_p_c)
                    * factorial(mb_pa_pc), factorial(a_b_c_1))
    pref *= (factorial(ja_pm) * factorial(ja_mm) * factorial(jb_pm)
             * factorial(jb_mm) * factorial(jc_pm) * factorial(jc_mm))
    s = Fraction(0)
    k = 0
    while True:
        d = [k, a_p_b_m_c - k, ja_mm - k, jb_pm - k,
             (jc2 - jb2 + ma2) // 2 + k, (jc2 - ja2 - mb2) // 2 + k]
        if d[1] < 0 or d[2] < 0 or d[3] < 0:
            break
        if d[4] >= 0 and d[5] >= 0:
            den = 1
            for x in d:
                den *= factorial(x)
            s += Fraction((-1) ** k, den)
        k += 1
    if s == 0:
        return 0.0
    sign = 1.0 if s > 0 else -1.0
    return sign * sqrt(float(s * s * pref))


@lru_cache(maxsize=None)
def cg_tensor(ja2, jb2, jc2):
    """C[ia, ib, ic] = <ja ma; jb mb | jc mc>, m = -j + i (ascending)."""
    c = np.zeros((ja2 + 1, jb2 + 1, jc2 + 1))
    for ia in range(ja2 + 1):
        for ib in range(jb2 + 1):
            ic2 = (-ja2 + 2 * ia) + (-jb2 + 2 * ib)  # doubled mc
            ic = (ic2 + jc2) // 2
            if abs(ic2) <= jc2 and (ic2 + jc2) % 2 == 0:
                c[ia, ib, ic] = cg(ja2, -ja2 + 2 * ia, jb2, -jb2 + 2 * ib, jc2, ic2)
    c.setflags(write=False)
    return c


def recoupling_F(jd2, je2, ja2, jb2, jc2, J2):
    """F^{jD jE}_{jA jB jC J} of Ch. 5, Eq. f (reading: 4th factor C_{A,E->J}).

    F = 1/(2J+1) * sum over all m of
        C_{A,B->D} C_{D,C->J} C_{B,C->E} C_{A,E->J}.
    Returns 0 when any of the four couplings is forbidden.
    """
    if not (triangle(ja2, jb2, jd2) and triangle(jd2, jc2, J2)
            and triangle(jb2, jc2, je2) and triangle(ja2, je2, J2)):
        return 0.0
    c_abd = cg_tensor(ja2, jb2, jd2)
    c_dcj = cg_tensor(jd2, jc2, J2)
    c_bce = cg_tensor(jb2, jc2, je2)
    c_aej = cg_tensor(ja2, je2, J2)
    # indices: a b c d e M
    val = np.einsum('abd,dcM,bce,aeM->', c_abd, c_dcj, c_bce, c_aej)
    return float(val) / (J2 + 1)


def sixj_from_F(ja2, jb2, jd2, jc2, J2, je2):
    """{ja jb jd; jc J je} = F^{jd je}_{ja jb jc J} / alpha (Ch. 5, Eq. sixj).

    alpha = (-1)^(ja+jb+jc+J) sqrt((2jd+1)(2je+1)).
    """
    ph2 = ja2 + jb2 + jc2 + J2
    if ph2 % 2:
        return 0.0
    alpha = (-1) ** (ph2 // 2) * sqrt((jd2 + 1) * (je2 + 1))
    return recoupling_F(jd2, je2, ja2, jb2, jc2, J2) / alpha


def omega(j2):
    """omega_j of Ch. 5, Eq. singletomega: (omega)_{m,-m} = (-1)^(j-m)/sqrt(2j+1)."""
    w = np.zeros((j2 + 1, j2 + 1))
    for i in range(j2 + 1):
        m2 = -j2 + 2 * i
        w[i, j2 - i] = (-1) ** ((j2 - m2) // 2) / sqrt(j2 + 1)
    return w


def cup(j2):
    """cup_j = sqrt(2j+1) omega_j (Ch. 5, Eq. cupj)."""
    return sqrt(j2 + 1) * omega(j2)


def cap(j2):
    """cap_j = (-1)^(2j) sqrt(2j+1) omega_j (Ch. 5, Eq. capj)."""
    return (-1) ** j2 * sqrt(j2 + 1) * omega(j2)


def generators(j2):
    """(Jz, J+, J-) of the spin-j irrep in the ascending spin basis.

    Ch. 5, Eq. irrepz and Eq. irrepladder:
    J+- |j m> = sqrt(j(j+1) - m(m+-1)) |j, m+-1>.
    """
    n = j2 + 1
    jz = np.zeros((n, n))
    jp = np.zeros((n, n))
    j = j2 / 2.0
    for i in range(n):
        m = -j + i
        jz[i, i] = m
        if i + 1 < n:
            jp[i + 1, i] = sqrt(j * (j + 1) - m * (m + 1))
    return jz, jp, jp.T.copy()
