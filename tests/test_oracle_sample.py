"""Pins of oracle.sample: single dense elements of a contraction and of its
gradients equal the full dense oracle (contract.contract, contract_grad) at
every index of small SU(2) contractions, with several pair patterns, trees
and directions.  No GPU."""
import itertools

import numpy as np
import pytest

from oracle import contract as oc
from oracle import sample
from oracle import su2


def _case(name):
    rng = np.random.default_rng(hash(name) % 2**32)
    if name == "recouple_pairs_1_3":  # the large-sector workload's pattern at tiny size
        sp = [0, 1, 2]
        dl = [list(rng.integers(1, 3, 3)) for _ in range(6)]
        la = [su2.Leg(sp, dl[l], 1) for l in range(4)]
        lb = [su2.Leg(sp, dl[1], -1), su2.Leg(sp, dl[3], -1), su2.Leg(sp, dl[4], 1), su2.Leg([1], [2], 1)]
        return la, su2.left_comb(4), lb, su2.left_comb(4), [1, 3], [0, 1]
    if name == "reversed_pairs_mixed_dirs":  # pairs out of order, incoming free legs, non-comb tree
        la = [su2.Leg([0, 1], [2, 1], -1), su2.Leg([1, 2], [1, 2], 1), su2.Leg([0, 1, 2], [1, 1, 1], 1)]
        lb = [su2.Leg([0, 1, 2], [1, 1, 1], -1), su2.Leg([1], [2], 1), su2.Leg([1, 2], [1, 2], -1)]
        return la, su2.left_comb(3), lb, [(1, 2), (0, 3)], [2, 1], [0, 2]
    raise KeyError(name)


@pytest.mark.parametrize("name", ["recouple_pairs_1_3", "reversed_pairs_mixed_dirs"])
def test_sampled_elements_equal_the_dense_oracle(name):
    la, ta, lb, tb, pa, pb = _case(name)
    rng = np.random.default_rng(1)
    a = rng.standard_normal(su2.layout(la, ta)[2])
    b = rng.standard_normal(su2.layout(lb, tb)[2])
    lc, tc, c, resid = oc.contract("su2", (la, ta, a), (lb, tb, b), pa, pb)
    assert resid < 1e-12
    g = rng.standard_normal(len(c))
    da, db, r2 = oc.contract_grad("su2", (la, ta, a), (lb, tb, b), pa, pb, g)
    assert r2 < 1e-12
    Cd, dAd, dBd = su2.embed(lc, tc, c), su2.embed(la, ta, da), su2.embed(lb, tb, db)
    A, B, G = (la, ta, a), (lb, tb, b), (lc, tc, g)
    for idx in itertools.product(*[range(n) for n in Cd.shape]):
        assert abs(sample.contraction_element(su2, A, B, pa, pb, idx) - Cd[idx]) < 1e-12
        assert abs(sample.element(su2, (lc, tc, c), idx) - Cd[idx]) < 1e-12
    for idx in itertools.product(*[range(n) for n in dAd.shape]):
        assert abs(sample.grad_a_element(su2, A, B, pa, pb, G, idx) - dAd[idx]) < 1e-12
    for idx in itertools.product(*[range(n) for n in dBd.shape]):
        assert abs(sample.grad_b_element(su2, A, B, pa, pb, G, idx) - dBd[idx]) < 1e-12
    # the pins are not vacuous: a planted sign error in one block is caught
    bad = c.copy()
    bad[0] = -bad[0] if bad[0] != 0 else 1.0
    assert any(abs(sample.element(su2, (lc, tc, bad), idx) - Cd[idx]) > 1e-9
               for idx in itertools.product(*[range(n) for n in Cd.shape]))


def test_drawn_indices_avoid_structural_zeros():
    """Indices drawn with J_z conserved land on nonzero elements of a random
    invariant tensor, while the dense tensor vanishes wherever J_z is not
    conserved (so a uniform draw would mostly compare zero with zero)."""
    la, ta, _, _, _, _ = _case("reversed_pairs_mixed_dirs")
    rng = np.random.default_rng(2)
    a = rng.standard_normal(su2.layout(la, ta)[2])
    Ad = su2.embed(la, ta, a)
    idxs = sample.draw_indices(su2, la, ta, rng, 200)
    assert np.mean([abs(Ad[tuple(i)]) > 1e-12 for i in idxs]) > 0.9
    mvals = [np.concatenate([np.tile(np.arange(-j, j + 1, 2), d) for j, d in zip(l.labels, l.degens)]) for l in la]
    tot = sum(l.dir * mv.reshape([-1 if k == i else 1 for k in range(len(la))]) for i, (l, mv) in enumerate(zip(la, mvals)))
    assert np.all(Ad[tot != 0] == 0) and np.count_nonzero(tot != 0) > 0
