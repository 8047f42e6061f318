"""Pins of the blockwise symmetric eigendecomposition oracle (oracle/eig.py)
against the dense matrix's own eigendecomposition and the mathematics of the
spectral decomposition, independent of the GPU path."""
import numpy as np
import pytest

from oracle import eig, su2, svd, u1, z2f


def _mod(group):
    return {"u1": u1, "z2f": z2f, "su2": su2}[group]


def _tot(group):
    return su2.left_comb(2) if group == "su2" else 0


def _sym_tensor(group, legs, nrow, seed):
    """A random symmetric tensor: the symmetric part of a random invariant
    operator (rows = legs 0..nrow-1), extracted back into blocks."""
    m = _mod(group)
    tot = _tot(group)
    n = m.layout(legs, tot)[2]
    d = m.embed(legs, tot, np.random.default_rng(seed).standard_normal(n))
    r = int(np.prod(d.shape[:nrow]))
    M = d.reshape(r, -1)
    Ms = 0.5 * (M + M.T)
    blocks, resid = m.extract(legs, tot, Ms.reshape(d.shape))
    assert resid < 1e-12
    return (legs, tot, blocks)


def _u1_rank2():
    a = u1.Leg([-2, -1, 0, 1], [2, 3, 4, 1], -1)
    return [a, u1.Leg(a.labels, a.degens, 1)], 1


def _u1_rank4():
    a, b = u1.Leg([-1, 0, 1], [2, 3, 1], -1), u1.Leg([0, 1], [2, 2], 1)
    return [a, b, u1.Leg(a.labels, a.degens, 1), u1.Leg(b.labels, b.degens, -1)], 2


def _z2f_rank4():
    a, b = z2f.Leg([0, 1], [3, 2], 1), z2f.Leg([0, 1], [1, 2], -1)
    return [a, b, z2f.Leg(a.labels, a.degens, -1), z2f.Leg(b.labels, b.degens, 1)], 2


def _su2(dirs):
    def f():
        a = su2.Leg([0, 1, 2, 3], [3, 2, 4, 2], dirs)
        return [a, su2.Leg(a.labels, a.degens, -dirs)], 1
    return f


CASES = [("u1", _u1_rank2), ("u1", _u1_rank4), ("z2f", _z2f_rank4), ("su2", _su2(-1)), ("su2", _su2(1))]
IDS = ["u1_rank2", "u1_rank4", "z2f_rank4", "su2_in_out", "su2_out_in"]


def _dense_values(group, fac, keep=None):
    kept = {x: f[1][:(keep[x] if keep else len(f[1]))] for x, f in fac.items()}
    return svd.dense_values(group, {x: v for x, v in kept.items() if len(v)})


def _bond_matrix(group, U, V):
    m = _mod(group)
    du, dv = m.embed(*U), m.embed(*V)
    return du.reshape(-1, du.shape[-1]), dv.reshape(dv.shape[0], -1)


@pytest.mark.parametrize("group,case", CASES, ids=IDS)
def test_eigenvalues_are_those_of_the_dense_matrix(group, case):
    legs, nrow = case()
    T = _sym_tensor(group, legs, nrow, 3)
    M = svd.matrix(group, T, nrow)
    assert np.allclose(M, M.T, atol=1e-13)
    fac, _ = eig.eig(group, T, nrow)
    ours = np.sort(_dense_values(group, fac))
    dense = np.linalg.eigvalsh(M)
    # the blocks cover the dense matrix (no zero rows outside them here)
    assert len(ours) == len(dense)
    assert np.allclose(ours, dense, rtol=1e-12, atol=1e-12)
    # each block's values come ordered by |lam| descending
    for _, lam, _ in fac.values():
        assert np.all(np.diff(np.abs(lam)) <= 1e-15)


@pytest.mark.parametrize("group,case", CASES, ids=IDS)
def test_factors_rebuild_the_matrix_and_hold_its_eigenvectors(group, case):
    legs, nrow = case()
    T = _sym_tensor(group, legs, nrow, 5)
    M = svd.matrix(group, T, nrow)
    fac, _ = eig.eig(group, T, nrow)
    keep = eig.truncation({x: f[1] for x, f in fac.items()}, group=group)
    U, kept, V = eig.factors(group, T, nrow, keep, fac=fac)
    Um, Vm = _bond_matrix(group, U, V)
    lam = svd.dense_values(group, kept)
    assert np.allclose(Um @ np.diag(lam) @ Vm, M, atol=1e-12)
    # U is an isometry whose columns are eigenvectors of the dense matrix
    assert np.allclose(Um.T @ Um, np.eye(len(lam)), atol=1e-12)
    assert np.allclose(M @ Um, Um * lam[None, :], atol=1e-12)
    # absorbing the values into either factor gives the same product
    for absorb in (1, 2):
        A, _, B = eig.factors(group, T, nrow, keep, absorb=absorb, fac=fac)
        Am, Bm = _bond_matrix(group, A, B)
        assert np.allclose(Am @ Bm, M, atol=1e-12)
    # U and V hold nothing outside their blocks
    m = _mod(group)
    for legsX, tot, d in (U, V):
        assert m.extract(legsX, tot, m.embed(legsX, tot, d))[1] < 1e-12


@pytest.mark.parametrize("group,case", CASES, ids=IDS)
def test_truncation_is_the_best_low_rank_approximation(group, case):
    # Eckart-Young for a symmetric matrix: the best approximation of rank k
    # keeps the k eigenvalues of largest magnitude; the error is the norm of
    # the dropped ones
    legs, nrow = case()
    T = _sym_tensor(group, legs, nrow, 7)
    M = svd.matrix(group, T, nrow)
    dense = np.linalg.eigvalsh(M)
    mags = np.sort(np.abs(dense))[::-1]
    fac, _ = eig.eig(group, T, nrow)
    for chi in (1, 3, 8, 15):
        keep = eig.truncation({x: f[1] for x, f in fac.items()}, chi=chi, group=group)
        n = sum(k * (x + 1 if group == "su2" else 1) for x, k in keep.items())
        assert n <= chi
        if n == 0:  # SU(2): the largest multiplet alone is wider than chi
            continue
        U, kept, V = eig.factors(group, T, nrow, keep, absorb=1, fac=fac)
        Um, Vm = _bond_matrix(group, U, V)
        err = np.linalg.norm(M - Um @ Vm)
        assert err == pytest.approx(np.sqrt(np.sum(mags[n:] ** 2)), rel=1e-10, abs=1e-12)
        if group != "su2":  # no multiplets: exactly chi values kept
            assert n == min(chi, len(dense))


def test_single_charge_is_the_plain_eigendecomposition():
    a = u1.Leg([0], [7], -1)
    legs = [a, u1.Leg([0], [7], 1)]
    T = _sym_tensor("u1", legs, 1, 9)
    M = T[2].reshape(7, 7)
    fac, _ = eig.eig("u1", T, 1)
    lam = fac[0][1]
    ref = np.linalg.eigvalsh(M)
    assert np.allclose(np.sort(lam), ref, atol=1e-13)
    assert np.allclose(fac[0][0] @ np.diag(lam) @ fac[0][2], M, atol=1e-12)


def test_positive_matrix_eigenvalues_are_its_singular_values():
    # a density matrix rho = X X^T: eigenvalues = singular values
    legs, nrow = _u1_rank4()
    T = _sym_tensor("u1", legs, nrow, 11)
    M = svd.matrix("u1", T, nrow)
    m = u1
    rho = (M @ M.T).reshape(m.embed(*T).shape)
    blocks, resid = m.extract(legs, 0, rho)
    assert resid < 1e-12
    fac, _ = eig.eig("u1", (legs, 0, blocks), nrow)
    sfac, _ = svd.svd("u1", (legs, 0, blocks), nrow)
    for x in fac:
        assert np.all(fac[x][1] >= -1e-12)
        assert np.allclose(fac[x][1], sfac[x][1], atol=1e-11)


def test_non_square_structures_are_refused():
    a = u1.Leg([0, 1], [2, 3], -1)
    with pytest.raises(ValueError):
        eig.eig("u1", ([a, u1.Leg([0, 1], [2, 2], 1)], 0, np.zeros(8)), 1)
    with pytest.raises(ValueError):
        eig.eig("u1", ([a, u1.Leg([0, 1], [2, 3], -1)], 0, np.zeros(13)), 1)
    with pytest.raises(ValueError):
        eig.eig("u1", ([a, u1.Leg([0, 1], [2, 3], 1)], 1, np.zeros(6)), 1)
