"""GPU parity of the blockwise symmetric eigendecomposition
(include/symtensor.h, sym_eig_*) against the FP64 oracle (oracle/eig.py).

What is unique is compared element by element: the eigenvalues (each
block's, ordered by |lambda|), the truncation counts (integer decisions each
side takes on its own FP64 values) and the truncated product
U diag(lambda) V.  Eigenvectors are unique up to signs (and rotations inside
degenerate eigenvalues), so for them the test checks what makes them valid:
U is an isometry densely and M U = U diag(lambda) for the dense matrix M.
Tolerance: 1e-12 relative to the largest |lambda| (FP64 on both sides; the
shifted Jacobi's eigenvalues carry a few ulp of the block's Frobenius norm).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import eig as oeig  # noqa: E402
from oracle import su2 as osu2  # noqa: E402
from oracle import svd as osvd  # noqa: E402
from oracle import u1 as ou1  # noqa: E402
from oracle import z2f as oz2f  # noqa: E402

TOL = 1e-12


def _P():
    import paper_1203_2222_gb300 as P
    return P


def _mods(group):
    P = _P()
    return {"u1": (P.U1, ou1), "z2f": (P.Z2F, oz2f), "su2": (P.SU2, osu2)}[group]


def _otot(group):
    return osu2.left_comb(2) if group == "su2" else 0


def _sym_values(group, legs, nrow, seed, psd=False):
    """Blocks of a random symmetric tensor (the symmetric part of a random
    invariant operator; psd: X X^T), built by the oracle on the host."""
    _, m = _mods(group)
    ol = [m.Leg(*l) for l in legs]
    n = m.layout(ol, _otot(group))[2]
    d = m.embed(ol, _otot(group), np.random.default_rng(seed).standard_normal(n))
    r = int(np.prod(d.shape[:nrow]))
    M = d.reshape(r, -1)
    M = M @ M.T if psd else 0.5 * (M + M.T)
    vals, resid = m.extract(ol, _otot(group), M.reshape(d.shape))
    assert resid < 1e-12
    return vals


def _dense_bond(group, X, first_is_bond):
    _, m = _mods(group)
    legs = [m.Leg(*l) for l in X.structure.legs]
    d = m.embed(legs, _otot(group) if group == "su2" else X.structure.total, X.data.cpu().numpy())
    return d.reshape(d.shape[0], -1) if first_is_bond else d.reshape(-1, d.shape[-1])


def _check(group, legs, nrow, values, chi=None, cutoff=0.0):
    P = _P()
    g, m = _mods(group)
    S = P.Structure(g, legs)
    T = P.SymTensor(S, torch.as_tensor(values, dtype=torch.float64).cuda())
    To = ([m.Leg(*l) for l in legs], _otot(group), np.asarray(values, dtype=np.float64))
    plan = P.eig_plan(S, nrow)
    lam = plan.execute(T.data).cpu().numpy()
    fac, _ = oeig.eig(group, To, nrow)
    lmax = max(float(np.max(np.abs(f[1]))) for f in fac.values())
    off = 0
    for x, (_, lo, _) in sorted(fac.items()):
        got = lam[off:off + len(lo)]
        off += len(lo)
        assert np.all(np.diff(np.abs(got)) <= TOL * lmax), x  # |lambda| descending
        assert np.max(np.abs(np.sort(got) - np.sort(lo))) <= TOL * lmax, x
    assert off == len(lam) == plan.nsv
    sweeps, _ = plan.stats()
    assert max(sweeps) < 64
    keep = plan.truncation(lam, chi, cutoff)
    ko = oeig.truncation({x: fac[x][1] for x in fac}, chi, cutoff, group=group)
    assert keep == [ko[x] for x in plan.labels]
    M = osvd.matrix(group, To, nrow)
    Uo, kept, Vo = oeig.factors(group, To, nrow, ko, absorb=1, fac=fac)
    Ud, Vd = m.embed(*Uo), m.embed(*Vo)
    ref = Ud.reshape(-1, Ud.shape[-1]) @ Vd.reshape(Vd.shape[0], -1)
    for absorb in (0, 1, 2):
        U, Lk, V = P.eig(T, nrow, chi=chi, cutoff=cutoff, absorb=absorb)
        Lk = Lk.cpu().numpy()
        assert np.max(np.abs(np.sort(Lk) - np.sort(np.concatenate([kept[x] for x in sorted(kept)])))) <= TOL * lmax
        Um, Vm = _dense_bond(group, U, False), _dense_bond(group, V, True)
        ld = osvd.dense_values(group, {x: Lk[o:o + k] for x, k, o in zip(
            [x for x, k in zip(plan.labels, keep) if k], [k for k in keep if k],
            np.cumsum([0] + [k for k in keep if k])[:-1])})
        prod = Um @ (np.diag(ld) if absorb == 0 else np.eye(len(ld))) @ Vm
        assert np.max(np.abs(prod - ref)) <= TOL * lmax
        if absorb == 0:
            assert np.max(np.abs(Um.T @ Um - np.eye(len(ld)))) <= TOL
            assert np.max(np.abs(M @ Um - Um * ld[None, :])) <= TOL * lmax
    if chi is None and not cutoff:
        assert np.max(np.abs(ref - M)) <= TOL * lmax
    P.device_status()
    return plan


def _u1_op(D, seed):
    rng = np.random.default_rng(seed)
    qs = list(range(-3, 4))
    d = [int(x) for x in rng.integers(1, D, len(qs))]
    return qs, d


def test_u1_rank2_operator():
    qs, d = _u1_op(40, 1)
    legs = [(qs, d, -1), (qs, d, 1)]
    _check("u1", legs, 1, _sym_values("u1", legs, 1, 2))
    _check("u1", legs, 1, _sym_values("u1", legs, 1, 3), chi=50)


def test_u1_rank4_operator_with_multi_warp_blocks():
    # fused blocks of up to a few hundred rows: several lanes' rows per column
    a = ([-1, 0, 1], [9, 14, 6], -1)
    b = ([0, 1, 2], [7, 11, 5], 1)
    legs = [a, b, (a[0], a[1], 1), (b[0], b[1], -1)]
    _check("u1", legs, 2, _sym_values("u1", legs, 2, 4))
    _check("u1", legs, 2, _sym_values("u1", legs, 2, 5, psd=True), cutoff=1e-3)


def test_z2f_rank4_operator():
    a = ([0, 1], [13, 9], 1)
    b = ([0, 1], [4, 7], -1)
    legs = [a, b, (a[0], a[1], -1), (b[0], b[1], 1)]
    _check("z2f", legs, 2, _sym_values("z2f", legs, 2, 6))
    _check("z2f", legs, 2, _sym_values("z2f", legs, 2, 7), chi=40)


@pytest.mark.parametrize("dirs", [-1, 1], ids=["in_out", "out_in"])
def test_su2_rank2_operator(dirs):
    sp = [0, 1, 2, 3, 4]
    d = [12, 9, 15, 6, 4]
    legs = [(sp, d, dirs), (sp, d, -dirs)]
    _check("su2", legs, 1, _sym_values("su2", legs, 1, 8))
    _check("su2", legs, 1, _sym_values("su2", legs, 1, 9), chi=60)


def test_degenerate_and_zero_blocks():
    # a block that is exactly zero (every eigenvalue 0) and one proportional
    # to the identity (one eigenvalue, fully degenerate) next to a random one
    qs = [-1, 0, 1]
    d = [5, 8, 6]
    legs = [(qs, d, -1), (qs, d, 1)]
    v = _sym_values("u1", legs, 1, 10)
    v[:25] = 0.0                   # charge -1: 5 x 5 zero block
    v[25:89] = np.eye(8).ravel() * 2.5  # charge 0: 2.5 I
    _check("u1", legs, 1, v)


def test_non_square_structures_are_refused():
    P = _P()
    from paper_1203_2222_gb300 import _lib as L
    qs = [0, 1]
    S = P.Structure(P.U1, [(qs, [2, 3], -1), (qs, [2, 2], 1)])
    with pytest.raises(P.SymError):
        P.eig_plan(S, 1)
    S = P.Structure(P.U1, [(qs, [2, 3], -1), (qs, [2, 3], 1)], total=1)
    with pytest.raises(P.SymError):
        P.eig_plan(S, 1)
    S = P.Structure(P.U1, [(qs, [2, 3], -1), (qs, [2, 3], 1)])
    plan = P.svd_plan(S, 1)  # an SVD plan does not run as an eigendecomposition
    x = torch.zeros(S.numel, dtype=torch.float64, device="cuda")
    lam = torch.zeros(plan.nsv, dtype=torch.float64, device="cuda")
    import ctypes
    rc = L.lib.sym_eig_execute(plan._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(lam.data_ptr()), None)
    assert rc == L.SYM_ERR_ARG
