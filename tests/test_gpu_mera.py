"""MERA-patch energy and its gradient through the library, against the FP64 oracle.

E = <psi|h|psi>/<psi|psi> for psi = (1 x 1 x u x 1 x 1)(w x w) t at the full
bond dimension chi = 48 (U(1), charges -4..4) is contracted block-sparsely
by paper_1203_2222_gb300.networks and densely by oracle.mera; the gradients
with respect to u and w (autograd through the library's adjoint) are checked
against central finite differences of the oracle's energy along random
symmetric directions, and the checkpointed environment must give the same
gradient as the stored one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _setup(dtype):
    import paper_1203_2222_gb300 as P
    from paper_1203_2222_gb300 import networks, synthetic
    spec = synthetic.u1_mera()
    S = networks.mera_structures(spec)
    h, one = networks.mera_h_and_identity(S, spec)
    d = {}
    for n in ("t", "w", "u"):
        x = synthetic.normal(spec["seeds"][n], S[n].numel)
        d[n] = torch.as_tensor(x / np.sqrt(spec["chi"])).to(dtype).cuda()  # O(1) contractions
    d["h"] = torch.as_tensor(h).to(dtype).cuda()
    d["1"] = torch.as_tensor(one).to(dtype).cuda()
    return P, networks, spec, S, d


def _oracle_energy(spec, S, host):
    from oracle import mera, u1
    from paper_1203_2222_gb300 import synthetic
    legs = {n: [u1.Leg(*l) for l in spec[n]] for n in ("t", "w", "u", "h")}
    dense = {n: u1.embed(legs[n], 0, host[n]) for n in ("t", "w", "u")}
    H = mera.h_dense(legs["h"], lambda *a: synthetic.mera_h_entry(spec["delta"], *a))
    return mera.energy(dense["t"], dense["w"], dense["u"], H)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)], ids=["float64", "float32"])
def test_mera_energy_against_oracle(dtype, tol):
    P, networks, spec, S, d = _setup(dtype)
    E = float(networks.mera_energy(S, d["t"], d["w"], d["u"], d["h"], d["1"]))
    host = {n: d[n].double().cpu().numpy() for n in ("t", "w", "u")}
    E_ref = _oracle_energy(spec, S, host)
    assert abs(E - E_ref) <= tol * abs(E_ref), (E, E_ref)
    P.device_status()


def test_mera_gradients_against_oracle_finite_differences():
    P, networks, spec, S, d = _setup(torch.float64)
    u = d["u"].clone().requires_grad_(True)
    w = d["w"].clone().requires_grad_(True)
    E = networks.mera_energy(S, d["t"], w, u, d["h"], d["1"])
    gu, gw = torch.autograd.grad(E, [u, w])
    # the checkpointed environment recomputes rho in the backward: same gradient
    u2 = d["u"].clone().requires_grad_(True)
    w2 = d["w"].clone().requires_grad_(True)
    E2 = networks.mera_energy(S, d["t"], w2, u2, d["h"], d["1"], checkpoint=True)
    gu2, gw2 = torch.autograd.grad(E2, [u2, w2])
    assert torch.allclose(gu, gu2, rtol=1e-12, atol=1e-15) and torch.allclose(gw, gw2, rtol=1e-12, atol=1e-15)
    host = {n: d[n].double().cpu().numpy() for n in ("t", "w", "u")}
    rng = np.random.default_rng(9)
    eps = 1e-5
    for name, g in (("u", gu), ("w", gw)):
        delta = rng.standard_normal(S[name].numel)
        delta /= np.linalg.norm(delta)
        plus, minus = dict(host), dict(host)
        plus[name] = host[name] + eps * delta
        minus[name] = host[name] - eps * delta
        fd = (_oracle_energy(spec, S, plus) - _oracle_energy(spec, S, minus)) / (2 * eps)
        an = float(np.dot(g.cpu().numpy(), delta))
        assert abs(an - fd) <= 1e-6 * max(abs(fd), np.linalg.norm(g.cpu().numpy())), (name, an, fd)
    P.device_status()


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-6), (torch.float32, 2e-5)], ids=["float64", "float32"])
def test_mera_gradients_of_every_tensor_against_oracle_fd(dtype, tol):
    """The gradient with respect to t, w and u (split-BF16 x3 and FP64, the
    environment checkpointed as the bench runs it) against FP64 central
    finite differences of the oracle's dense energy along several directions
    per tensor: the gradient's own direction (so the check sees its norm)
    and three random unit directions.  The error bar is relative to the
    gradient's norm: a gradient with relative error r misses any unit
    directional derivative by at most r |g|."""
    P, networks, spec, S, d = _setup(dtype)
    t = d["t"].clone().requires_grad_(True)
    u = d["u"].clone().requires_grad_(True)
    w = d["w"].clone().requires_grad_(True)
    E = networks.mera_energy(S, t, w, u, d["h"], d["1"], checkpoint=True)
    grads = dict(zip(("t", "w", "u"), (g.double().cpu().numpy() for g in torch.autograd.grad(E, [t, w, u]))))
    torch.cuda.synchronize()
    host = {n: d[n].double().cpu().numpy() for n in ("t", "w", "u")}
    rng = np.random.default_rng(17)
    eps = 1e-5
    for name, g in grads.items():
        gn = np.linalg.norm(g)
        assert gn > 0
        dirs = [g / gn] + [v / np.linalg.norm(v) for v in (rng.standard_normal(S[name].numel) for _ in range(3))]
        for k, delta in enumerate(dirs):
            plus, minus = dict(host), dict(host)
            plus[name] = host[name] + eps * delta
            minus[name] = host[name] - eps * delta
            fd = (_oracle_energy(spec, S, plus) - _oracle_energy(spec, S, minus)) / (2 * eps)
            an = float(np.dot(g, delta))
            assert abs(an - fd) <= tol * gn, (name, k, an, fd, gn)
    P.device_status()
