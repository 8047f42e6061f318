"""The autotuner on the device: a coordinate descent over two planning
parameters on a small MPO step installs its choice, and the contraction
planned under it still matches the FP64 oracle (forward and gradients)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_autotune_installs_its_choice_and_keeps_parity():
    import paper_1203_2222_gb300 as P
    from paper_1203_2222_gb300 import autotune
    import tests.test_gpu_parity as T
    qs = [-2, -1, 0, 1, 2]
    la = [(qs, [7, 19, 33, 21, 5], -1), (*T.MPO, -1), (*T.PHYS, -1), (qs, [6, 17, 40, 23, 9], 1)]
    lb = [(*T.MPO, 1), (*T.PHYS, -1), (*T.PHYS, 1), (*T.MPO, -1)]
    SA, SB = P.Structure(P.U1, la), P.Structure(P.U1, lb)
    a = torch.randn(SA.numel, device="cuda", requires_grad=True)
    b = torch.randn(SB.numel, device="cuda", requires_grad=True)
    g = None

    def step():
        nonlocal g
        C = P.contract(P.SymTensor(SA, a), P.SymTensor(SB, b), [1, 2], [0, 2])
        if g is None:
            g = torch.randn(C.structure.numel, device="cuda")
        torch.autograd.grad(C.data, [a, b], grad_outputs=g)

    start = P.tune_get()
    try:
        params, ms, hist = autotune.tune(step, space={"direct_chunk": [64, 256], "direct_max": [0, 4]},
                                         reps=2, warmup=1, trials=1, rounds=1, starts=())
        assert P.tune_get() == params and ms > 0
        assert len(hist) >= 3 and all(h["ms"] > 0 for h in hist)
        assert params["direct_chunk"] in (64, 256, start["direct_chunk"])
        for dtype in T.DTYPES:  # planned under the chosen parameters
            T._contract_case("u1", la, lb, [1, 2], [0, 2], dtype)
    finally:
        P.tune_set(**start)
