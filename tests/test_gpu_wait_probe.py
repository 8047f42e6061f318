"""Failure detection on the GPU without a fault: one bounded device-side
wait that nothing completes expires after its limit, sets a device error word
(the library's, or the no-allocation entry point's static one), and
sym_device_status reports SYM_ERR_TIMEOUT once and then clears it; the
context stays usable for a tensor-core contraction checked against the
oracle."""
import time

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_expired_wait_is_reported_once_and_the_context_stays_usable():
    from paper_1203_2222_gb300 import _lib as L
    lib = L.lib
    assert lib.sym_device_status() == L.SYM_OK  # nothing pending before the probe
    for word in (0, 1):
        t0 = time.perf_counter()
        assert lib.sym_wait_probe(20000, word) == L.SYM_OK
        assert time.perf_counter() - t0 >= 0.02  # the wait ran to its 20 ms limit
        assert lib.sym_device_status() == L.SYM_ERR_TIMEOUT, word
        assert b"bounded device-side wait" in lib.sym_last_error()
        assert lib.sym_device_status() == L.SYM_OK  # read once, then cleared
    assert lib.sym_wait_probe(0, 0) == L.SYM_ERR_ARG
    assert lib.sym_wait_probe(2000001, 0) == L.SYM_ERR_ARG
    assert lib.sym_wait_probe(10, 2) == L.SYM_ERR_ARG
    # a contraction whose sectors span several tensor-core tiles, after the expiry
    from tests.test_gpu_parity import _contract_case
    qs = [-1, 0, 1]
    la = [(qs, [70, 150, 33], -1), (qs, [5, 9, 2], 1), (qs, [90, 140, 61], 1)]
    lb = [(qs, [90, 140, 61], -1), (qs, [100, 131, 7], 1)]
    assert _contract_case("u1", la, lb, [2], [0], torch.float32) <= 2e-5
    assert lib.sym_device_status() == L.SYM_OK
