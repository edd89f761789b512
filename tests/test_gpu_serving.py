"""Serving (continuous batching): requests for circuits of different grids and
depths are admitted by memory and slots and interleaved slice quantum by
quantum on separate streams; a request's amplitudes must be the same alone and
in the mix, over-cap requests must fail loudly."""
import numpy as np
import pytest

import tn_inputs as I
from oracle import circuit as OC
from oracle import statevector as SV

from _lib import tnlib

pytestmark = pytest.mark.gpu


def _req(rows, cols, depth, seed, k, nb):
    n = rows * cols
    return dict(rows=rows, cols=cols, depth=depth, seed=seed, num_open=k, bitstrings=I.bitstrings(n, nb, seed))


@pytest.mark.parametrize("mode,tol", [("c64", 1e-5), ("split_bf16", 1e-4), ("scaled_fp16", 2e-2)])
def test_alone_equals_in_the_mix(mode, tol):
    T = tnlib()
    target = _req(4, 5, 12, 21, 3, 2)
    srv = T.Server(max_inflight=4, slices_per_quantum=4, precision=mode, plan_trials=8, max_log2_intermediate=12)
    try:
        alone, st = srv.wait(srv.submit(**target))
        assert st["status"] == 0 and st["slices"] >= 2
        others = [_req(4, 4, 10, 30 + i, i % 4, 1 + i % 3) for i in range(6)] + \
                 [_req(5, 4, 14, 40 + i, 2, 2) for i in range(3)]
        tickets = [srv.submit(**r) for r in others[:4]]
        tt = srv.submit(**target)
        tickets += [srv.submit(**r) for r in others[4:]]
        mixed, st2 = srv.wait(tt)
        for t in tickets:
            srv.wait(t)
    finally:
        srv.close()
    assert np.array_equal(alone, mixed)
    gates = OC.random_circuit(4, 5, 12, 21)
    n = 20
    open_q = tuple(range(n - 3, n))
    ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in target["bitstrings"]], open_q)
    assert np.linalg.norm(alone - ref) <= tol * np.linalg.norm(ref)


def test_over_cap_and_over_budget_requests_fail_loudly():
    T = tnlib()
    srv = T.Server(max_inflight=2, precision="c64", plan_trials=4, max_log2_cmac=20.0)
    try:
        with pytest.raises(T.TnError) as e:
            srv.wait(srv.submit(**_req(6, 6, 16, 2, 0, 1)))
        assert e.value.status == 6          # TN_ETOOBIG
        ok, st = srv.wait(srv.submit(**_req(3, 3, 4, 1, 1, 1)))
        assert st["status"] == 0
    finally:
        srv.close()
    srv = T.Server(max_inflight=2, precision="c64", plan_trials=4, hbm_budget_bytes=1 << 20)
    try:
        with pytest.raises(T.TnError) as e:
            srv.wait(srv.submit(**_req(4, 4, 8, 1, 0, 1)))
        assert e.value.status == 3          # TN_EHBM
    finally:
        srv.close()
