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


def test_stems_stay_resident_for_later_requests_of_a_circuit():
    """The second and later requests for a circuit reuse its resident stem
    (leaf tensors and phase-0 intermediates) instead of rebuilding it, also
    while several of them are in flight at once; their amplitudes are
    bit-identical to those of a server that builds the stem afresh, and match
    the state vector."""
    T = tnlib()
    rows, cols, depth, seed, k = 4, 5, 12, 23, 3
    n = rows * cols
    reqs = [dict(rows=rows, cols=cols, depth=depth, seed=seed, num_open=k,
                 bitstrings=I.bitstrings(n, 2, 100 + i)) for i in range(5)]
    kw = dict(max_inflight=4, slices_per_quantum=2, precision="c64", plan_trials=8, max_log2_intermediate=12)
    srv = T.Server(**kw)
    try:
        first, st0 = srv.wait(srv.submit(**reqs[0]))
        assert st0["stem_reused"] == 0
        tickets = [srv.submit(**r) for r in reqs[1:]]
        shared = []
        for t in tickets:
            o, st = srv.wait(t)
            assert st["stem_reused"] == 1 and st["planned_here"] == 0
            shared.append(o)
    finally:
        srv.close()
    fresh = []
    for r in reqs[1:]:
        srv = T.Server(**kw)
        try:
            o, st = srv.wait(srv.submit(**r))
            assert st["stem_reused"] == 0
            fresh.append(o)
        finally:
            srv.close()
    for a, b in zip(shared, fresh):
        assert np.array_equal(a, b)
    gates = OC.random_circuit(rows, cols, depth, seed)
    psi = SV.simulate(gates, n)
    open_q = tuple(range(n - k, n))
    for r, o in zip(reqs, [first] + shared):
        ref = SV.amplitudes(psi, n, [I.bits_of(w, n) for w in r["bitstrings"]], open_q)
        assert np.linalg.norm(o - ref) <= 1e-5 * np.linalg.norm(ref)
